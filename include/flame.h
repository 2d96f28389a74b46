/*
 * flame.h -- C ABI of the GB300 implementation of one fused lattice-Boltzmann
 * time step for 3-D periodic Hall-MHD (the FLAME scheme of Foldes et al.,
 * arXiv 2212.11024: D3Q27 central-moment fluid, Sec. 3.1, plus three D3Q7 BGK
 * magnetic populations with the Hall term in their equilibrium, Sec. 3.2).
 *
 * Problem statement (Sec. 3.3, 4.1, 5): given a periodic nx x ny x nz lattice,
 * the lattice viscosity and resistivity (through the relaxation times), the
 * Hall length d_i and initial rho, u, B, advance n time steps and return u,
 * B, J, energies and spectra.  Everything is in lattice units
 * (dx = dt = 1, c_s^2 = 1/3, C^2 = 1/4, alpha_H = d_i).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers, h_* host pointers.  The caller
 *    owns all of them, including the population state; the library never
 *    frees caller memory.  The library owns the context and, after the first
 *    flame_reduce / flame_spectra call, an internal device workspace that
 *    flame_destroy releases.
 *  - Work is queued asynchronously on the stream given to flame_create.
 *    Calls that return host data (flame_reduce, flame_spectra, flame_sync,
 *    flame_init) synchronise that stream.
 *  - Errors are returned as flame_status; nothing throws across the ABI.  A
 *    CUDA error, or a non-finite value seen by the step kernel, is sticky:
 *    every later call on the context returns it.  Asynchronous CUDA errors
 *    surface at the next synchronising call.
 *  - Fields are structure-of-arrays [component][z][y][x], x fastest, with
 *    N3 = nx*ny*nz sites per component.  Gradients are [3a+b][z][y][x] for
 *    d_a F_b.
 *  - A z-slab context (flame_params.halo_z = 1) of nz planes takes its
 *    initial fields (flame_init) on nz + 2 planes -- one plane of the
 *    neighbouring slabs' fields below and above, for the z-derivatives --
 *    and writes every per-site output (moments, populations, probe,
 *    reductions) for its own nz planes, N3 = nx*ny*nz sites.
 *
 * Populations are numbered in natural slot order: q = 0..26 the fluid
 * population on App. A's D3Q27 velocity q, q = 27 + 7b + i the magnetic
 * component b (x, y, z) on D3Q7 velocity i (rest, +x, -x, +y, -y, +z, -z).
 * flame_populations and the adjoint vectors use this order.
 *
 * Population state (flame_state_bytes bytes, 256-byte aligned; opaque to
 * callers, who move it only with flame_get_state / flame_set_state): 48
 * storage slots of N3 values.  Storage slot (cx+1) + 3(cy+1) + 9(cz+1) holds
 * the fluid population on velocity (cx, cy, cz), storage slot 27 + 3i + b
 * the magnetic component b on D3Q7 velocity i; this order makes the rows an
 * odd AA step reads into a few runs of consecutive slots.  The state is
 * updated in place with the AA access pattern, so which site and slot hold a
 * given population depends on the step parity (flame_info).  A slot stores
 * the population's deviation from the rest equilibrium of the reference
 * state (rho0, B_ref) divided by its lattice weight, as FP32, FP16 or BF16
 * (round to nearest even).
 */
#ifndef FLAME_H
#define FLAME_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FLAME_OK = 0,
    FLAME_ERR_PARAM = 1,     /* invalid argument or parameter                          */
    FLAME_ERR_CFL = 2,       /* whistler CFL violated and strict_cfl set (flame_init)   */
    FLAME_ERR_NONFINITE = 3, /* a non-finite density, velocity or field was produced   */
    FLAME_ERR_CUDA = 4,      /* a CUDA runtime or cuFFT call failed                     */
    FLAME_ERR_STATE = 5,     /* state blob or call order inconsistent                   */
    FLAME_ERR_TIMEOUT = 6    /* a device-side wait (a staged copy of the row kernel)
                                exceeded its limit; the step was not completed          */
} flame_status;

typedef enum { FLAME_FP32 = 1, FLAME_FP16 = 2, FLAME_BF16 = 3 } flame_storage;

/* Collision scheme.  FLAME_SCHEME is the paper's (central-moment fluid,
 * Sec. 3.1.2; Hall BGK magnetic with the current from the magnetic
 * moments, Sec. 3.2).  The others are the variants the paper names:
 * FLAME_BGK_FLUID  fluid collision f* = f - omega (f - f^mhd(0)) (Sec. 3.1.1);
 * FLAME_EMHD       electron MHD: U neglected against alpha_H J in the
 *                  magnetic equilibrium (end of Sec. 5);
 * FLAME_FD_CURRENT J from the second-order central-difference curl of the
 *                  pre-collision B (one extra pass writing B per step; the
 *                  paper contrasts this with its moment-based current). */
typedef enum { FLAME_SCHEME = 0, FLAME_BGK_FLUID = 1, FLAME_EMHD = 2, FLAME_FD_CURRENT = 3 } flame_variant;

typedef struct {
    int nx, ny, nz;   /* lattice size, each >= 1                                          */
    double tau_nu;    /* fluid relaxation time 1/omega = nu/c_s^2 + 1/2 > 1/2 (Sec. 3.1.1) */
    double tau_eta;   /* magnetic relaxation time 1/omega_B = eta/C^2 + 1/2 > 1/2 (Sec. 3.2) */
    double d_i;       /* Hall coefficient alpha_H, the ion inertial length in lattice
                         units (Sec. 3.3 with U_0 = V_A, rho = 1); 0 gives resistive MHD   */
    int storage;      /* flame_storage                                                    */
    double rho0;      /* reference density of the deviation encoding (> 0, normally 1)   */
    double B_ref[3];  /* reference field of the deviation encoding (normally the mean
                         field, which the scheme conserves exactly)                       */
    int init_noneq;   /* 1: flame_init adds the first-order non-equilibrium parts        */
    int check_every;  /* > 0: flame_step synchronises and checks the non-finite flag
                         every check_every steps; 0: only flame_sync checks               */
    int strict_cfl;   /* 1: flame_init fails with FLAME_ERR_CFL if pi d_i max(V_A,|u|) > 1 */
    int graph_steps;  /* 0: one kernel launch per step; even G > 0: flame_step replays a
                         captured CUDA graph of G steps for each whole chunk of G steps
                         (removes launch overhead on small lattices); flame_create
                         captures the graph that starts at parity 0                      */
    int variant;      /* flame_variant (FLAME_SCHEME = 0 by default); the adjoint
                         entry points support FLAME_SCHEME only                          */
    int kernel;       /* 0: automatic -- FP16/BF16 storage (any variant) with nx even
                         uses the row kernel (two sites per thread in packed FP32
                         pairs), in the tiling timed fastest for the row length: x rows
                         staged in shared memory by TMA, a whole row per block tile
                         (most lengths that are multiples of 8 from 64 to 1024) or half a
                         row (608, 624, 640), or unstaged pairs loaded and stored
                         straight from HBM (every other even length); odd nx and FP32
                         storage use the one-site kernel; 1: always the one-site kernel;
                         2: staged whole rows (nx a multiple of 8 in 64..1024), 3: staged
                         half rows (nx > 256 a multiple of 16), 4: unstaged pairs (nx
                         even), where they apply, else the one-site kernel.  All compute the same step in FP32; results
                         agree to FP32 rounding before encoding (the row kernel's tilings
                         agree bit for bit). */
    int halo_z;       /* 0: a periodic nx x ny x nz lattice.  1: one z-slab of a larger
                         periodic lattice split along z (the one-direction domain split
                         of Sec. 4): the state holds the slab's nz planes between two
                         ghost planes (nz + 2 planes; plane 0 below, nz + 1 above) that
                         carry the neighbouring slabs' boundary populations, z is not
                         wrapped, and the caller exchanges the ghost planes after every
                         step (flame_halo_exchange, or the runs of flame_halo_plan over
                         any transport).  Not with FLAME_FD_CURRENT; the spectral and
                         adjoint entry points refuse slab contexts.                     */
} flame_params;

typedef struct {
    long long step;   /* steps taken since flame_init / flame_set_state             */
    int parity;       /* AA parity: 0 = every slot holds its natural population     */
    int nonfinite;    /* sticky non-finite flag (read at the last synchronising call) */
    double cfl;       /* pi d_i max(V_A, |u|) of the initial fields (Sec. 3.4)       */
    double max_speed; /* max over sites of max(|B|/sqrt(rho), |u|) at flame_init      */
} flame_info_t;

/* Scalar diagnostics written by flame_reduce (indices into h_scalars). */
enum {
    FLAME_S_MASS = 0,       /* sum rho                                          */
    FLAME_S_MOMX = 1,       /* sum rho u_x (2: y, 3: z)                         */
    FLAME_S_BX = 4,         /* <B_x> (5: y, 6: z)                               */
    FLAME_S_EU = 7,         /* 1/2 <|u|^2>                                      */
    FLAME_S_EB = 8,         /* 1/2 <|B - <B>|^2>                                */
    FLAME_S_HC = 9,         /* <u . (B - <B>)>, cross-helicity                   */
    FLAME_S_J2 = 10,        /* <|J|^2>; eta <|J|^2> is the magnetic dissipation  */
    FLAME_S_UMAX = 11,      /* max |u|                                          */
    FLAME_S_DIVB = 12,      /* rms of -(omega_B/C^2) Tr(Lambda), eq. LB_B_div     */
    FLAME_S_NONFINITE = 13, /* number of sites with a non-finite moment         */
    FLAME_NSCALARS = 14
};

typedef struct flame_ctx flame_ctx;

/* Bytes of the population state: 48 * N3 * (4 for FP32, 2 for FP16/BF16),
 * with N3 = nx * ny * (nz + 2 halo_z).
 * graph_steps must be 0 or a positive even number. 
 * Returns 0 for invalid parameters. */
size_t flame_state_bytes(const flame_params *p);

/* Create a context over caller-owned device state d_state (flame_state_bytes,
 * 256-byte aligned) and a cudaStream_t `stream` (NULL: legacy default
 * stream).  Checks: sizes >= 1, ny and nz <= 65535, N3 < 2^31, tau > 1/2, rho0 > 0, finite
 * d_i >= 0, valid storage.  Errors: FLAME_ERR_PARAM (then *out = NULL),
 * FLAME_ERR_CUDA if the current device cannot be queried. */
flame_status flame_create(flame_ctx **out, const flame_params *p, void *d_state, void *stream);

/* Create a context without a population state, for the field-level
 * diagnostics of a whole periodic lattice whose u and B the caller holds --
 * a lattice split into z-slabs, whose slab contexts refuse the FFT
 * diagnostics: flame_spectra_fields, flame_energy_budget and
 * flame_band_energy with given fields (they use the parameters' tau_nu,
 * tau_eta and d_i).  Every call that needs a state (flame_init,
 * flame_step, flame_moments, flame_spectra, flame_set_state, ...) returns
 * FLAME_ERR_STATE.  Errors: as flame_create, and FLAME_ERR_PARAM for a slab
 * (halo_z = 1). */
flame_status flame_create_fields(flame_ctx **out, const flame_params *p, void *stream);

/* Fill the state with the populations of the initial fields (time t = 0):
 * f = f^mhd(0)(rho, u, B) (Sec. 3.1.1: 6th-order Hermite equilibrium plus
 * the Lorentz stress term) and g = g^Hall(0)(u, B, J0) (eq. gHall_eq) with
 * J0 = curl B; with init_noneq, plus the first-order non-equilibrium parts
 * -(rho c_s^2/omega)(grad u + grad u^T) projected on w_i H2_i/(2 c_s^4) for
 * f and -(W_i/omega_B) xi_ia d_a B_b for g, which make the step's current
 * equal curl B at t = 0.  d_rho [N3] may be NULL (rho = 1); d_u, d_B [3][N3]
 * are required; d_gradu, d_gradB [9][N3] may be NULL (periodic second-order
 * central differences of d_u, d_B).  All FP64.  Resets step and parity.
 * Synchronises to evaluate the whistler CFL number pi d_i max(V_A, |u|)
 * (Sec. 3.4): FLAME_ERR_CFL if it exceeds 1 and strict_cfl is set. */
flame_status flame_init(flame_ctx *ctx, const double *d_rho, const double *d_u, const double *d_B,
                        const double *d_gradu, const double *d_gradB);

/* flame_init from FP32 fields: the same initial populations, with d_rho,
 * d_u, d_B, d_gradu, d_gradB given as FP32 device arrays of the same layout
 * (half the bytes a caller moves to the device).  Gradients are taken in
 * FP64 from the FP32 values; the per-site arithmetic is that of flame_init.
 * Errors and synchronisation as flame_init. */
flame_status flame_init_f32(flame_ctx *ctx, const float *d_rho, const float *d_u, const float *d_B,
                            const float *d_gradu, const float *d_gradB);

/* Advance n >= 0 time steps, one fused kernel launch per step (or, with
 * graph_steps = G, graph replays of G launches; the graph starting at
 * parity 0 is captured by flame_create, the other on its first use, each on
 * a private stream): moments
 * (eqs. LB_moments2, mag_field_LB), current from the 3x3 Hall system (eqs.
 * LB_density_current, soe_current_density), central-moment fluid collision
 * (eqs. cm_collision_step, collision_matrix), Hall-equilibrium BGK magnetic
 * collision (eqs. gHall_eq, MHD_LBscheme) and periodic streaming (eq. stream),
 * in place.  Asynchronous unless check_every > 0.  Errors: FLAME_ERR_PARAM
 * (n < 0), FLAME_ERR_STATE (flame_init not called), sticky errors. */
flame_status flame_step(flame_ctx *ctx, int n);

/* Synchronise the stream and report sticky errors (CUDA, non-finite). */
flame_status flame_sync(flame_ctx *ctx);

/* Step count, parity, CFL number and the sticky non-finite flag. */
flame_status flame_info(flame_ctx *ctx, flame_info_t *out);

/* Macroscopic fields of the current pre-collision populations, FP64:
 * rho [N3], u [3][N3], B [3][N3], J [3][N3] (J from the Hall linear system,
 * as in the step).  Any pointer may be NULL.  Asynchronous. */
flame_status flame_moments(flame_ctx *ctx, double *d_rho, double *d_u, double *d_B, double *d_J);

/* flame_moments written as FP32 (the precision the per-site arithmetic of
 * 16-bit storage has; FP32 storage rounds its FP64 per-site moments): rho
 * [N3], u [3][N3], B [3][N3], J [3][N3], any may be NULL.  Asynchronous. */
flame_status flame_moments_f32(flame_ctx *ctx, float *d_rho, float *d_u, float *d_B, float *d_J);

/* Host-buffer forms of flame_init_f32 and flame_moments_f32, for a run whose
 * fields live in host memory.  The fields cross the host link in chunks of z
 * planes (at most FLAME_IO_CHUNKS, each of whole planes) on a second stream
 * of the context, each chunk's kernel starting as soon as its data has
 * arrived (or been written), so that the copies overlap the kernels.  With
 * page-locked host memory (cudaHostAlloc, cudaHostRegister) the copies are
 * asynchronous; pageable memory works through the driver's staging, with
 * less overlap.  The device workspace is the context's field workspace
 * (6 N3 doubles, allocated on first use and shared with flame_spectra).
 * Both calls return when the caller's buffers are no longer in use. */
enum { FLAME_IO_CHUNKS = 32 };

/* flame_init_f32 from host memory: h_rho [N3] (NULL: rho = 1), h_u, h_B
 * [3][N3] FP32, in flame_init_f32's layout (a z-slab's fields with its
 * ghost planes); the gradients are the periodic central differences.  The
 * same initial populations as flame_init_f32 of the same fields, to the bit.
 * Synchronises (the CFL check).  Errors as flame_init_f32, FLAME_ERR_CUDA for
 * a failed copy. */
flame_status flame_init_f32_host(flame_ctx *ctx, const float *h_rho, const float *h_u, const float *h_B);

/* flame_moments_f32 into host memory: h_rho [N3], h_u, h_B, h_J [3][N3]
 * FP32 of the updated sites, any may be NULL; equal to flame_moments_f32's
 * fields to the bit.  h_scalars: NULL, or FLAME_NSCALARS entries that
 * receive flame_reduce's scalars of the same state, computed on the
 * context's stream while the fields are copied out.  Synchronises.  Errors:
 * FLAME_ERR_STATE (no flame_init), FLAME_ERR_CUDA, FLAME_ERR_NONFINITE as
 * flame_reduce (only with h_scalars). */
flame_status flame_moments_f32_host(flame_ctx *ctx, float *h_rho, float *h_u, float *h_B, float *h_J,
                                    double *h_scalars);

/* Moments at a list of sites, for time series such as the velocity at a
 * fixed point that Sec. 4.1-4.2 follow: d_sites [nsites] linear site indices
 * (z*ny + y)*nx + x (device), d_out [nsites][10] FP64 (device): rho, u[3],
 * B[3], J[3] of the current pre-collision populations.  An index outside the
 * lattice yields NaNs for that entry.  Asynchronous.  Errors:
 * FLAME_ERR_PARAM, FLAME_ERR_STATE (no flame_init). */
flame_status flame_probe(flame_ctx *ctx, int nsites, const long long *d_sites, double *d_out);

/* The current pre-collision populations decoded to FP64 in natural order,
 * d_f [48][N3] in natural slot order, whatever the AA parity.
 * Asynchronous. */
flame_status flame_populations(flame_ctx *ctx, double *d_f);

/* FP64 scalar diagnostics of the current state (Sec. 4.4, 5: energies,
 * cross-helicity, magnetic dissipation, div B estimate).  h_scalars has
 * FLAME_NSCALARS entries (indices FLAME_S_*).  Synchronises. */
flame_status flame_reduce(flame_ctx *ctx, double *h_scalars);

/* Raw FP64 sums of the scalar diagnostics over the context's sites, for
 * combining the slabs of a lattice split along z (add the sums of every
 * slab -- the maximum for FLAME_SUM_UMAX -- and call flame_reduce_combine);
 * h_sums has FLAME_NSUMS entries.  Synchronises.  Errors as flame_reduce. */
enum {
    FLAME_SUM_RHO = 0,       /* sum rho                                */
    FLAME_SUM_MOMX = 1,      /* sum rho u_x (2: y, 3: z)               */
    FLAME_SUM_BX = 4,        /* sum B_x (5: y, 6: z)                   */
    FLAME_SUM_U2 = 7,        /* sum |u|^2                              */
    FLAME_SUM_DB2 = 8,       /* sum |B - B_ref|^2                      */
    FLAME_SUM_UDB = 9,       /* sum u . (B - B_ref)                    */
    FLAME_SUM_UX = 10,       /* sum u_x (11: y, 12: z)                 */
    FLAME_SUM_J2 = 13,       /* sum |J|^2                              */
    FLAME_SUM_UMAX = 14,     /* max |u| (combine by maximum)           */
    FLAME_SUM_DIV2 = 15,     /* sum ((omega_B/C^2) Tr Lambda)^2        */
    FLAME_SUM_NONFINITE = 16,/* sites with a non-finite moment         */
    FLAME_SUM_SITES = 17,    /* number of sites summed                 */
    FLAME_NSUMS = 18
};
flame_status flame_reduce_sums(flame_ctx *ctx, double *h_sums);

/* The FLAME_S_* scalars of flame_reduce from raw sums (those of one context,
 * or the combination of several slabs'), with the reference field B_ref of p.
 * Host only, no GPU needed.  Returns 0, or -1 for NULL arguments or a zero
 * site count. */
int flame_reduce_combine(const flame_params *p, const double *h_sums, double *h_scalars);

/* The step kernel flame_step launches for these parameters (with a state
 * allocated as flame_create requires): FLAME_KERNEL_SITE (one site per
 * thread), FLAME_KERNEL_ROWS (x rows staged in shared memory, two sites per
 * thread), FLAME_KERNEL_HALF_ROWS (half rows staged) or FLAME_KERNEL_PAIRS
 * (site pairs unstaged); the choice flame_params.kernel leaves to the
 * library, or the one it forces where it applies.  Host only, no GPU
 * needed.  Returns 0 for invalid parameters. */
enum { FLAME_KERNEL_SITE = 1, FLAME_KERNEL_ROWS = 2, FLAME_KERNEL_HALF_ROWS = 3, FLAME_KERNEL_PAIRS = 4 };
int flame_step_kernel(const flame_params *p);

/* The halo exchange of a lattice split along z into slab contexts (halo_z =
 * 1; the paper splits its domain along one direction and exchanges the
 * boundary nodes every step, Sec. 4).  Under the AA pattern only the odd
 * step crosses a slab face: it reads, at each face, the populations that
 * leave the neighbouring slab's boundary plane towards this one (9 fluid
 * and 3 magnetic storage slots of that plane) and writes back the ones that
 * leave this slab towards the neighbour.  So after a step that leaves the
 * state at AA parity 1, every ghost plane receives those slots of the
 * neighbour's boundary plane; after a step that leaves parity 0, the same
 * slots of every ghost plane go back into the neighbour's boundary plane.
 *
 * flame_halo_plan: the runs of storage slots this slab sends through face
 * `face` (0: towards z - 1, 1: towards z + 1) and receives there, after a
 * step that left the state at `parity`: run 0 fluid (9 slots), run 1
 * magnetic (3 slots).  A run is nslots slot-planes; slot-plane (slot, plane)
 * is nx*ny contiguous values starting at element (slot * N3s + plane * nx *
 * ny) of the state, N3s = nx*ny*(nz + 2).  Through a face, this slab's send
 * run r pairs with the neighbour's receive run r of the opposite face.
 * Host only.  Returns 0, or -1 for invalid arguments (p not a slab, parity
 * not 0/1, face not 0/1, NULL outputs). */
typedef struct {
    int first_slot;  /* first storage slot of the run                         */
    int nslots;      /* consecutive storage slots                             */
    int plane;       /* plane of the state, 0 .. nz + 1 (0 and nz + 1: ghosts) */
} flame_halo_run;
int flame_halo_plan(const flame_params *p, int parity, int face, flame_halo_run send[2], flame_halo_run recv[2]);

/* The exchange between two slab contexts on one device (or on devices with
 * peer access), `upper` being the slab above `lower` (the same context for a
 * lattice of one slab, whose exchange is its periodic wrap in z): the copies
 * of flame_halo_plan in both directions through the face between them, as
 * cudaMemcpy2DAsync on lower's stream.  Call it for every pair of
 * neighbouring slabs after each step, once all slabs have taken that step;
 * the work of both contexts must be ordered with that stream (one stream for
 * all slabs, or events).  Errors: FLAME_ERR_PARAM (not slab contexts, or
 * nx, ny or storage differ), FLAME_ERR_STATE (not initialised, or at
 * different step parities), FLAME_ERR_CUDA. */
flame_status flame_halo_exchange(flame_ctx *lower, flame_ctx *upper);

/* Shell energy spectra of u and B - <B> (Sec. 4.4): with
 * F_hat(m) = N3^-1 sum_x F(x) exp(-2 pi i m.x/N), h_Eu[n] and h_Eb[n] are
 * 1/2 sum |F_hat|^2 over the modes with round(|m|) = n, n = 0..nshell-1
 * (modes beyond are dropped; summed over every shell they give 1/2<|F|^2>);
 * 1 <= nshell <= 4096, else FLAME_ERR_PARAM.
 * FFTs by cuFFT (FP64), shell sums in FP64.  Either output may be NULL.
 * Synchronises. */
flame_status flame_spectra(flame_ctx *ctx, int nshell, double *h_Eu, double *h_Eb);

/* flame_spectra of given FP64 fields d_u and d_B ([3][N3] each, device,
 * both required: FLAME_ERR_PARAM otherwise) instead of the state's u and B.
 * As there, the m = 0 mode of B (its mean) is left out, so h_Eb is the
 * spectrum of B - <B>.  Works on every non-slab context, including one from
 * flame_create_fields.  Synchronises. */
flame_status flame_spectra_fields(flame_ctx *ctx, int nshell, const double *d_u, const double *d_B, double *h_Eu,
                                  double *h_Eb);

/* Magnetic energy in a band of shells (the spectra of Sec. 4.4) and its
 * gradient, the loss of the differentiable runs:
 *   L = sum_{lo <= n <= hi} E_B(n),  E_B(n) = 1/2 sum_{round|m| = n} |F(B)(m)|^2,
 * F(B) = N3^-1 FFT(B) (shell 0 is the mean field; lo >= 1 leaves it out).
 * d_B: [3][N3] FP64 field (device), or NULL for the B of the current state.
 * h_L (host, required) receives L.  d_dLdB (device, [3][N3] FP64, may be
 * NULL) receives dL/dB = N3^-1 Re IFFT(mask F(B)).  d_adj (device, [48][N3]
 * FP32, may be NULL) receives the seed of flame_step_adjoint for a loss of
 * the current state: dL/df of the pre-collision populations in natural slot
 * order, 0 for the fluid and dL/dB_b for every D3Q7 velocity of component b
 * (B_b is their sum, eq. mag_field_LB).  cuFFT (FP64).  The first call
 * allocates a workspace (3 N3 doubles and 3 half spectra).  Synchronises.
 * Errors: FLAME_ERR_PARAM (lo < 0, hi < lo, h_L NULL), FLAME_ERR_STATE (no
 * flame_init and d_B NULL), FLAME_ERR_CUDA, sticky errors. */
flame_status flame_band_energy(flame_ctx *ctx, int lo, int hi, const double *d_B, double *h_L, double *d_dLdB,
                               float *d_adj);

/* Wavenumber energy budget of eq. mhd_en_trans (Sec. 4.4) of fields u, B:
 *   S(n) = sum_{round|m| < n} Re[F(u)* . (F(u.grad u) - F(J x B))
 *                                - F(B)* . F(curl(V x B))]
 *   D(n) = sum_{round|m| < n} k^2 (nu |F(u)|^2 + eta |F(B)|^2)
 *   E(n) = 1/2 sum_{round|m| = n} (|F(u)|^2 + |F(B)|^2)
 * with F = N3^-1 FFT, k = 2 pi m / N, spectral derivatives (the Nyquist
 * wavenumber of an even axis set to zero, also in k^2), J = curl B spectral,
 * V = u - d_i J (the Hall term in the induction flux; V = u for d_i = 0),
 * nu = c_s^2 (tau_nu - 1/2), eta = C^2 (tau_eta - 1/2) and d_i of the
 * context.  Then d/dt sum_{n' < n} E(n') = -S(n) - D(n) for the
 * incompressible equations.  d_u, d_B: [3][N3] FP64 device fields, or both
 * NULL for the moments of the current state.  h_E, h_S, h_D: nshell host
 * doubles each (any may be NULL), 1 <= nshell <= 1024.  cuFFT (FP64): 24
 * transforms.  The first call allocates a workspace of 15 N3 doubles and 9
 * half spectra.  Synchronises.  Errors: FLAME_ERR_PARAM (nshell, only one of
 * d_u / d_B given), FLAME_ERR_STATE (no flame_init and no fields),
 * FLAME_ERR_CUDA, sticky errors. */
flame_status flame_energy_budget(flame_ctx *ctx, int nshell, const double *d_u, const double *d_B, double *h_E,
                                 double *h_S, double *h_D);

/* Copy the raw population state (flame_state_bytes) to d_dst, with the step
 * count and parity needed to resume.  Asynchronous. */
flame_status flame_get_state(flame_ctx *ctx, void *d_dst, long long *step, int *parity);

/* Replace the population state with d_src (flame_state_bytes, written by
 * flame_get_state with the same parameters) and set step and parity.
 * Errors: FLAME_ERR_STATE (parity not 0/1, step < 0).  Asynchronous. */
flame_status flame_set_state(flame_ctx *ctx, const void *d_src, long long step, int parity);

/* Adjoint (vector-Jacobian product) of one flame_step, for gradients of a
 * loss of a later state (the hand-written reverse of Sec. 3's collision and
 * streaming; the paper has no adjoint, its equations define the forward map).
 * d_state: a state blob (flame_state_bytes, as written by flame_get_state)
 * holding the pre-collision populations at time t with AA parity `parity`.
 * d_adj_in: [48][N3] FP32, dL/df(t+1) for the physical pre-collision
 * populations at t+1 in natural slot order (the layout of
 * flame_populations).  d_adj_out: [48][N3] FP32, receives dL/df(t); must not
 * alias d_adj_in.  d_ddi: one device double, overwritten with this step's
 * contribution to dL/d(d_i).  Forward quantities are recomputed from
 * d_state in FP32; the d_i contribution is summed in FP64.  Asynchronous.
 * The first call allocates a small per-block workspace.  Errors:
 * FLAME_ERR_PARAM (null or aliased pointers), FLAME_ERR_STATE (parity),
 * FLAME_ERR_CUDA. */
flame_status flame_step_adjoint(flame_ctx *ctx, const void *d_state, int parity, const float *d_adj_in,
                                float *d_adj_out, double *d_ddi);

/* Adjoint of flame_init for rho = 1 and central-difference gradients (the
 * d_gradu = d_gradB = NULL case): given d_adj0 = dL/df(0) ([48][N3] FP32,
 * natural order) and the FP64 fields d_u, d_B it was built from, writes
 * dL/du ([3][N3], FP64, may be NULL), dL/dB ([3][N3], may be NULL; not both)
 * and the initial state's contribution to dL/d(d_i) into *d_ddi (device).
 * Includes the transposed periodic central-difference stencil of J0 = curl B
 * and of the non-equilibrium parts.  The first call allocates 24 N3 doubles
 * of workspace.  Asynchronous.  Errors: FLAME_ERR_PARAM, FLAME_ERR_CUDA. */
flame_status flame_init_adjoint(flame_ctx *ctx, const double *d_u, const double *d_B, const float *d_adj0,
                                double *d_ubar, double *d_Bbar, double *d_ddi);

/* Largest block count flame_reduce_static accepts; its device scratch holds
 * this many blocks' partial sums (139,264 bytes per device). */
#define FLAME_STATIC_REDUCE_BLOCKS_MAX 1024

/* flame_reduce without any allocation, for callers that must not call
 * cudaMalloc (flame_reduce allocates a workspace on its first call, which
 * can synchronise the device and stall queued work, and some hosts give all
 * device memory to their own caching allocator).  The paper has no
 * counterpart; it is a property of this library's interface.
 * Writes the same FLAME_NSCALARS scalars as flame_reduce, FP64, to device
 * memory d_scalars (caller-owned), asynchronously on the context's stream;
 * the non-finite count is in d_scalars[FLAME_S_NONFINITE], not in the
 * status.  nblocks: reduction blocks, 1..FLAME_STATIC_REDUCE_BLOCKS_MAX, or
 * 0 for 4 per SM; larger values fail with FLAME_ERR_PARAM.
 * The partial sums live in a fixed device array that each device holds from
 * library load until exit.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, with the device made
 * current): make that first call before any stream capture.  The array is
 * shared by all contexts on the device and keeps the last call's contents;
 * every call overwrites what it reads, and calls that overlap on the GPU
 * race on it.  Errors: FLAME_ERR_PARAM, FLAME_ERR_STATE (no flame_init),
 * FLAME_ERR_CUDA, sticky context errors. */
flame_status flame_reduce_static(flame_ctx *ctx, int nblocks, double *d_scalars);

/* Test hook for the failure path of the row kernel's waits (the paper has no
 * counterpart).  The row kernel stages its tiles with copies that complete
 * on shared-memory barriers, and every wait on a barrier gives up after a
 * bounded number of polls, sets a flag and ends the launch without writing
 * the state.  After this call the next flame_step launches one step whose
 * barriers are armed but never fed (no copy is issued), with a limit of
 * `tries` polls per wait, synchronises, and returns FLAME_ERR_TIMEOUT
 * (sticky, like any failure); the state and the step count are left as they
 * were.  Errors: FLAME_ERR_PARAM (tries == 0, or the context does not run
 * the row kernel: FP16/BF16 storage (any variant), kernel = 0, nx as listed
 * at flame_params.kernel), FLAME_ERR_STATE (before flame_init). */
flame_status flame_debug_stall_next_step(flame_ctx *ctx, unsigned tries);

/* Release the context and its internal workspace (not the caller's state). */
void flame_destroy(flame_ctx *ctx);

/* Human-readable text of a status code (static storage). */
const char *flame_status_string(flame_status s);

/* The velocity tables the kernels use: c27 [27*3] (App. A order) and
 * xi7 [7*3].  Returns 0. Host only, no GPU needed. */
int flame_lattice(int *c27, int *xi7);

#ifdef __cplusplus
}
#endif
#endif
