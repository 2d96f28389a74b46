// flame_internal.h -- kernel launchers shared by the translation units of
// libflame.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace flame {

// Per-run constants of the step (lattice units).
struct StepConsts {
  float omega;    // 1 / tau_nu          (Sec. 3.1.1)
  float omegaB;   // 1 / tau_eta         (Sec. 3.2)
  float alphaH;   // Hall coefficient d_i
  float rho0;     // reference density of the deviation encoding
  float Bref[3];  // reference field of the deviation encoding
};

// The lattice a context updates.  A periodic lattice updates all its nz
// planes (z0 = 0, nzi = nz).  A z-slab of a larger lattice (flame_params
// .halo_z) holds its nzi planes between two ghost planes, nz = nzi + 2, and
// updates planes z0 = 1 .. nzi; its ghost planes hold the neighbouring
// slabs' boundary slots, exchanged between steps.
struct Grid {
  int nx, ny, nz;  // planes held in the state
  long long n3;    // nx * ny * nz: the stride between storage slots
  int z0, nzi;     // the planes updated: z0 .. z0 + nzi - 1
  long long n3i;   // nx * ny * nzi: the sites updated, and the size of per-site outputs
};

// Scheme variants (flame_variant).
constexpr int kVarFlame = 0;      // the paper's scheme
constexpr int kVarBgkFluid = 1;   // BGK fluid collision
constexpr int kVarEmhd = 2;       // electron MHD magnetic equilibrium
constexpr int kVarFdCurrent = 3;  // J from the central-difference curl of B

// storage: 1 FP32, 2 FP16, 3 BF16 (flame_storage).  Bfd: scratch for the
// pre-collision B - B_ref, [3][N3] values of the storage's element type,
// required by kVarFdCurrent only.
// kernel (flame_params.kernel): 0 the row kernel where step_row_supported
// (whole rows, half rows or the unstaged pair kernel as row_segments
// chooses), else the one-site kernel; 1 always the one-site kernel; 2 the
// row kernel on whole rows, 3 on half rows and 4 the pair kernel, where they
// apply (else the one-site kernel).
cudaError_t launch_step(int storage, int odd, void* pop, Grid g, const StepConsts& k, unsigned* flag,
                        cudaStream_t s, int variant = kVarFlame, void* Bfd = nullptr, int kernel = 0);

// The step for 16-bit storage, two sites per thread in packed FP32 pairs
// (step_row.cuh): as a persistent kernel over x rows staged in shared memory
// (64 <= nx <= 1024 with nx a multiple of 8, a 16-byte aligned state; half
// rows for nx > 256 a multiple of 16 only), or unstaged (the pair kernel,
// any even nx); every variant.  Automatic choice: the faster of these by row
// length, for every even nx.  flag bit 1: a
// non-finite moment; bit 2: a staged copy did not complete within the wait
// limit.
bool step_row_supported(Grid g, int storage, int variant, const void* pop, int kernel = 0);
// The segments per tile launch_step_row uses (0: the pair kernel, no staging).
int row_segments(int nx, int kernel);
// step_row_supported with staged rows (the kernels whose copies have waits).
bool step_row_staged(Grid g, int storage, int variant, const void* pop, int kernel = 0);
// Settles the launch configuration of the kernel launch_step would use
// (no launch); needed once before stream capture.
cudaError_t prepare_step(int storage, const void* pop, Grid g, int variant, int kernel);
// Bfd: the pre-collision B - B_ref ([3][N3], storage type) that launch_bfield wrote,
// read by kVarFdCurrent only.  stall_tries > 0: the failure-path test -- the
// launch arms its barriers without issuing copies and gives up after
// stall_tries polls per wait.  kernel as for launch_step (0, 2 or 3).
cudaError_t launch_step_row(int storage, int odd, void* pop, Grid g, const StepConsts& k, unsigned* flag,
                            cudaStream_t s, int variant = kVarFlame, const void* Bfd = nullptr,
                            unsigned stall_tries = 0, int kernel = 0);
// The pre-pass of kVarFdCurrent: B - B_ref of the pre-collision populations
// at every site into Bfd ([3][N3] in the storage's element type).
cudaError_t launch_bfield(int storage, int odd, const void* pop, Grid g, void* Bfd, cudaStream_t s);

cudaError_t launch_init(int storage, void* pop, Grid g, const StepConsts& k, int noneq, const double* rho,
                        const double* u, const double* B, const double* gu, const double* gB,
                        unsigned* speed_bits, cudaStream_t s);

// The same from FP32 fields (flame_init_f32).
cudaError_t launch_init_f32(int storage, void* pop, Grid g, const StepConsts& k, int noneq, const float* rho,
                            const float* u, const float* B, const float* gu, const float* gB,
                            unsigned* speed_bits, cudaStream_t s);

// ostride: the stride between the components of u, B and J (0: N3).
cudaError_t launch_moments(int storage, int odd, const void* pop, Grid g, const StepConsts& k, double* rho,
                           double* u, double* B, double* J, cudaStream_t s, long long ostride = 0);
// The same, written as FP32 (flame_moments_f32).
cudaError_t launch_moments_f32(int storage, int odd, const void* pop, Grid g, const StepConsts& k, float* rho,
                               float* u, float* B, float* J, cudaStream_t s, long long ostride = 0);

// The chunks of planes the host-buffer calls (flame_init_f32_host,
// flame_moments_f32_host) move and compute one at a time: np planes from z0
// in io_chunk_count(np) chunks, chunk j covering planes
// [io_first(z0, np, n, j), io_first(z0, np, n, j + 1)).
constexpr int kIoChunks = 32;
inline int io_chunk_count(int np) { return np < kIoChunks ? np : kIoChunks; }
inline int io_first(int z0, int np, int n, int j) { return z0 + (int)((long long)np * j / n); }
// The chunk of planes [0, nz) in n chunks that holds plane q.
inline int io_chunk_of(int nz, int n, int q) {
  int j = 0;
  while (j + 1 < n && io_first(0, nz, n, j + 1) <= q) ++j;
  return j;
}
// The initialisation of planes [a, b) takes central differences along z, so
// it reads planes a - 1 .. b (periodic over the nz planes held).  With the
// held planes copied in order in n chunks, it can start once chunk
// io_init_needs(...) has arrived.
inline int io_init_needs(int nz, int n, int a, int b) {
  int m = io_chunk_of(nz, n, b - 1);
  const int lo = io_chunk_of(nz, n, (a - 1 + nz) % nz), hi = io_chunk_of(nz, n, b % nz);
  if (lo > m) m = lo;
  if (hi > m) m = hi;
  return m;
}

cudaError_t launch_populations(int storage, int odd, const void* pop, Grid g, const StepConsts& k,
                               double* f, cudaStream_t s);

// Number of FP64 partial sums per block written by the reduction.
constexpr int kRedVals = 17;
// Upper bound on the reduction's block count (its partials fill
// kRedBlocksMax * kRedVals doubles of scratch).
constexpr int kRedBlocksMax = 1024;

// Moments of the listed sites: out[10 j + (rho, u[3], B[3], J[3])].
cudaError_t launch_probe(int storage, int odd, const void* pop, Grid g, const StepConsts& k, int n,
                         const long long* sites, double* out, cudaStream_t s);

cudaError_t launch_reduce(int storage, int odd, const void* pop, Grid g, const StepConsts& k, int nblocks,
                          double* partials, double* out, cudaStream_t s);

// Only the first stage of launch_reduce: per-block partial sums
// (kRedVals doubles per block) of the reduce kernel into `partials`.
cudaError_t launch_reduce_partials(int storage, int odd, const void* pop, Grid g, const StepConsts& k, int nblocks,
                                   double* partials, cudaStream_t s);

// Read-only view of a context for entry points outside api.cu.
struct CtxView {
  void* state;
  int storage;
  int parity;
  int device;
  int nsm;
  int initialized;
  int status;  // flame_status of the context (sticky errors)
  cudaStream_t stream;
  Grid g;
  StepConsts k;
  double Bref[3];
  double tau_nu, tau_eta, d_i;  // the context's parameters in FP64
};

// Adjoint kernels (adjoint.cu).  The step adjoint reads the forward state at
// time t (AA parity `odd`), lambda_{t+1} and writes lambda_t (FP32, natural
// slot order [48][N3]); both write one partial d(loss)/d(d_i) per block into
// `partials` (adjoint_partials_needed(g) doubles) and its sum into *ddi.
long long adjoint_partials_needed(Grid g);
cudaError_t launch_step_adjoint(int storage, int odd, const void* pop, Grid g, const StepConsts& k, const float* lin,
                                float* lout, double* partials, double* ddi, cudaStream_t s);
// ws: 24 * N3 doubles of workspace.
cudaError_t launch_init_adjoint(Grid g, const StepConsts& k, const double* u, const double* B, const float* lam,
                                double* ws, double* partials, double* ubar, double* Bbar, double* ddi,
                                cudaStream_t s);

cudaError_t launch_shell_bin(const void* spec /* cufftDoubleComplex */, Grid g, int nshell, int zero_mean,
                             double* shells, cudaStream_t s);

// The stride, in elements, between fields handed to cuFFT: N3 rounded up to
// a multiple of 32, so that every field of an array of fields starts on a
// 256-byte boundary (cuFFT's transforms need at least the alignment of the
// complex type, which an odd N3 would break).
inline long long fft_stride(long long n) { return (n + 31) & ~31LL; }

}  // namespace flame

struct flame_ctx;
// Fills *v from the context; returns 0, or -1 for a null context.
int flame_ctx_view(const flame_ctx* c, flame::CtxView* v);
// The context's slot for the spectral diagnostics' workspace (spectral.cu),
// released by flame_destroy through flame::spectral_ws_free.
void** flame_ctx_spectral_slot(flame_ctx* c);
namespace flame {
void spectral_ws_free(void* ws);
}
// Records a failed CUDA call in the context's sticky status, as the entry
// points of api.cu do (FLAME_ERR_CUDA unless an error is already recorded);
// returns FLAME_ERR_CUDA, or FLAME_OK for e == cudaSuccess.
int flame_ctx_cuda_fail(flame_ctx* c, cudaError_t e);
