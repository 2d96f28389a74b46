// api.cu -- the C ABI declared in include/flame.h.
#include <cufft.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "flame.h"
#include "flame_internal.h"
#include "lattice.cuh"

namespace {
// An NVTX range over one entry point: the host-side span of each call shows on
// a profiler's timeline (header-only NVTX; without a tool attached a push and
// a pop cost a few nanoseconds).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
}  // namespace

struct flame_ctx {
  flame_params p;
  void* state;
  cudaStream_t stream;
  int device;
  int nsm;
  long long step;
  int parity;
  bool initialized;
  flame_status sticky;
  double cfl, max_speed;
  int nonfinite;
  unsigned* d_flags;  // [0] non-finite flag, [1] max speed (float bits)
  // internal workspace (lazily allocated)
  double* d_red;      // kRedBlocksMax * kRedVals partials + kRedVals result
  double* d_fields;   // 6 * fft_stride(N3) doubles: u, B for spectra; FP32 fields of the host-buffer calls
  void* d_spec;       // nz * ny * (nx/2+1) cufftDoubleComplex
  double* d_shells;   // 2 * nshell_cap doubles
  int nshell_cap;
  cufftHandle plan;
  bool has_plan;
  void* d_bfield;            // [3][N3] values of the storage type, FLAME_FD_CURRENT only
  cudaGraphExec_t graph[2];  // graph_steps launches starting at parity 0 / 1
  bool has_graph[2];
  double* d_adj_partials;  // adjoint_partials_needed doubles
  double* d_adj_ws;        // 24 * N3 doubles (initialisation adjoint)
  flame::StepConsts k;
  flame::Grid g;
  unsigned stall_tries;  // > 0: the next flame_step runs the wait-failure test (flame_debug_stall_next_step)
  void* spectral;        // workspace of the spectral diagnostics (spectral.cu), lazily allocated
  // the host-buffer calls: their copy stream and events, created on first use
  cudaStream_t io_stream;
  cudaEvent_t io_ev[flame::kIoChunks + 1];
  int n_io_ev;  // events created
  bool has_io_stream;
  size_t io_max_pitch;  // the device's largest pitch of a 2-D copy, in bytes
};

namespace {

size_t elem_bytes(int storage) { return storage == FLAME_FP32 ? 4 : (storage == FLAME_FP16 || storage == FLAME_BF16) ? 2 : 0; }

flame_status check_params(const flame_params* p) {
  if (!p) return FLAME_ERR_PARAM;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return FLAME_ERR_PARAM;
  if (p->halo_z != 0 && p->halo_z != 1) return FLAME_ERR_PARAM;
  if (p->ny > 65535 || p->nz > 65533) return FLAME_ERR_PARAM;  // grid y / z launch dimensions
  const long long n3 = (long long)p->nx * p->ny * (p->nz + 2 * p->halo_z);
  if (n3 >= (1ll << 31)) return FLAME_ERR_PARAM;
  // the finite-difference current needs B on the ghost planes, which hold only
  // the slots a face exchanges
  if (p->halo_z && p->variant == FLAME_FD_CURRENT) return FLAME_ERR_PARAM;
  if (!(p->tau_nu > 0.5) || !(p->tau_eta > 0.5) || !std::isfinite(p->tau_nu) || !std::isfinite(p->tau_eta))
    return FLAME_ERR_PARAM;
  if (!(p->d_i >= 0.0) || !std::isfinite(p->d_i)) return FLAME_ERR_PARAM;
  if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return FLAME_ERR_PARAM;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->B_ref[a])) return FLAME_ERR_PARAM;
  if (elem_bytes(p->storage) == 0) return FLAME_ERR_PARAM;
  if (p->check_every < 0) return FLAME_ERR_PARAM;
  if (p->graph_steps < 0 || (p->graph_steps & 1)) return FLAME_ERR_PARAM;
  if (p->variant < FLAME_SCHEME || p->variant > FLAME_FD_CURRENT) return FLAME_ERR_PARAM;
  if (p->kernel < 0 || p->kernel > 4) return FLAME_ERR_PARAM;
  return FLAME_OK;
}

flame_status cuda_fail(flame_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return FLAME_OK;
  if (c && c->sticky == FLAME_OK) c->sticky = FLAME_ERR_CUDA;
  return FLAME_ERR_CUDA;
}

flame_status usable(flame_ctx* c) {
  if (!c) return FLAME_ERR_PARAM;
  if (c->sticky != FLAME_OK) return c->sticky;
  return FLAME_OK;
}

// Synchronise, then fold CUDA errors and the non-finite flag into the
// sticky status.
flame_status sync_and_check(flame_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  unsigned flag = 0;
  e = cudaMemcpy(&flag, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (flag & 2u) {
    if (c->sticky == FLAME_OK) c->sticky = FLAME_ERR_TIMEOUT;
  }
  if (flag & 1u) {
    c->nonfinite = 1;
    if (c->sticky == FLAME_OK) c->sticky = FLAME_ERR_NONFINITE;
  }
  return c->sticky;
}

int reduce_blocks(const flame_ctx* c) {
  long long want = (long long)c->nsm * 4;
  const long long per = (c->g.n3i + 255) / 256;
  if (want > per) want = per;
  if (want < 1) want = 1;
  if (want > flame::kRedBlocksMax) want = flame::kRedBlocksMax;
  return (int)want;
}

// FP64 power of a D2Z half spectrum binned into integer shells.
__global__ void shell_bin_kernel(const cufftDoubleComplex* __restrict__ F, flame::Grid g, int nshell,
                                 int zero_mean, double* __restrict__ shells) {
  extern __shared__ double hist[];
  for (int i = threadIdx.x; i < nshell; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  const int hx = g.nx / 2 + 1;
  const long long total = (long long)g.nz * g.ny * hx;
  const double inv = 1.0 / ((double)g.n3 * (double)g.n3);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(t % hx);
    const int ky = (int)((t / hx) % g.ny);
    const int kz = (int)(t / ((long long)hx * g.ny));
    const int my = ky <= g.ny / 2 ? ky : ky - g.ny;
    const int mz = kz <= g.nz / 2 ? kz : kz - g.nz;
    if (zero_mean && kx == 0 && my == 0 && mz == 0) continue;
    const long long m2 = (long long)kx * kx + (long long)my * my + (long long)mz * mz;
    const int n = __double2int_rn(sqrt((double)m2));
    if (n >= nshell) continue;
    const double w = (kx == 0 || (g.nx % 2 == 0 && kx == g.nx / 2)) ? 1.0 : 2.0;
    const cufftDoubleComplex v = F[t];
    atomicAdd(&hist[n], w * (v.x * v.x + v.y * v.y) * inv);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nshell; i += blockDim.x)
    if (hist[i] != 0.0) atomicAdd(&shells[i], hist[i]);
}

}  // namespace

namespace flame {
cudaError_t launch_shell_bin(const void* spec, Grid g, int nshell, int zero_mean, double* shells, cudaStream_t s) {
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  shell_bin_kernel<<<nsm * 2, 256, (size_t)nshell * sizeof(double), s>>>(
      static_cast<const cufftDoubleComplex*>(spec), g, nshell, zero_mean, shells);
  return cudaGetLastError();
}
}  // namespace flame

int flame_ctx_view(const flame_ctx* c, flame::CtxView* v) {
  if (!c || !v) return -1;
  v->state = c->state;
  v->storage = c->p.storage;
  v->parity = c->parity;
  v->device = c->device;
  v->nsm = c->nsm;
  v->initialized = c->initialized ? 1 : 0;
  v->status = (int)c->sticky;
  v->stream = c->stream;
  v->g = c->g;
  v->k = c->k;
  for (int a = 0; a < 3; ++a) v->Bref[a] = c->p.B_ref[a];
  v->tau_nu = c->p.tau_nu;
  v->tau_eta = c->p.tau_eta;
  v->d_i = c->p.d_i;
  return 0;
}

int flame_ctx_cuda_fail(flame_ctx* c, cudaError_t e) { return (int)cuda_fail(c, e); }

void** flame_ctx_spectral_slot(flame_ctx* c) { return c ? &c->spectral : nullptr; }

extern "C" {

static cudaError_t capture_graph(flame_ctx* c, int parity);

size_t flame_state_bytes(const flame_params* p) {
  if (check_params(p) != FLAME_OK) return 0;
  return (size_t)flame::kPop * (size_t)p->nx * (size_t)p->ny * (size_t)(p->nz + 2 * p->halo_z) *
         elem_bytes(p->storage);
}

// flame_create and flame_create_fields (d_state null: no population state).
static flame_status create_ctx(flame_ctx** out, const flame_params* p, void* d_state, void* stream) {
  flame_ctx* c = new (std::nothrow) flame_ctx;
  if (!c) return FLAME_ERR_PARAM;
  std::memset(static_cast<void*>(c), 0, sizeof(*c));
  c->p = *p;
  c->state = d_state;
  c->stream = static_cast<cudaStream_t>(stream);
  c->sticky = FLAME_OK;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return FLAME_ERR_CUDA;
  }
  if (cudaMalloc(&c->d_flags, 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemsetAsync(c->d_flags, 0, 2 * sizeof(unsigned), c->stream) != cudaSuccess) {
    cudaFree(c->d_flags);
    delete c;
    return FLAME_ERR_CUDA;
  }
  if (d_state && p->variant == FLAME_FD_CURRENT &&
      cudaMalloc(&c->d_bfield, 3 * elem_bytes(p->storage) * (size_t)p->nx * p->ny * p->nz) != cudaSuccess) {
    cudaFree(c->d_flags);
    delete c;
    return FLAME_ERR_CUDA;
  }
  c->k.omega = (float)(1.0 / p->tau_nu);
  c->k.omegaB = (float)(1.0 / p->tau_eta);
  c->k.alphaH = (float)p->d_i;
  c->k.rho0 = (float)p->rho0;
  for (int a = 0; a < 3; ++a) c->k.Bref[a] = (float)p->B_ref[a];
  c->g.nx = p->nx;
  c->g.ny = p->ny;
  c->g.nz = p->nz + 2 * p->halo_z;
  c->g.n3 = (long long)p->nx * p->ny * c->g.nz;
  c->g.z0 = p->halo_z;
  c->g.nzi = p->nz;
  c->g.n3i = (long long)p->nx * p->ny * p->nz;
  // The graph of the first G steps after flame_init (parity 0) is captured
  // here, with the context, so that the first flame_step does not pay for
  // the capture; the parity-1 graph is captured on its first use.
  if (d_state && p->graph_steps > 0 && capture_graph(c, 0) != cudaSuccess) {
    flame_destroy(c);
    return FLAME_ERR_CUDA;
  }
  *out = c;
  return FLAME_OK;
}

flame_status flame_create(flame_ctx** out, const flame_params* p, void* d_state, void* stream) {
  if (!out) return FLAME_ERR_PARAM;
  *out = nullptr;
  flame_status st = check_params(p);
  if (st != FLAME_OK) return st;
  if (!d_state || (reinterpret_cast<uintptr_t>(d_state) & 255u) != 0) return FLAME_ERR_PARAM;
  return create_ctx(out, p, d_state, stream);
}

flame_status flame_create_fields(flame_ctx** out, const flame_params* p, void* stream) {
  if (!out) return FLAME_ERR_PARAM;
  *out = nullptr;
  flame_status st = check_params(p);
  if (st != FLAME_OK) return st;
  if (p->halo_z) return FLAME_ERR_PARAM;  // the field diagnostics take whole periodic lattices
  return create_ctx(out, p, nullptr, stream);
}

}  // extern "C"

// flame_init, flame_init_f32 and flame_init_f32_host: `launch` queues the
// initialisation on the context's stream once the flags are cleared; the CFL
// number then comes from the maximum speed the initialisation recorded.
template <class Launch>
static flame_status init_with(flame_ctx* c, Launch&& launch) {
  // a fresh initial state clears a previous non-finite condition
  c->sticky = FLAME_OK;
  c->nonfinite = 0;
  cudaError_t e = cudaMemsetAsync(c->d_flags, 0, 2 * sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = launch();
  if (e != cudaSuccess) return cuda_fail(c, e);
  unsigned bits = 0;
  e = cudaMemcpyAsync(&bits, c->d_flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  float sp;
  std::memcpy(&sp, &bits, sizeof(sp));
  c->max_speed = sp;
  c->cfl = M_PI * c->p.d_i * c->max_speed;
  c->step = 0;
  c->parity = 0;
  c->initialized = true;
  if (!std::isfinite(c->max_speed)) {
    c->nonfinite = 1;
    c->sticky = FLAME_ERR_NONFINITE;
    return c->sticky;
  }
  if (c->p.strict_cfl && c->cfl > 1.0) return FLAME_ERR_CFL;
  return FLAME_OK;
}

// flame_init and flame_init_f32: the fields' element type F (double or float).
template <class F>
static flame_status init_from(flame_ctx* c, const F* d_rho, const F* d_u, const F* d_B, const F* d_gradu,
                              const F* d_gradB) {
  if (!c) return FLAME_ERR_PARAM;
  if (c->sticky == FLAME_ERR_CUDA) return c->sticky;
  if (!c->state) return FLAME_ERR_STATE;
  if (!d_u || !d_B) return FLAME_ERR_PARAM;
  return init_with(c, [&]() -> cudaError_t {
    if constexpr (sizeof(F) == sizeof(double))
      return flame::launch_init(c->p.storage, c->state, c->g, c->k, c->p.init_noneq, d_rho, d_u, d_B, d_gradu,
                                d_gradB, c->d_flags + 1, c->stream);
    else
      return flame::launch_init_f32(c->p.storage, c->state, c->g, c->k, c->p.init_noneq, d_rho, d_u, d_B, d_gradu,
                                    d_gradB, c->d_flags + 1, c->stream);
  });
}

extern "C" {

flame_status flame_init(flame_ctx* c, const double* d_rho, const double* d_u, const double* d_B,
                        const double* d_gradu, const double* d_gradB) {
  const Range range("flame_init");
  return init_from<double>(c, d_rho, d_u, d_B, d_gradu, d_gradB);
}

flame_status flame_init_f32(flame_ctx* c, const float* d_rho, const float* d_u, const float* d_B,
                            const float* d_gradu, const float* d_gradB) {
  const Range range("flame_init_f32");
  return init_from<float>(c, d_rho, d_u, d_B, d_gradu, d_gradB);
}

// Capture graph_steps step launches starting at `parity` into c->graph[parity].
static cudaError_t capture_graph(flame_ctx* c, int parity) {
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  // launch configuration (shared-memory opt-in, occupancy) is settled
  // before capture, so the captured launches call no configuration API
  e = flame::prepare_step(c->p.storage, c->state, c->g, c->p.variant, c->p.kernel);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < c->p.graph_steps && le == cudaSuccess; ++i)
      le = flame::launch_step(c->p.storage, parity ^ (i & 1), c->state, c->g, c->k, c->d_flags, cs, c->p.variant,
                              c->d_bfield, c->p.kernel);
    e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[parity], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e == cudaSuccess) c->has_graph[parity] = true;
  return e;
}

flame_status flame_step(flame_ctx* c, int n) {
  const Range range("flame_step");
  flame_status st = usable(c);
  if (st != FLAME_OK) return st;
  if (n < 0) return FLAME_ERR_PARAM;
  if (c->stall_tries && n > 0) {
    // The wait-failure test: one launch whose waits all run out; it leaves
    // the state as it was, so step and parity do not advance.
    cudaError_t e = flame::launch_step_row(c->p.storage, c->parity, c->state, c->g, c->k, c->d_flags, c->stream,
                                           c->p.variant, c->d_bfield, c->stall_tries, c->p.kernel);
    c->stall_tries = 0;
    if (e != cudaSuccess) return cuda_fail(c, e);
    return sync_and_check(c);
  }
  if (!c->initialized) return FLAME_ERR_STATE;
  const int G = c->p.graph_steps;
  while (G > 0 && n >= G) {
    if (!c->has_graph[c->parity]) {
      cudaError_t e = capture_graph(c, c->parity);
      if (e != cudaSuccess) return cuda_fail(c, e);
    }
    cudaError_t e = cudaGraphLaunch(c->graph[c->parity], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    const long long before = c->step;
    c->step += G;
    n -= G;
    if (c->p.check_every > 0 && c->step / c->p.check_every != before / c->p.check_every) {
      st = sync_and_check(c);
      if (st != FLAME_OK) return st;
    }
  }
  for (int i = 0; i < n; ++i) {
    cudaError_t e = flame::launch_step(c->p.storage, c->parity, c->state, c->g, c->k, c->d_flags, c->stream,
                                       c->p.variant, c->d_bfield, c->p.kernel);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->parity ^= 1;
    ++c->step;
    if (c->p.check_every > 0 && c->step % c->p.check_every == 0) {
      st = sync_and_check(c);
      if (st != FLAME_OK) return st;
    }
  }
  return FLAME_OK;
}

flame_status flame_sync(flame_ctx* c) {
  if (!c) return FLAME_ERR_PARAM;
  if (c->sticky == FLAME_ERR_CUDA) return c->sticky;
  return sync_and_check(c);
}

flame_status flame_info(flame_ctx* c, flame_info_t* out) {
  if (!c || !out) return FLAME_ERR_PARAM;
  out->step = c->step;
  out->parity = c->parity;
  out->nonfinite = c->nonfinite;
  out->cfl = c->cfl;
  out->max_speed = c->max_speed;
  return FLAME_OK;
}

flame_status flame_moments(flame_ctx* c, double* d_rho, double* d_u, double* d_B, double* d_J) {
  const Range range("flame_moments");
  flame_status st = usable(c);
  if (st != FLAME_OK && st != FLAME_ERR_NONFINITE) return st;
  if (!c->initialized) return FLAME_ERR_STATE;
  return cuda_fail(c, flame::launch_moments(c->p.storage, c->parity, c->state, c->g, c->k, d_rho, d_u, d_B, d_J,
                                            c->stream));
}

flame_status flame_moments_f32(flame_ctx* c, float* d_rho, float* d_u, float* d_B, float* d_J) {
  const Range range("flame_moments_f32");
  flame_status st = usable(c);
  if (st != FLAME_OK && st != FLAME_ERR_NONFINITE) return st;
  if (!c->initialized) return FLAME_ERR_STATE;
  return cuda_fail(c, flame::launch_moments_f32(c->p.storage, c->parity, c->state, c->g, c->k, d_rho, d_u, d_B,
                                                d_J, c->stream));
}

flame_status flame_populations(flame_ctx* c, double* d_f) {
  const Range range("flame_populations");
  flame_status st = usable(c);
  if (st != FLAME_OK && st != FLAME_ERR_NONFINITE) return st;
  if (!c->initialized) return FLAME_ERR_STATE;
  if (!d_f) return FLAME_ERR_PARAM;
  return cuda_fail(c, flame::launch_populations(c->p.storage, c->parity, c->state, c->g, c->k, d_f, c->stream));
}

flame_status flame_probe(flame_ctx* c, int nsites, const long long* d_sites, double* d_out) {
  const Range range("flame_probe");
  flame_status st = usable(c);
  if (st != FLAME_OK && st != FLAME_ERR_NONFINITE) return st;
  if (!c->initialized) return FLAME_ERR_STATE;
  if (nsites < 0 || (nsites > 0 && (!d_sites || !d_out))) return FLAME_ERR_PARAM;
  return cuda_fail(c, flame::launch_probe(c->p.storage, c->parity, c->state, c->g, c->k, nsites, d_sites, d_out,
                                          c->stream));
}

// The raw FP64 sums of the reduction over the context's sites (FLAME_NSUMS
// entries: the kRedVals partial sums, then the site count).
static flame_status reduce_raw(flame_ctx* c, double* r) {
  flame_status st = usable(c);
  if (st != FLAME_OK && st != FLAME_ERR_NONFINITE) return st;
  if (!c->initialized) return FLAME_ERR_STATE;
  cudaError_t e;
  if (!c->d_red) {
    e = cudaMalloc(&c->d_red, sizeof(double) * (size_t)(flame::kRedBlocksMax + 1) * flame::kRedVals);
    if (e != cudaSuccess) {
      c->d_red = nullptr;
      return cuda_fail(c, e);
    }
  }
  const int nb = reduce_blocks(c);
  double* out = c->d_red + (size_t)flame::kRedBlocksMax * flame::kRedVals;
  e = flame::launch_reduce(c->p.storage, c->parity, c->state, c->g, c->k, nb, c->d_red, out, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  e = cudaMemcpyAsync(r, out, sizeof(double) * flame::kRedVals, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  r[FLAME_SUM_SITES] = (double)c->g.n3i;
  return FLAME_OK;
}

static_assert(flame::kIoChunks == FLAME_IO_CHUNKS, "the chunk limit the header states");
static_assert(flame::kRedVals == FLAME_SUM_SITES, "the reduction's partial sums precede the site count");

flame_status flame_reduce_sums(flame_ctx* c, double* h) {
  const Range range("flame_reduce_sums");
  if (!h) return FLAME_ERR_PARAM;
  flame_status st = reduce_raw(c, h);
  if (st != FLAME_OK) return st;
  return h[FLAME_SUM_NONFINITE] > 0 ? FLAME_ERR_NONFINITE : FLAME_OK;
}

int flame_step_kernel(const flame_params* p) {
  if (check_params(p) != FLAME_OK) return 0;
  flame::Grid g{};
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz + 2 * p->halo_z;
  g.n3 = (long long)p->nx * p->ny * g.nz;
  g.z0 = p->halo_z;
  g.nzi = p->nz;
  g.n3i = (long long)p->nx * p->ny * p->nz;
  // flame_create requires a 256-byte aligned state; only the alignment is
  // looked at
  const void* aligned = reinterpret_cast<const void*>(static_cast<uintptr_t>(256));
  if (!flame::step_row_supported(g, p->storage, p->variant, aligned, p->kernel)) return FLAME_KERNEL_SITE;
  switch (flame::row_segments(g.nx, p->kernel)) {
    case 0: return FLAME_KERNEL_PAIRS;
    case 2: return FLAME_KERNEL_HALF_ROWS;
  }
  return FLAME_KERNEL_ROWS;
}

int flame_reduce_combine(const flame_params* p, const double* r, double* h) {
  if (!p || !r || !h || !(r[FLAME_SUM_SITES] > 0)) return -1;
  const double n3 = r[FLAME_SUM_SITES];
  double Bm[3];
  h[FLAME_S_MASS] = r[FLAME_SUM_RHO];
  for (int a = 0; a < 3; ++a) {
    h[FLAME_S_MOMX + a] = r[FLAME_SUM_MOMX + a];
    Bm[a] = r[FLAME_SUM_BX + a] / n3;
    h[FLAME_S_BX + a] = Bm[a];
  }
  h[FLAME_S_EU] = 0.5 * r[FLAME_SUM_U2] / n3;
  // E_B and H_c about the mean field: the sums are taken about B_ref
  double dbm2 = 0.0, hc_corr = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double d = Bm[a] - p->B_ref[a];
    dbm2 += d * d;
    hc_corr += (r[FLAME_SUM_UX + a] / n3) * d;
  }
  h[FLAME_S_EB] = 0.5 * (r[FLAME_SUM_DB2] / n3 - dbm2);
  h[FLAME_S_HC] = r[FLAME_SUM_UDB] / n3 - hc_corr;
  h[FLAME_S_J2] = r[FLAME_SUM_J2] / n3;
  h[FLAME_S_UMAX] = r[FLAME_SUM_UMAX];
  h[FLAME_S_DIVB] = std::sqrt(r[FLAME_SUM_DIV2] / n3);
  h[FLAME_S_NONFINITE] = r[FLAME_SUM_NONFINITE];
  return 0;
}

flame_status flame_reduce(flame_ctx* c, double* h) {
  const Range range("flame_reduce");
  if (!h) return FLAME_ERR_PARAM;
  double r[FLAME_NSUMS];
  flame_status st = reduce_raw(c, r);
  if (st != FLAME_OK) return st;
  flame_reduce_combine(&c->p, r, h);
  return r[FLAME_SUM_NONFINITE] > 0 ? FLAME_ERR_NONFINITE : FLAME_OK;
}

// The field workspace: 6 fft_stride(N3) doubles, allocated on first use.
static cudaError_t fields_ws(flame_ctx* c) {
  if (c->d_fields) return cudaSuccess;
  const cudaError_t e = cudaMalloc(&c->d_fields, 6 * (size_t)flame::fft_stride(c->g.n3) * sizeof(double));
  if (e != cudaSuccess) c->d_fields = nullptr;
  return e;
}

// ---------------------------------------------------------------------------
// Host-buffer calls: the fields move between host and device in chunks of z
// planes on a second stream, each chunk's kernel running as soon as its data
// is there, so that the copies over the host link overlap the kernels.

// The copy stream and events, created on first use, and the field workspace.
static cudaError_t io_ready(flame_ctx* c) {
  cudaError_t e = fields_ws(c);
  if (e == cudaSuccess && !c->has_io_stream) {
    e = cudaStreamCreateWithFlags(&c->io_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) c->has_io_stream = true;
  }
  while (e == cudaSuccess && c->n_io_ev < flame::kIoChunks + 1) {
    e = cudaEventCreateWithFlags(&c->io_ev[c->n_io_ev], cudaEventDisableTiming);
    if (e == cudaSuccess) ++c->n_io_ev;
  }
  if (e == cudaSuccess && c->io_max_pitch == 0) {
    int mp = 0;
    e = cudaDeviceGetAttribute(&mp, cudaDevAttrMaxPitch, c->device);
    c->io_max_pitch = e == cudaSuccess && mp > 0 ? (size_t)mp : 0;
  }
  return e;
}

// Elements [off, off + count) of each of ncomp components `stride` apart:
// one 2-D copy (a row per component) where the stride is within the
// device's pitch limit -- each copy over the host link carries a fixed
// cost, so fewer and larger copies move more -- else one copy per component.
static cudaError_t copy_comps(float* dst, const float* src, int ncomp, long long stride, long long off,
                              long long count, cudaMemcpyKind kind, cudaStream_t s, size_t max_pitch) {
  const size_t pitch = (size_t)stride * sizeof(float);
  if (ncomp > 1 && pitch <= max_pitch)
    return cudaMemcpy2DAsync(dst + off, pitch, src + off, pitch, (size_t)count * sizeof(float), (size_t)ncomp, kind,
                             s);
  for (int a = 0; a < ncomp; ++a) {
    const cudaError_t e =
        cudaMemcpyAsync(dst + a * stride + off, src + a * stride + off, (size_t)count * sizeof(float), kind, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// A field of a host-buffer call: its host array, its place in the workspace
// and its components (`stride` apart in both).
struct IoField {
  float* h;
  float* d;
  int ncomp;
};

// Drops the fields without a host array and merges each field that follows
// the previous one both in host memory and in the workspace into it, so that
// fields the caller keeps in one array move in one copy.  Returns the count.
static int io_merge(IoField* f, int n, long long stride) {
  const auto follows = [stride](const float* p, int ncomp, const float* q) {
    return reinterpret_cast<uintptr_t>(p) + (uintptr_t)ncomp * (uintptr_t)stride * sizeof(float) ==
           reinterpret_cast<uintptr_t>(q);
  };
  int m = 0;
  for (int i = 0; i < n; ++i) {
    if (!f[i].h) continue;
    if (m > 0 && follows(f[m - 1].h, f[m - 1].ncomp, f[i].h) && follows(f[m - 1].d, f[m - 1].ncomp, f[i].d)) {
      f[m - 1].ncomp += f[i].ncomp;
      continue;
    }
    f[m++] = f[i];
  }
  return m;
}

flame_status flame_init_f32_host(flame_ctx* c, const float* h_rho, const float* h_u, const float* h_B) {
  const Range range("flame_init_f32_host");
  if (!c) return FLAME_ERR_PARAM;
  if (c->sticky == FLAME_ERR_CUDA) return c->sticky;
  if (!c->state) return FLAME_ERR_STATE;
  if (!h_u || !h_B) return FLAME_ERR_PARAM;
  const cudaError_t er = io_ready(c);
  if (er != cudaSuccess) return cuda_fail(c, er);
  const flame::Grid g = c->g;
  const long long n3 = g.n3, plane = (long long)g.nx * g.ny;
  float* d_u = reinterpret_cast<float*>(c->d_fields);
  float* d_B = d_u + 3 * n3;
  float* d_rho = h_rho ? d_u + 6 * n3 : nullptr;
  // the host arrays are only read (the copies run host to device)
  IoField f[3] = {{const_cast<float*>(h_u), d_u, 3}, {const_cast<float*>(h_B), d_B, 3},
                  {const_cast<float*>(h_rho), d_rho, 1}};
  const int nf = io_merge(f, 3, n3);
  // the planes held are copied in nc chunks, the updated planes initialised in ni
  const int nc = flame::io_chunk_count(g.nz), ni = flame::io_chunk_count(g.nzi);
  const flame_status st = init_with(c, [&]() -> cudaError_t {
    // the copies overwrite the workspace only after the work queued before
    cudaError_t e = cudaEventRecord(c->io_ev[flame::kIoChunks], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->io_stream, c->io_ev[flame::kIoChunks], 0);
    int queued = 0;
    for (int j = 0; j < nc && e == cudaSuccess; ++j) {
      const int a = flame::io_first(0, g.nz, nc, j), b = flame::io_first(0, g.nz, nc, j + 1);
      const long long off = a * plane, cnt = (b - a) * plane;
      for (int k = 0; k < nf && e == cudaSuccess; ++k)
        e = copy_comps(f[k].d, f[k].h, f[k].ncomp, n3, off, cnt, cudaMemcpyHostToDevice, c->io_stream,
                       c->io_max_pitch);
      if (e == cudaSuccess) e = cudaEventRecord(c->io_ev[j], c->io_stream);
      // every chunk of updated planes whose planes and z neighbours have now arrived
      for (int i = 0; i < ni && e == cudaSuccess; ++i) {
        const int ia = flame::io_first(g.z0, g.nzi, ni, i), ib = flame::io_first(g.z0, g.nzi, ni, i + 1);
        if (flame::io_init_needs(g.nz, nc, ia, ib) != j) continue;
        flame::Grid sg = g;
        sg.z0 = ia;
        sg.nzi = ib - ia;
        sg.n3i = plane * (ib - ia);
        e = cudaStreamWaitEvent(c->stream, c->io_ev[j], 0);
        if (e == cudaSuccess)
          e = flame::launch_init_f32(c->p.storage, c->state, sg, c->k, c->p.init_noneq, d_rho, d_u, d_B, nullptr,
                                     nullptr, c->d_flags + 1, c->stream);
        ++queued;
      }
    }
    if (e == cudaSuccess && queued != ni) e = cudaErrorInvalidValue;
    return e;
  });
  // no copy from the caller's buffers is in flight after the return
  const cudaError_t es = cudaStreamSynchronize(c->io_stream);
  if (st == FLAME_OK && es != cudaSuccess) return cuda_fail(c, es);
  return st;
}

flame_status flame_moments_f32_host(flame_ctx* c, float* h_rho, float* h_u, float* h_B, float* h_J,
                                    double* h_scalars) {
  const Range range("flame_moments_f32_host");
  const flame_status su = usable(c);
  if (su != FLAME_OK && su != FLAME_ERR_NONFINITE) return su;
  if (!c->initialized) return FLAME_ERR_STATE;
  cudaError_t e = io_ready(c);
  if (e != cudaSuccess) return cuda_fail(c, e);
  const flame::Grid g = c->g;
  const long long n3i = g.n3i, plane = (long long)g.nx * g.ny;
  // the requested fields, one after another in the workspace, components n3i apart
  float* w = reinterpret_cast<float*>(c->d_fields);
  float* d_rho = h_rho ? w : nullptr;
  w += h_rho ? n3i : 0;
  float* d_u = h_u ? w : nullptr;
  w += h_u ? 3 * n3i : 0;
  float* d_B = h_B ? w : nullptr;
  w += h_B ? 3 * n3i : 0;
  float* d_J = h_J ? w : nullptr;
  IoField f[4] = {{h_rho, d_rho, 1}, {h_u, d_u, 3}, {h_B, d_B, 3}, {h_J, d_J, 3}};
  const int nf = io_merge(f, 4, n3i);
  const int n = flame::io_chunk_count(g.nzi);
  for (int j = 0; j < n && e == cudaSuccess; ++j) {
    const int a = flame::io_first(g.z0, g.nzi, n, j), b = flame::io_first(g.z0, g.nzi, n, j + 1);
    const long long off = (a - g.z0) * plane;
    flame::Grid sg = g;
    sg.z0 = a;
    sg.nzi = b - a;
    sg.n3i = plane * (b - a);
    e = flame::launch_moments_f32(c->p.storage, c->parity, c->state, sg, c->k, d_rho ? d_rho + off : nullptr,
                                  d_u ? d_u + off : nullptr, d_B ? d_B + off : nullptr, d_J ? d_J + off : nullptr,
                                  c->stream, n3i);
    if (e == cudaSuccess) e = cudaEventRecord(c->io_ev[j], c->stream);
  }
  for (int j = 0; j < n && e == cudaSuccess; ++j) {
    const int a = flame::io_first(g.z0, g.nzi, n, j), b = flame::io_first(g.z0, g.nzi, n, j + 1);
    const long long off = (a - g.z0) * plane, cnt = (b - a) * plane;
    e = cudaStreamWaitEvent(c->io_stream, c->io_ev[j], 0);
    for (int k = 0; k < nf && e == cudaSuccess; ++k)
      e = copy_comps(f[k].h, f[k].d, f[k].ncomp, n3i, off, cnt, cudaMemcpyDeviceToHost, c->io_stream,
                     c->io_max_pitch);
  }
  flame_status st = FLAME_OK;
  if (e == cudaSuccess && h_scalars) {
    // the scalars of the same state, on the context's stream while the fields are copied out
    double r[FLAME_NSUMS];
    st = reduce_raw(c, r);
    if (st == FLAME_OK) {
      flame_reduce_combine(&c->p, r, h_scalars);
      if (r[FLAME_SUM_NONFINITE] > 0) st = FLAME_ERR_NONFINITE;
    }
  }
  const cudaError_t es = cudaStreamSynchronize(c->io_stream);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(c, e);
  return st;
}

// Shell spectra of the state's u, B (d_u = d_B = null) or of given FP64
// fields [3][N3] each.
static flame_status spectra_of(flame_ctx* c, int nshell, const double* d_u, const double* d_B, double* h_Eu,
                               double* h_Eb) {
  flame_status st = usable(c);
  if (st != FLAME_OK && st != FLAME_ERR_NONFINITE) return st;
  if (c->p.halo_z) return FLAME_ERR_PARAM;  // a slab holds only part of the spectrum's lattice
  if (!d_u && !c->initialized) return FLAME_ERR_STATE;
  if (nshell < 1 || nshell > 4096) return FLAME_ERR_PARAM;  // shell histogram lives in shared memory
  cudaError_t e;
  const size_t n3 = (size_t)flame::fft_stride(c->g.n3);  // aligned stride between the six fields
  const size_t nc = (size_t)c->g.nz * c->g.ny * (c->g.nx / 2 + 1);
  e = fields_ws(c);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (!c->d_spec) {
    e = cudaMalloc(&c->d_spec, nc * sizeof(cufftDoubleComplex));
    if (e != cudaSuccess) {
      c->d_spec = nullptr;
      return cuda_fail(c, e);
    }
  }
  if (nshell > c->nshell_cap) {
    cudaFree(c->d_shells);
    c->d_shells = nullptr;
    e = cudaMalloc(&c->d_shells, 2 * (size_t)nshell * sizeof(double));
    if (e != cudaSuccess) {
      c->nshell_cap = 0;
      return cuda_fail(c, e);
    }
    c->nshell_cap = nshell;
  }
  if (!c->has_plan) {
    if (cufftPlan3d(&c->plan, c->g.nz, c->g.ny, c->g.nx, CUFFT_D2Z) != CUFFT_SUCCESS) return cuda_fail(c, cudaErrorUnknown);
    c->has_plan = true;
  }
  if (cufftSetStream(c->plan, c->stream) != CUFFT_SUCCESS) return cuda_fail(c, cudaErrorUnknown);
  double* u = c->d_fields;
  double* B = c->d_fields + 3 * n3;
  if (!d_u) {
    e = flame::launch_moments(c->p.storage, c->parity, c->state, c->g, c->k, nullptr, u, B, nullptr, c->stream,
                              (long long)n3);
  } else {
    // each component to its aligned place in the workspace (cuFFT input)
    const size_t row = (size_t)c->g.n3 * sizeof(double);
    e = cudaMemcpy2DAsync(u, n3 * sizeof(double), d_u, row, row, 3, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(B, n3 * sizeof(double), d_B, row, row, 3, cudaMemcpyDeviceToDevice, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_shells, 0, 2 * (size_t)nshell * sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  for (int f = 0; f < 6; ++f) {
    double* src = c->d_fields + (size_t)f * n3;
    if (cufftExecD2Z(c->plan, src, static_cast<cufftDoubleComplex*>(c->d_spec)) != CUFFT_SUCCESS)
      return cuda_fail(c, cudaErrorUnknown);
    e = flame::launch_shell_bin(c->d_spec, c->g, nshell, f >= 3, c->d_shells + (f >= 3 ? nshell : 0), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
  }
  double* tmp = static_cast<double*>(std::malloc(2 * (size_t)nshell * sizeof(double)));
  if (!tmp) return FLAME_ERR_PARAM;
  e = cudaMemcpyAsync(tmp, c->d_shells, 2 * (size_t)nshell * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    std::free(tmp);
    return cuda_fail(c, e);
  }
  for (int i = 0; i < nshell; ++i) {
    if (h_Eu) h_Eu[i] = 0.5 * tmp[i];
    if (h_Eb) h_Eb[i] = 0.5 * tmp[nshell + i];
  }
  std::free(tmp);
  return FLAME_OK;
}

flame_status flame_spectra(flame_ctx* c, int nshell, double* h_Eu, double* h_Eb) {
  const Range range("flame_spectra");
  return spectra_of(c, nshell, nullptr, nullptr, h_Eu, h_Eb);
}

flame_status flame_spectra_fields(flame_ctx* c, int nshell, const double* d_u, const double* d_B, double* h_Eu,
                                  double* h_Eb) {
  const Range range("flame_spectra_fields");
  if (!c || !d_u || !d_B) return FLAME_ERR_PARAM;
  return spectra_of(c, nshell, d_u, d_B, h_Eu, h_Eb);
}

flame_status flame_get_state(flame_ctx* c, void* d_dst, long long* step, int* parity) {
  if (!c || !d_dst) return FLAME_ERR_PARAM;
  if (c->sticky == FLAME_ERR_CUDA) return c->sticky;
  if (!c->initialized) return FLAME_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(d_dst, c->state, flame_state_bytes(&c->p), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (step) *step = c->step;
  if (parity) *parity = c->parity;
  return FLAME_OK;
}

flame_status flame_set_state(flame_ctx* c, const void* d_src, long long step, int parity) {
  if (!c || !d_src) return FLAME_ERR_PARAM;
  if (c->sticky == FLAME_ERR_CUDA) return c->sticky;
  if (!c->state || (parity != 0 && parity != 1) || step < 0) return FLAME_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(c->state, d_src, flame_state_bytes(&c->p), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  e = cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  c->sticky = FLAME_OK;
  c->nonfinite = 0;
  c->step = step;
  c->parity = parity;
  c->initialized = true;
  return FLAME_OK;
}

flame_status flame_step_adjoint(flame_ctx* c, const void* d_state, int parity, const float* d_adj_in,
                                float* d_adj_out, double* d_ddi) {
  const Range range("flame_step_adjoint");
  if (!c || !d_state || !d_adj_in || !d_adj_out || !d_ddi) return FLAME_ERR_PARAM;
  if (c->p.variant != FLAME_SCHEME || c->p.halo_z) return FLAME_ERR_PARAM;
  if (c->sticky == FLAME_ERR_CUDA) return c->sticky;
  if (parity != 0 && parity != 1) return FLAME_ERR_STATE;
  if (d_adj_in == d_adj_out) return FLAME_ERR_PARAM;
  cudaError_t e;
  if (!c->d_adj_partials) {
    e = cudaMalloc(&c->d_adj_partials, sizeof(double) * (size_t)flame::adjoint_partials_needed(c->g));
    if (e != cudaSuccess) {
      c->d_adj_partials = nullptr;
      return cuda_fail(c, e);
    }
  }
  return cuda_fail(c, flame::launch_step_adjoint(c->p.storage, parity, d_state, c->g, c->k, d_adj_in, d_adj_out,
                                                 c->d_adj_partials, d_ddi, c->stream));
}

flame_status flame_init_adjoint(flame_ctx* c, const double* d_u, const double* d_B, const float* d_adj0,
                                double* d_ubar, double* d_Bbar, double* d_ddi) {
  const Range range("flame_init_adjoint");
  if (!c || !d_u || !d_B || !d_adj0 || !d_ddi || (!d_ubar && !d_Bbar)) return FLAME_ERR_PARAM;
  if (c->p.variant != FLAME_SCHEME || c->p.halo_z) return FLAME_ERR_PARAM;
  if (c->sticky == FLAME_ERR_CUDA) return c->sticky;
  cudaError_t e;
  if (!c->d_adj_partials) {
    e = cudaMalloc(&c->d_adj_partials, sizeof(double) * (size_t)flame::adjoint_partials_needed(c->g));
    if (e != cudaSuccess) {
      c->d_adj_partials = nullptr;
      return cuda_fail(c, e);
    }
  }
  if (!c->d_adj_ws) {
    e = cudaMalloc(&c->d_adj_ws, sizeof(double) * 24 * (size_t)c->g.n3);
    if (e != cudaSuccess) {
      c->d_adj_ws = nullptr;
      return cuda_fail(c, e);
    }
  }
  return cuda_fail(c, flame::launch_init_adjoint(c->g, c->k, d_u, d_B, d_adj0, c->d_adj_ws, c->d_adj_partials,
                                                 d_ubar, d_Bbar, d_ddi, c->stream));
}

int flame_halo_plan(const flame_params* p, int parity, int face, flame_halo_run send[2], flame_halo_run recv[2]) {
  if (!p || !p->halo_z || p->nz < 1 || (parity != 0 && parity != 1) || (face != 0 && face != 1) || !send || !recv)
    return -1;
  // Storage slots of the populations moving down (c_z = -1: fluid slots
  // 0..8 of the velocity cube, magnetic D3Q7 velocity -z) and up (c_z = +1:
  // fluid 18..26, magnetic +z).  The face towards z - 1 trades the ones that
  // cross it: down-movers arrive in the lower ghost plane, up-movers leave
  // the first plane; through the face towards z + 1 the reverse.
  const int down_f = 0, up_f = 18, down_m = flame::kQ + 3 * 6, up_m = flame::kQ + 3 * 5;
  const int lo_ghost = 0, first = 1, last = p->nz, hi_ghost = p->nz + 1;
  auto set = [](flame_halo_run* r, int f, int m, int plane) {
    r[0] = flame_halo_run{f, 9, plane};
    r[1] = flame_halo_run{m, 3, plane};
  };
  if (parity == 1) {
    // before an odd step: ghost planes receive the neighbours' boundary slots
    if (face == 0) {
      set(send, up_f, up_m, first);
      set(recv, down_f, down_m, lo_ghost);
    } else {
      set(send, down_f, down_m, last);
      set(recv, up_f, up_m, hi_ghost);
    }
  } else {
    // after an odd step: what it wrote into the ghost planes goes back
    if (face == 0) {
      set(send, down_f, down_m, lo_ghost);
      set(recv, up_f, up_m, first);
    } else {
      set(send, up_f, up_m, hi_ghost);
      set(recv, down_f, down_m, last);
    }
  }
  return 0;
}

flame_status flame_halo_exchange(flame_ctx* lo, flame_ctx* up) {
  const Range range("flame_halo_exchange");
  if (!lo || !up) return FLAME_ERR_PARAM;
  if (!lo->p.halo_z || !up->p.halo_z || lo->p.nx != up->p.nx || lo->p.ny != up->p.ny ||
      lo->p.storage != up->p.storage)
    return FLAME_ERR_PARAM;
  if (lo->sticky == FLAME_ERR_CUDA) return lo->sticky;
  if (up->sticky == FLAME_ERR_CUDA) return up->sticky;
  if (!lo->initialized || !up->initialized || lo->parity != up->parity) return FLAME_ERR_STATE;
  const size_t eb = elem_bytes(lo->p.storage);
  const size_t plane = (size_t)lo->g.nx * lo->g.ny;
  // through the face between them: lower's face 1 with upper's face 0
  flame_halo_run ls[2], lr[2], us[2], ur[2];
  flame_halo_plan(&lo->p, lo->parity, 1, ls, lr);
  flame_halo_plan(&up->p, up->parity, 0, us, ur);
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
    // lower -> upper, then upper -> lower; one strided copy per run
    char* ubase = static_cast<char*>(up->state);
    char* lbase = static_cast<char*>(lo->state);
    e = cudaMemcpy2DAsync(ubase + ((size_t)ur[r].first_slot * up->g.n3 + ur[r].plane * plane) * eb, up->g.n3 * eb,
                          lbase + ((size_t)ls[r].first_slot * lo->g.n3 + ls[r].plane * plane) * eb, lo->g.n3 * eb,
                          plane * eb, ls[r].nslots, cudaMemcpyDeviceToDevice, lo->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(lbase + ((size_t)lr[r].first_slot * lo->g.n3 + lr[r].plane * plane) * eb, lo->g.n3 * eb,
                            ubase + ((size_t)us[r].first_slot * up->g.n3 + us[r].plane * plane) * eb, up->g.n3 * eb,
                            plane * eb, us[r].nslots, cudaMemcpyDeviceToDevice, lo->stream);
  }
  return cuda_fail(lo, e);
}

flame_status flame_debug_stall_next_step(flame_ctx* c, unsigned tries) {
  flame_status st = usable(c);
  if (st != FLAME_OK) return st;
  if (!c->initialized) return FLAME_ERR_STATE;
  if (tries == 0 || !flame::step_row_staged(c->g, c->p.storage, c->p.variant, c->state, c->p.kernel))
    return FLAME_ERR_PARAM;
  c->stall_tries = tries;
  return FLAME_OK;
}

void flame_destroy(flame_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->has_plan) cufftDestroy(c->plan);
  for (int p = 0; p < 2; ++p)
    if (c->has_graph[p]) cudaGraphExecDestroy(c->graph[p]);
  cudaFree(c->d_flags);
  cudaFree(c->d_red);
  cudaFree(c->d_fields);
  cudaFree(c->d_spec);
  cudaFree(c->d_shells);
  cudaFree(c->d_adj_partials);
  cudaFree(c->d_adj_ws);
  cudaFree(c->d_bfield);
  flame::spectral_ws_free(c->spectral);
  for (int j = 0; j < c->n_io_ev; ++j) cudaEventDestroy(c->io_ev[j]);
  if (c->has_io_stream) cudaStreamDestroy(c->io_stream);
  delete c;
}

const char* flame_status_string(flame_status s) {
  switch (s) {
    case FLAME_OK: return "ok";
    case FLAME_ERR_PARAM: return "invalid parameter";
    case FLAME_ERR_CFL: return "whistler CFL condition violated";
    case FLAME_ERR_NONFINITE: return "non-finite value in the state";
    case FLAME_ERR_CUDA: return "CUDA error";
    case FLAME_ERR_STATE: return "inconsistent state or call order";
    case FLAME_ERR_TIMEOUT: return "a device-side wait exceeded its limit";
  }
  return "unknown status";
}

int flame_lattice(int* c27, int* xi7) {
  for (int i = 0; i < flame::kQ; ++i) {
    if (c27) {
      c27[3 * i + 0] = flame::cx27(i);
      c27[3 * i + 1] = flame::cy27(i);
      c27[3 * i + 2] = flame::cz27(i);
    }
  }
  for (int i = 0; i < flame::kM; ++i) {
    if (xi7) {
      xi7[3 * i + 0] = flame::mx7(i);
      xi7[3 * i + 1] = flame::my7(i);
      xi7[3 * i + 2] = flame::mz7(i);
    }
  }
  return 0;
}

}  // extern "C"
