// reduce_static.cu -- flame_reduce_static: the FP64 scalar diagnostics of
// flame_reduce computed without allocating any memory.
//
// Who needs this: callers that must not call cudaMalloc.  flame_reduce
// allocates its workspace with cudaMalloc on its first call, and cudaMalloc
// may synchronise the device, so it stalls work that is already queued.
// Hosts that give a framework's caching allocator every byte of device
// memory, or that run under a fixed memory budget, may not be able to let
// a library allocate at all.  This variant keeps its scratch in a fixed-size
// device array that exists from the moment the library is loaded, so a
// call queues kernels and nothing else.
//
// The scratch is one array per device, shared by every context on that
// device and kept between calls.  Each call overwrites the per-block
// partial sums it later reads, so no entry has to start at zero.  Two calls
// that overlap on the GPU (different streams, or different contexts on one
// device) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "flame.h"
#include "flame_internal.h"

namespace {

// Per-block partial sums: FLAME_STATIC_REDUCE_BLOCKS_MAX blocks of
// kRedVals doubles, 139,264 bytes per device that loads the library.
static __device__ __align__(256) double g_reduce_scratch[FLAME_STATIC_REDUCE_BLOCKS_MAX * flame::kRedVals];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices];  // device address of g_reduce_scratch, per device

// Set-up, once per device, with that device current: the device address of
// the scratch array.  In host code `g_reduce_scratch` names a host-side
// stand-in, never a usable device address.
cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

// Sum the partials in a fixed order and turn the raw sums into the
// FLAME_S_* scalars (the same formulas flame_reduce applies on the host).
__global__ void finalize_kernel(const double* __restrict__ partials, int nblocks, double n3, double br0, double br1,
                                double br2, double* __restrict__ out) {
  __shared__ double r[flame::kRedVals];
  const int v = threadIdx.x;
  if (v < flame::kRedVals) {
    double a = partials[v];
    for (int b = 1; b < nblocks; ++b) {
      const double t = partials[(long long)b * flame::kRedVals + v];
      a = (v == 14) ? fmax(a, t) : a + t;
    }
    r[v] = a;
  }
  __syncthreads();
  if (v != 0) return;
  const double br[3] = {br0, br1, br2};
  double bm[3], dbm2 = 0.0, hc_corr = 0.0;
  out[FLAME_S_MASS] = r[0];
  for (int a = 0; a < 3; ++a) {
    out[FLAME_S_MOMX + a] = r[1 + a];
    bm[a] = r[4 + a] / n3;
    out[FLAME_S_BX + a] = bm[a];
    const double d = bm[a] - br[a];
    dbm2 += d * d;
    hc_corr += (r[10 + a] / n3) * d;
  }
  out[FLAME_S_EU] = 0.5 * r[7] / n3;
  out[FLAME_S_EB] = 0.5 * (r[8] / n3 - dbm2);
  out[FLAME_S_HC] = r[9] / n3 - hc_corr;
  out[FLAME_S_J2] = r[13] / n3;
  out[FLAME_S_UMAX] = r[14];
  out[FLAME_S_DIVB] = sqrt(r[15] / n3);
  out[FLAME_S_NONFINITE] = r[16];
}

}  // namespace

extern "C" flame_status flame_reduce_static(flame_ctx* ctx, int nblocks, double* d_scalars) {
  flame::CtxView v;
  if (flame_ctx_view(ctx, &v) != 0 || !d_scalars) return FLAME_ERR_PARAM;
  if (v.status != FLAME_OK && v.status != FLAME_ERR_NONFINITE) return static_cast<flame_status>(v.status);
  if (!v.initialized) return FLAME_ERR_STATE;
  if (nblocks < 0 || nblocks > FLAME_STATIC_REDUCE_BLOCKS_MAX) return FLAME_ERR_PARAM;
  if (nblocks == 0) {
    long long want = (long long)v.nsm * 4;
    const long long per = (v.g.n3i + 255) / 256;
    if (want > per) want = per;
    if (want > FLAME_STATIC_REDUCE_BLOCKS_MAX) want = FLAME_STATIC_REDUCE_BLOCKS_MAX;
    nblocks = want < 1 ? 1 : (int)want;
  }
  // failures are recorded in the context's sticky status, as in flame_reduce
  double* scratch = nullptr;
  cudaError_t e = scratch_address(v.device, &scratch);
  if (e != cudaSuccess) return static_cast<flame_status>(flame_ctx_cuda_fail(ctx, e));
  e = flame::launch_reduce_partials(v.storage, v.parity, v.state, v.g, v.k, nblocks, scratch, v.stream);
  if (e != cudaSuccess) return static_cast<flame_status>(flame_ctx_cuda_fail(ctx, e));
  finalize_kernel<<<1, 32, 0, v.stream>>>(scratch, nblocks, (double)v.g.n3i, v.Bref[0], v.Bref[1], v.Bref[2],
                                          d_scalars);
  return static_cast<flame_status>(flame_ctx_cuda_fail(ctx, cudaGetLastError()));
}
