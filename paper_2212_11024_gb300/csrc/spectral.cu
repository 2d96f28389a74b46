// spectral.cu -- Fourier-space diagnostics behind the C ABI (Sec. 4.4):
//  - flame_band_energy: the magnetic energy in a band of spectral shells and
//    its gradient with respect to B, the loss of the differentiable runs;
//  - flame_energy_budget: the wavenumber-by-wavenumber energy budget, the
//    flux S_MHD(k) and the dissipation D(k) of eq. mhd_en_trans.
//
// Conventions (those of flame_spectra): F(f) = N3^-1 sum_x f(x) exp(-i k.x),
// k = 2 pi m / N per axis, shell n = round(|m|).  Derivatives are spectral,
// with the Nyquist wavenumber of an even axis set to zero.  Everything is
// FP64: cuFFT D2Z / Z2D transforms (unnormalised; the factors of N3 are
// applied in the kernels below) and FP64 shell sums in shared memory.
#include <cufft.h>

#include <cmath>
#include <cstring>
#include <new>

#include "flame.h"
#include "flame_internal.h"

namespace flame {

// Per-context workspace: real fields of N3 doubles and half spectra of
// H = nz * ny * (nx/2 + 1) complex values, grown on demand.
struct SpectralWs {
  Grid g;
  cufftHandle d2z, z2d;
  bool has_d2z, has_z2d;
  double* real;
  int nreal;
  cufftDoubleComplex* cplx;
  int ncplx;
  double* hist;  // kMaxShell * 3 doubles of shell sums, then one scalar
};

void spectral_ws_free(void* p) {
  SpectralWs* w = static_cast<SpectralWs*>(p);
  if (!w) return;
  if (w->has_d2z) cufftDestroy(w->d2z);
  if (w->has_z2d) cufftDestroy(w->z2d);
  cudaFree(w->real);
  cudaFree(w->cplx);
  cudaFree(w->hist);
  delete w;
}

namespace {

constexpr int kMaxShell = 1024;  // shell sums of three quantities in shared memory: 24 KB

struct HalfGrid {
  int nx, ny, nz, hx;
  long long h;   // nz * ny * hx modes of a half spectrum
  long long hp;  // stride between the half spectra of an array (h, 256-byte aligned)
  long long np;  // stride between the real fields of an array (N3, 256-byte aligned)
};

HalfGrid half(const Grid& g) {
  HalfGrid q;
  q.nx = g.nx;
  q.ny = g.ny;
  q.nz = g.nz;
  q.hx = g.nx / 2 + 1;
  q.h = (long long)g.nz * g.ny * q.hx;
  q.hp = fft_stride(q.h);
  q.np = fft_stride(g.n3);
  return q;
}

// Mode t of the half spectrum: integer wavenumber m (x non-negative), the
// derivative wavenumbers k (Nyquist of an even axis set to zero) and the
// weight of the mode in a sum over the full spectrum (2 where its conjugate
// -m is not stored).
struct Mode {
  int mx, my, mz;
  double kx, ky, kz, w;
};

__device__ __forceinline__ Mode mode_of(long long t, const HalfGrid& q) {
  Mode m;
  const int ix = (int)(t % q.hx);
  const int iy = (int)((t / q.hx) % q.ny);
  const int iz = (int)(t / ((long long)q.hx * q.ny));
  m.mx = ix;
  m.my = iy <= q.ny / 2 ? iy : iy - q.ny;
  m.mz = iz <= q.nz / 2 ? iz : iz - q.nz;
  const double tp = 6.283185307179586;
  m.kx = (q.nx % 2 == 0 && ix == q.nx / 2) ? 0.0 : tp * ix / q.nx;
  m.ky = (q.ny % 2 == 0 && iy == q.ny / 2) ? 0.0 : tp * m.my / q.ny;
  m.kz = (q.nz % 2 == 0 && iz == q.nz / 2) ? 0.0 : tp * m.mz / q.nz;
  m.w = (ix == 0 || (q.nx % 2 == 0 && ix == q.nx / 2)) ? 1.0 : 2.0;
  return m;
}

__device__ __forceinline__ int shell_of(const Mode& m) {
  const long long m2 = (long long)m.mx * m.mx + (long long)m.my * m.my + (long long)m.mz * m.mz;
  return __double2int_rn(sqrt((double)m2));
}

__device__ __forceinline__ cufftDoubleComplex times_ik(double k, cufftDoubleComplex v) {
  return make_cuDoubleComplex(-k * v.y, k * v.x);
}

// out_c = i (k x F)_c: the transform of the curl.
__global__ void curl_kernel(const cufftDoubleComplex* __restrict__ F, cufftDoubleComplex* __restrict__ out,
                            HalfGrid q) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < q.h; t += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(t, q);
    const cufftDoubleComplex a = F[t], b = F[q.hp + t], c = F[2 * q.hp + t];
    const cufftDoubleComplex x = make_cuDoubleComplex(m.ky * c.x - m.kz * b.x, m.ky * c.y - m.kz * b.y);
    const cufftDoubleComplex y = make_cuDoubleComplex(m.kz * a.x - m.kx * c.x, m.kz * a.y - m.kx * c.y);
    const cufftDoubleComplex z = make_cuDoubleComplex(m.kx * b.x - m.ky * a.x, m.kx * b.y - m.ky * a.y);
    out[t] = times_ik(1.0, x);
    out[q.hp + t] = times_ik(1.0, y);
    out[2 * q.hp + t] = times_ik(1.0, z);
  }
}

// out_a = i k_a F: the transform of the gradient of one component.
__global__ void grad_kernel(const cufftDoubleComplex* __restrict__ F, cufftDoubleComplex* __restrict__ out,
                            HalfGrid q) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < q.h; t += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(t, q);
    const cufftDoubleComplex v = F[t];
    out[t] = times_ik(m.kx, v);
    out[q.hp + t] = times_ik(m.ky, v);
    out[2 * q.hp + t] = times_ik(m.kz, v);
  }
}

// nl = inv * sum_a u_a G_a: component b of u . grad u, from the unnormalised
// inverse transforms G_a of i k_a F(u_b).
// (fields of an array are np apart)
__global__ void advect_kernel(const double* __restrict__ u, const double* __restrict__ G, double* __restrict__ nl,
                              long long n3, long long np, double inv) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n3; s += (long long)gridDim.x * blockDim.x)
    nl[s] = inv * (u[s] * G[s] + u[np + s] * G[np + s] + u[2 * np + s] * G[2 * np + s]);
}

// With J the unnormalised inverse transform of F(curl B): N = nl - J x B in
// place of nl, and W = (u - d_i J) x B in place of J.
__global__ void flux_fields_kernel(const double* __restrict__ u, const double* __restrict__ B, double* __restrict__ J,
                                   double* __restrict__ nl, long long n3, long long np, double inv, double di) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n3; s += (long long)gridDim.x * blockDim.x) {
    const double b[3] = {B[s], B[np + s], B[2 * np + s]};
    const double j[3] = {inv * J[s], inv * J[np + s], inv * J[2 * np + s]};
    const double v[3] = {u[s] - di * j[0], u[np + s] - di * j[1], u[2 * np + s] - di * j[2]};
    nl[s] -= j[1] * b[2] - j[2] * b[1];
    nl[np + s] -= j[2] * b[0] - j[0] * b[2];
    nl[2 * np + s] -= j[0] * b[1] - j[1] * b[0];
    J[s] = v[1] * b[2] - v[2] * b[1];
    J[np + s] = v[2] * b[0] - v[0] * b[2];
    J[2 * np + s] = v[0] * b[1] - v[1] * b[0];
  }
}

// Shell sums over the half spectrum (each mode with its weight), scaled by
// inv2 = N3^-2 for products of two unnormalised transforms:
//   pass 0: T += Re[F(u)* . X] with X = F(u.grad u - J x B); dis += k^2 (nu |F(u)|^2
//           + eta |F(B)|^2); en += 1/2 (|F(u)|^2 + |F(B)|^2)
//   pass 1: T -= Re[F(B)* . i k x X] with X = F((u - d_i J) x B)
// hist: T at [0, nshell), dis at [nshell, 2 nshell), en at [2 nshell, 3 nshell).
__global__ void budget_bin_kernel(const cufftDoubleComplex* __restrict__ Uh, const cufftDoubleComplex* __restrict__ Bh,
                                  const cufftDoubleComplex* __restrict__ X, HalfGrid q, int nshell, int pass, double nu,
                                  double eta, double inv2, double* __restrict__ hist) {
  extern __shared__ double sh[];
  for (int i = threadIdx.x; i < 3 * nshell; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < q.h; t += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(t, q);
    const int n = shell_of(m);
    if (n >= nshell) continue;
    if (pass == 0) {
      double tr = 0.0, pu = 0.0, pb = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cufftDoubleComplex a = Uh[c * q.hp + t], x = X[c * q.hp + t], b = Bh[c * q.hp + t];
        tr += a.x * x.x + a.y * x.y;
        pu += a.x * a.x + a.y * a.y;
        pb += b.x * b.x + b.y * b.y;
      }
      const double k2 = m.kx * m.kx + m.ky * m.ky + m.kz * m.kz;
      atomicAdd(&sh[n], m.w * inv2 * tr);
      atomicAdd(&sh[nshell + n], m.w * inv2 * k2 * (nu * pu + eta * pb));
      atomicAdd(&sh[2 * nshell + n], m.w * inv2 * 0.5 * (pu + pb));
    } else {
      const cufftDoubleComplex a = X[t], b = X[q.hp + t], c = X[2 * q.hp + t];
      // i k x X
      const cufftDoubleComplex cx = times_ik(1.0, make_cuDoubleComplex(m.ky * c.x - m.kz * b.x, m.ky * c.y - m.kz * b.y));
      const cufftDoubleComplex cy = times_ik(1.0, make_cuDoubleComplex(m.kz * a.x - m.kx * c.x, m.kz * a.y - m.kx * c.y));
      const cufftDoubleComplex cz = times_ik(1.0, make_cuDoubleComplex(m.kx * b.x - m.ky * a.x, m.kx * b.y - m.ky * a.y));
      const cufftDoubleComplex b0 = Bh[t], b1 = Bh[q.hp + t], b2 = Bh[2 * q.hp + t];
      const double tr = b0.x * cx.x + b0.y * cx.y + b1.x * cy.x + b1.y * cy.y + b2.x * cz.x + b2.y * cz.y;
      atomicAdd(&sh[n], -m.w * inv2 * tr);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nshell; i += blockDim.x)
    if (sh[i] != 0.0) atomicAdd(&hist[i], sh[i]);
}

// Band loss: L += 1/2 w |F(B)|^2 N3^-2 over the modes with lo <= shell <= hi;
// every other mode of F(B) is set to zero (the masked spectrum whose inverse
// transform is N3^2 dL/dB).
__global__ void band_kernel(cufftDoubleComplex* __restrict__ Bh, HalfGrid q, int lo, int hi, double inv2,
                            double* __restrict__ L) {
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < q.h; t += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(t, q);
    const int n = shell_of(m);
    if (n >= lo && n <= hi) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cufftDoubleComplex v = Bh[c * q.hp + t];
        acc += 0.5 * m.w * inv2 * (v.x * v.x + v.y * v.y);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) Bh[c * q.hp + t] = make_cuDoubleComplex(0.0, 0.0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(L, acc);
}

// dL/dB = inv2 * (inverse transform g of the masked spectrum, fields np
// apart) into dst (fields n3 apart) when given; and, when adj is given, the
// adjoint seed dL/df of the pre-collision populations in natural slot order:
// 0 for the fluid, dL/dB_b for every D3Q7 velocity of magnetic component b
// (B_b is the sum of those populations).
__global__ void band_grad_kernel(const double* __restrict__ g, long long n3, long long np, double inv2,
                                 double* __restrict__ dst, float* __restrict__ adj) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n3; s += (long long)gridDim.x * blockDim.x) {
    double v[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[b] = inv2 * g[b * np + s];
      if (dst) dst[b * n3 + s] = v[b];
    }
    if (adj) {
#pragma unroll
      for (int q = 0; q < 27; ++q) adj[q * n3 + s] = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int i = 0; i < 7; ++i) adj[(27 + 7 * b + i) * n3 + s] = (float)v[b];
    }
  }
}

int grid_for(long long n, int nsm) {
  long long b = (n + 255) / 256;
  const long long cap = (long long)nsm * 8;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// The workspace of a context, grown to nreal fields and ncplx half spectra,
// with both plans.
cudaError_t ensure_ws(flame_ctx* ctx, const CtxView& v, int nreal, int ncplx, SpectralWs** out) {
  void** slot = flame_ctx_spectral_slot(ctx);
  SpectralWs* w = static_cast<SpectralWs*>(*slot);
  if (!w) {
    w = new (std::nothrow) SpectralWs;
    if (!w) return cudaErrorMemoryAllocation;
    std::memset(static_cast<void*>(w), 0, sizeof(*w));
    w->g = v.g;
    *slot = w;
  }
  const size_t n3 = (size_t)fft_stride(v.g.n3);
  const size_t h = (size_t)fft_stride((long long)v.g.nz * v.g.ny * (v.g.nx / 2 + 1));
  cudaError_t e;
  if (w->nreal < nreal) {
    cudaFree(w->real);
    w->real = nullptr;
    w->nreal = 0;
    if ((e = cudaMalloc(&w->real, nreal * n3 * sizeof(double))) != cudaSuccess) return e;
    w->nreal = nreal;
  }
  if (w->ncplx < ncplx) {
    cudaFree(w->cplx);
    w->cplx = nullptr;
    w->ncplx = 0;
    if ((e = cudaMalloc(&w->cplx, ncplx * h * sizeof(cufftDoubleComplex))) != cudaSuccess) return e;
    w->ncplx = ncplx;
  }
  if (!w->hist && (e = cudaMalloc(&w->hist, (3 * kMaxShell + 1) * sizeof(double))) != cudaSuccess) return e;
  if (!w->has_d2z) {
    if (cufftPlan3d(&w->d2z, v.g.nz, v.g.ny, v.g.nx, CUFFT_D2Z) != CUFFT_SUCCESS) return cudaErrorUnknown;
    w->has_d2z = true;
  }
  if (!w->has_z2d) {
    if (cufftPlan3d(&w->z2d, v.g.nz, v.g.ny, v.g.nx, CUFFT_Z2D) != CUFFT_SUCCESS) return cudaErrorUnknown;
    w->has_z2d = true;
  }
  if (cufftSetStream(w->d2z, v.stream) != CUFFT_SUCCESS || cufftSetStream(w->z2d, v.stream) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  *out = w;
  return cudaSuccess;
}

cudaError_t d2z(SpectralWs* w, const double* src, cufftDoubleComplex* dst) {
  // the real input of an out-of-place D2Z transform is left unchanged
  return cufftExecD2Z(w->d2z, const_cast<double*>(src), dst) == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}
cudaError_t z2d(SpectralWs* w, cufftDoubleComplex* src, double* dst) {
  // overwrites src
  return cufftExecZ2D(w->z2d, src, dst) == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

flame_status fail(flame_ctx* ctx, cudaError_t e) { return static_cast<flame_status>(flame_ctx_cuda_fail(ctx, e)); }

// Common checks: a usable context; fields from the caller (given) or from the
// current state (then flame_init must have run).
flame_status usable_view(flame_ctx* ctx, CtxView* v, bool fields_given) {
  if (flame_ctx_view(ctx, v) != 0) return FLAME_ERR_PARAM;
  if (v->status != FLAME_OK && v->status != FLAME_ERR_NONFINITE) return static_cast<flame_status>(v->status);
  if (v->g.z0 != 0) return FLAME_ERR_PARAM;  // a z-slab holds only part of the lattice the spectra need
  if (!fields_given && !v->initialized) return FLAME_ERR_STATE;
  return FLAME_OK;
}

}  // namespace
}  // namespace flame

using flame::CtxView;
using flame::SpectralWs;

// Copy three caller fields (n3 apart) into workspace fields (np apart).
static cudaError_t load3(double* dst, const double* src, const flame::HalfGrid& q, long long n3, cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, q.np * sizeof(double), src, n3 * sizeof(double), n3 * sizeof(double), 3,
                           cudaMemcpyDeviceToDevice, st);
}

extern "C" flame_status flame_band_energy(flame_ctx* ctx, int lo, int hi, const double* d_B, double* h_L,
                                          double* d_dLdB, float* d_adj) {
  CtxView v;
  flame_status st = flame::usable_view(ctx, &v, d_B != nullptr);
  if (st != FLAME_OK) return st;
  if (!h_L || lo < 0 || hi < lo) return FLAME_ERR_PARAM;
  SpectralWs* w = nullptr;
  cudaError_t e = flame::ensure_ws(ctx, v, 3, 3, &w);
  if (e != cudaSuccess) return flame::fail(ctx, e);
  const long long n3 = v.g.n3;
  const flame::HalfGrid q = flame::half(v.g);
  const double inv2 = 1.0 / ((double)n3 * (double)n3);
  double* B = w->real;
  if (d_B)
    e = load3(B, d_B, q, n3, v.stream);
  else
    e = flame::launch_moments(v.storage, v.parity, v.state, v.g, v.k, nullptr, nullptr, B, nullptr, v.stream, q.np);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = flame::d2z(w, B + c * q.np, w->cplx + c * q.hp);
  double* L = w->hist + 3 * flame::kMaxShell;
  if (e == cudaSuccess) e = cudaMemsetAsync(L, 0, sizeof(double), v.stream);
  if (e != cudaSuccess) return flame::fail(ctx, e);
  flame::band_kernel<<<flame::grid_for(q.h, v.nsm), 256, 0, v.stream>>>(w->cplx, q, lo, hi, inv2, L);
  e = cudaGetLastError();
  if (e == cudaSuccess && (d_dLdB || d_adj)) {
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = flame::z2d(w, w->cplx + c * q.hp, B + c * q.np);
    if (e == cudaSuccess) {
      flame::band_grad_kernel<<<flame::grid_for(n3, v.nsm), 256, 0, v.stream>>>(B, n3, q.np, inv2, d_dLdB, d_adj);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_L, L, sizeof(double), cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  return flame::fail(ctx, e);
}

extern "C" flame_status flame_energy_budget(flame_ctx* ctx, int nshell, const double* d_u, const double* d_B,
                                            double* h_E, double* h_S, double* h_D) {
  CtxView v;
  if ((d_u == nullptr) != (d_B == nullptr)) return FLAME_ERR_PARAM;
  flame_status st = flame::usable_view(ctx, &v, d_u != nullptr);
  if (st != FLAME_OK) return st;
  if (nshell < 1 || nshell > flame::kMaxShell) return FLAME_ERR_PARAM;
  // real fields: u, B, J / W, G (a gradient), N; half spectra: F(u), F(B)
  // and one scratch triple
  SpectralWs* w = nullptr;
  cudaError_t e = flame::ensure_ws(ctx, v, 15, 9, &w);
  if (e != cudaSuccess) return flame::fail(ctx, e);
  const long long n3 = v.g.n3;
  const flame::HalfGrid q = flame::half(v.g);
  const long long np = q.np, hp = q.hp;
  const double inv = 1.0 / (double)n3, inv2 = inv * inv;
  double *u = w->real, *B = w->real + 3 * np, *J = w->real + 6 * np, *G = w->real + 9 * np, *NL = w->real + 12 * np;
  cufftDoubleComplex *Uh = w->cplx, *Bh = w->cplx + 3 * hp, *T = w->cplx + 6 * hp;
  if (d_u) {
    e = load3(u, d_u, q, n3, v.stream);
    if (e == cudaSuccess) e = load3(B, d_B, q, n3, v.stream);
  } else {
    e = flame::launch_moments(v.storage, v.parity, v.state, v.g, v.k, nullptr, u, B, nullptr, v.stream, np);
  }
  const double nu = (v.tau_nu - 0.5) / 3.0, eta = (v.tau_eta - 0.5) / 4.0;
  const int gh = flame::grid_for(q.h, v.nsm), gr = flame::grid_for(n3, v.nsm);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = flame::d2z(w, u + c * np, Uh + c * hp);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = flame::d2z(w, B + c * np, Bh + c * hp);
  if (e != cudaSuccess) return flame::fail(ctx, e);
  // J = curl B (times N3)
  flame::curl_kernel<<<gh, 256, 0, v.stream>>>(Bh, T, q);
  e = cudaGetLastError();
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = flame::z2d(w, T + c * hp, J + c * np);
  // u . grad u, one component at a time
  for (int b = 0; b < 3 && e == cudaSuccess; ++b) {
    flame::grad_kernel<<<gh, 256, 0, v.stream>>>(Uh + b * hp, T, q);
    e = cudaGetLastError();
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = flame::z2d(w, T + a * hp, G + a * np);
    if (e == cudaSuccess) {
      flame::advect_kernel<<<gr, 256, 0, v.stream>>>(u, G, NL + b * np, n3, np, inv);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    flame::flux_fields_kernel<<<gr, 256, 0, v.stream>>>(u, B, J, NL, n3, np, inv, v.d_i);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w->hist, 0, 3 * (size_t)nshell * sizeof(double), v.stream);
  const size_t shm = 3 * (size_t)nshell * sizeof(double);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    const double* src = pass == 0 ? NL : J;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = flame::d2z(w, src + c * np, T + c * hp);
    if (e == cudaSuccess) {
      flame::budget_bin_kernel<<<gh, 256, shm, v.stream>>>(Uh, Bh, T, q, nshell, pass, nu, eta, inv2, w->hist);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return flame::fail(ctx, e);
  double* tmp = new (std::nothrow) double[3 * (size_t)nshell];
  if (!tmp) return FLAME_ERR_PARAM;
  e = cudaMemcpyAsync(tmp, w->hist, 3 * (size_t)nshell * sizeof(double), cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess) {
    delete[] tmp;
    return flame::fail(ctx, e);
  }
  // S(n), D(n): sums over the shells below n
  double s = 0.0, d = 0.0;
  for (int n = 0; n < nshell; ++n) {
    if (h_S) h_S[n] = s;
    if (h_D) h_D[n] = d;
    if (h_E) h_E[n] = tmp[2 * nshell + n];
    s += tmp[n];
    d += tmp[nshell + n];
  }
  delete[] tmp;
  return FLAME_OK;
}
