// diag.cu -- kernels that read or write the population state outside the
// hot path: initialisation from macroscopic fields, moments and
// decoded populations (FP64), and the deterministic FP64 reduction of the
// scalar diagnostics.
#include "aa.cuh"

namespace flame {
namespace {

// ---------------------------------------------------------------------------
// Initialisation (once per run).  The arithmetic type R is FP64 for FP32
// storage and FP32 for 16-bit storage, whose encoding rounds to 2^-11 (FP16)
// or 2^-8 (BF16) relative, far above FP32's 2^-24; the gradients too are
// taken in R.

// Periodic central difference of field f along axis a at (x, y, z), in the
// per-site arithmetic type R (GB300's FP64 pipe is 1/64 of its FP32 rate, so
// 16-bit storage, whose values keep 11 or 8 bits, takes them in FP32).
template <class R, class F>
__device__ __forceinline__ R cdiff(const F* f, int a, int x, int y, int z, const Grid& g) {
  int xp = x, xm = x, yp = y, ym = y, zp = z, zm = z;
  if (a == 0) {
    xp = x + 1 == g.nx ? 0 : x + 1;
    xm = x == 0 ? g.nx - 1 : x - 1;
  } else if (a == 1) {
    yp = y + 1 == g.ny ? 0 : y + 1;
    ym = y == 0 ? g.ny - 1 : y - 1;
  } else {
    zp = z + 1 == g.nz ? 0 : z + 1;
    zm = z == 0 ? g.nz - 1 : z - 1;
  }
  return (R)0.5 * ((R)f[((long long)zp * g.ny + yp) * g.nx + xp] - (R)f[((long long)zm * g.ny + ym) * g.nx + xm]);
}

// F: the element type of the caller's fields (FP64 for flame_init, FP32 for
// flame_init_f32).
template <class T, class R, class F>
__global__ void init_kernel(T* __restrict__ pop, Grid g, StepConsts k, int noneq, const F* __restrict__ rho_f,
                            const F* __restrict__ u, const F* __restrict__ Bf, const F* __restrict__ gu,
                            const F* __restrict__ gB, unsigned* __restrict__ speed_bits) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  const bool in = x < g.nx && y < g.ny;
  float sp = 0.f;
  if (in) {
    const long long n3 = g.n3;
    const long long site = ((long long)z * g.ny + y) * g.nx + x;
    const R rho = rho_f ? (R)rho_f[site] : (R)1;
    const R U[3] = {(R)u[site], (R)u[n3 + site], (R)u[2 * n3 + site]};
    const R B[3] = {(R)Bf[site], (R)Bf[n3 + site], (R)Bf[2 * n3 + site]};
    R du[9], dB[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        du[3 * a + b] = gu ? (R)gu[(3 * a + b) * n3 + site] : cdiff<R>(u + b * n3, a, x, y, z, g);
        dB[3 * a + b] = gB ? (R)gB[(3 * a + b) * n3 + site] : cdiff<R>(Bf + b * n3, a, x, y, z, g);
      }
    const R J0[3] = {dB[5] - dB[7], dB[6] - dB[2], dB[1] - dB[3]};  // curl B
    const R omega = (R)k.omega, omegaB = (R)k.omegaB, aH = (R)k.alphaH;
    const R Br[3] = {(R)k.Bref[0], (R)k.Bref[1], (R)k.Bref[2]};
    const R b[3] = {B[0] - Br[0], B[1] - Br[1], B[2] - Br[2]};
    R N[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) N[a][c] = Br[a] * b[c] + b[a] * Br[c] + b[a] * b[c];
    const R miso = Br[0] * b[0] + Br[1] * b[1] + Br[2] * b[2] + (R)0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    const R trN3 = (N[0][0] + N[1][1] + N[2][2]) / (R)3;
    R Pn[3][3];  // first-order non-equilibrium stress -(rho cs^2/omega)(du + du^T)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) Pn[a][c] = noneq ? -(rho / ((R)3 * omega)) * (du[3 * a + c] + du[3 * c + a]) : (R)0;
    const R trPn3 = (Pn[0][0] + Pn[1][1] + Pn[2][2]) / (R)3;
    const R drho = rho - (R)k.rho0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int c[3] = {cx27(i), cy27(i), cz27(i)};
      R E = 0;  // prod(psi/w1) - 1, accumulated stably
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R uu = U[a] * U[a];
        const R ea = c[a] == 0 ? (R)-1.5 * uu : (R)3 * uu + (R)(3 * c[a]) * U[a];
        E = E + ea + E * ea;
      }
      R cNc = 0, cPc = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (c[a] * c[d] == 0) continue;
          cNc += (R)(c[a] * c[d]) * N[a][d];
          cPc += (R)(c[a] * c[d]) * Pn[a][d];
        }
      const R c2 = (R)(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
      const R L = (R)4.5 * (miso * (c2 - (R)1) - cNc + trN3);
      const R ne = (R)4.5 * (cPc - trPn3);
      pop[(long long)phys(i) * n3 + site] = Codec<T>::enc((float)(drho + rho * E + L + ne));
    }
    const R V[3] = {U[0] - aH * J0[0], U[1] - aH * J0[1], U[2] - aH * J0[2]};
#pragma unroll
    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
      for (int i = 0; i < kM; ++i) {
        const int xi[3] = {mx7(i), my7(i), mz7(i)};
        R l0 = 0, ne = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (xi[a] == 0) continue;
          l0 += (R)xi[a] * (V[a] * B[bb] - B[a] * V[bb]);
          ne += (R)xi[a] * dB[3 * a + bb];
        }
        const R v = b[bb] + (R)4 * l0 - (noneq ? ne / omegaB : (R)0);
        pop[(long long)phys(mslot(bb, i)) * n3 + site] = Codec<T>::enc((float)v);
      }
    const R va = sqrt((B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho);
    const R um = sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    sp = (float)fmax(va, um);
    if (!isfinite(sp)) sp = __uint_as_float(0x7f800000u);
  }
  // max speed: one atomic per warp (non-negative floats order like their bits)
  const unsigned m = __reduce_max_sync(0xffffffffu, in ? __float_as_uint(sp) : 0u);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(speed_bits, m);
}

// ---------------------------------------------------------------------------
// Moments and decoded populations.  Per-site arithmetic in R: FP64 for FP32
// storage, FP32 for 16-bit storage (whose stored values carry 11 or 8
// significant bits).  Density and field are formed as deviations from the
// reference (rho0, B_ref) and added to it in FP64, so sums over sites keep
// the FP64 reference exact.

template <class T, bool ODD, class R>
__device__ __forceinline__ void load_site(const T* __restrict__ pop, int site, const Nbr& nb, long long n3,
                                          R sf[kQ], R sg[3][kM]) {
#pragma unroll
  for (int i = 0; i < kQ; ++i) sf[i] = (R)Codec<T>::dec(pop[src27<ODD>(i, site, nb, n3)]);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int i = 0; i < kM; ++i) sg[b][i] = (R)Codec<T>::dec(pop[src7<ODD>(b, i, site, nb, n3)]);
}

template <class R>
struct SiteMoments {
  R drho, U[3], dB[3], J[3], trlam;  // drho = rho - rho0, dB = B - B_ref
  __device__ __forceinline__ double rho(const StepConsts& k) const { return (double)k.rho0 + (double)drho; }
  __device__ __forceinline__ double B(const StepConsts& k, int a) const { return (double)k.Bref[a] + (double)dB[a]; }
};

template <class R>
__device__ __forceinline__ SiteMoments<R> site_moments(const R sf[kQ], const R sg[3][kM], const StepConsts& k) {
  SiteMoments<R> m;
  R drho = 0, j[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const R t = (R)w27d(i) * sf[i];
    drho += t;
    if (cx27(i)) j[0] += (R)cx27(i) * t;
    if (cy27(i)) j[1] += (R)cy27(i) * t;
    if (cz27(i)) j[2] += (R)cz27(i) * t;
  }
  m.drho = drho;
  const R rho = (R)k.rho0 + drho;
#pragma unroll
  for (int a = 0; a < 3; ++a) m.U[a] = j[a] / rho;
  R lam[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    m.dB[b] = (R)0.25 * sg[b][0] + (R)0.125 * (sg[b][1] + sg[b][2] + sg[b][3] + sg[b][4] + sg[b][5] + sg[b][6]);
    lam[0][b] = (R)0.125 * (sg[b][1] - sg[b][2]);
    lam[1][b] = (R)0.125 * (sg[b][3] - sg[b][4]);
    lam[2][b] = (R)0.125 * (sg[b][5] - sg[b][6]);
  }
  m.trlam = lam[0][0] + lam[1][1] + lam[2][2];
  const R gq = (R)4 * (R)k.omegaB;
  const R* U = m.U;
  const R B[3] = {(R)k.Bref[0] + m.dB[0], (R)k.Bref[1] + m.dB[1], (R)k.Bref[2] + m.dB[2]};
  const R A[3] = {lam[1][2] - lam[2][1], lam[2][0] - lam[0][2], lam[0][1] - lam[1][0]};
  const R uxb[3] = {U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2], U[0] * B[1] - U[1] * B[0]};
  const R yv[3] = {-gq * (A[0] - (R)2 * uxb[0]), -gq * (A[1] - (R)2 * uxb[1]), -gq * (A[2] - (R)2 * uxb[2])};
  const R s = (R)2 * (R)k.alphaH * gq;
  const R yxb[3] = {yv[1] * B[2] - yv[2] * B[1], yv[2] * B[0] - yv[0] * B[2], yv[0] * B[1] - yv[1] * B[0]};
  const R yb = yv[0] * B[0] + yv[1] * B[1] + yv[2] * B[2];
  const R b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) m.J[a] = (yv[a] - s * yxb[a] + s * s * yb * B[a]) / ((R)1 + s * s * b2);
  return m;
}

// per-site arithmetic type of a storage type
template <class T>
struct SiteReal {
  using type = float;
};
template <>
struct SiteReal<float> {
  using type = double;
};

// O: the element type of the outputs (FP64 for flame_moments, FP32 for
// flame_moments_f32).
template <class T, bool ODD, class O>
__global__ void moments_kernel(const T* __restrict__ pop, Grid g, StepConsts k, O* __restrict__ rho,
                               O* __restrict__ u, O* __restrict__ B, O* __restrict__ J, long long os) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  if (x >= g.nx || y >= g.ny) return;
  const int site = (z * g.ny + y) * g.nx + x;
  const Nbr nb = make_nbr(x, y, z, g);
  using R = typename SiteReal<T>::type;
  R sf[kQ], sg[3][kM];
  load_site<T, ODD>(pop, site, nb, g.n3, sf, sg);
  const SiteMoments<R> m = site_moments(sf, sg, k);
  const long long o = site - (long long)g.z0 * g.nx * g.ny;  // index among the updated sites
  if (rho) rho[o] = (O)m.rho(k);
  for (int a = 0; a < 3; ++a) {
    if (u) u[a * os + o] = (O)m.U[a];
    if (B) B[a * os + o] = (O)m.B(k, a);
    if (J) J[a * os + o] = (O)m.J[a];
  }
}

template <class T, bool ODD>
__global__ void populations_kernel(const T* __restrict__ pop, Grid g, StepConsts k, double* __restrict__ f) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  if (x >= g.nx || y >= g.ny) return;
  const int site = (z * g.ny + y) * g.nx + x;
  const Nbr nb = make_nbr(x, y, z, g);
  double sf[kQ], sg[3][kM];
  load_site<T, ODD, double>(pop, site, nb, g.n3, sf, sg);
  const double Br[3] = {(double)k.Bref[0], (double)k.Bref[1], (double)k.Bref[2]};
  const double br2 = Br[0] * Br[0] + Br[1] * Br[1] + Br[2] * Br[2];
  const long long o = site - (long long)g.z0 * g.nx * g.ny;  // index among the updated sites
#pragma unroll 1
  for (int i = 0; i < kQ; ++i) {
    const double c2 = cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i);
    const double cb = cx27(i) * Br[0] + cy27(i) * Br[1] + cz27(i) * Br[2];
    const double ell = 4.5 * (0.5 * br2 * (c2 - 1.0 / 3.0) - cb * cb);  // rest Lorentz term / w
    f[(long long)i * g.n3i + o] = w27d(i) * ((double)k.rho0 + ell + sf[i]);
  }
  for (int b = 0; b < 3; ++b)
    for (int i = 0; i < kM; ++i) f[(long long)mslot(b, i) * g.n3i + o] = w7d(i) * (Br[b] + sg[b][i]);
}


// Moments at a list of sites (time series): out[j] = rho, u[3], B[3], J[3].
template <class T, bool ODD>
__global__ void probe_kernel(const T* __restrict__ pop, Grid g, StepConsts k, int n, const long long* __restrict__ sites,
                             double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long long sl = sites[j];
  if (sl < 0 || sl >= g.n3i) {
    for (int v = 0; v < 10; ++v) out[(long long)j * 10 + v] = nan("");
    return;
  }
  const int site = (int)(sl + (long long)g.z0 * g.nx * g.ny);
  const int x = site % g.nx, y = (site / g.nx) % g.ny, z = site / (g.nx * g.ny);
  const Nbr nb = make_nbr(x, y, z, g);
  using R = typename SiteReal<T>::type;
  R sf[kQ], sg[3][kM];
  load_site<T, ODD>(pop, site, nb, g.n3, sf, sg);
  const SiteMoments<R> m = site_moments(sf, sg, k);
  double* o = out + (long long)j * 10;
  o[0] = m.rho(k);
  for (int a = 0; a < 3; ++a) {
    o[1 + a] = (double)m.U[a];
    o[4 + a] = m.B(k, a);
    o[7 + a] = (double)m.J[a];
  }
}

template <class T>
cudaError_t probe_t(int odd, const void* pop, Grid g, const StepConsts& k, int n, const long long* sites, double* out,
                    cudaStream_t s) {
  const int tb = 64, nb = (n + tb - 1) / tb;
  if (odd)
    probe_kernel<T, true><<<nb, tb, 0, s>>>(static_cast<const T*>(pop), g, k, n, sites, out);
  else
    probe_kernel<T, false><<<nb, tb, 0, s>>>(static_cast<const T*>(pop), g, k, n, sites, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 reduction of the scalar diagnostics: per block, then a fixed-order
// final sum (deterministic).  Partial layout (kRedVals):
//   0 sum rho, 1-3 sum rho u, 4-6 sum B, 7 sum |u|^2, 8 sum |B - Bref|^2,
//   9 sum u.(B - Bref), 10-12 sum u, 13 sum |J|^2, 14 max |u|,
//   15 sum ((omega_B/C^2) Tr Lambda)^2, 16 non-finite sites.
template <class T, bool ODD>
__global__ void reduce_kernel(const T* __restrict__ pop, Grid g, StepConsts k, double* __restrict__ partials) {
  double acc[kRedVals];
#pragma unroll
  for (int v = 0; v < kRedVals; ++v) acc[v] = 0.0;
  const long long n3 = g.n3;
  const long long off = (long long)g.z0 * g.nx * g.ny;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n3i; s += (long long)gridDim.x * blockDim.x) {
    const int site = (int)(s + off);
    const int x = site % g.nx, y = (site / g.nx) % g.ny, z = site / (g.nx * g.ny);
    const Nbr nb = make_nbr(x, y, z, g);
    using R = typename SiteReal<T>::type;
    R sf[kQ], sg[3][kM];
    load_site<T, ODD>(pop, site, nb, n3, sf, sg);
    const SiteMoments<R> m = site_moments(sf, sg, k);
    const R* b = m.dB;
    const R uu = m.U[0] * m.U[0] + m.U[1] * m.U[1] + m.U[2] * m.U[2];
    const R dv = (R)4 * (R)k.omegaB * m.trlam;
    const bool ok = isfinite(m.drho + uu + b[0] + b[1] + b[2] + m.J[0] + m.J[1] + m.J[2]);
    if (!ok) {
      acc[16] += 1.0;
      continue;
    }
    const double rho = m.rho(k);
    acc[0] += rho;
    for (int a = 0; a < 3; ++a) {
      acc[1 + a] += rho * (double)m.U[a];
      acc[4 + a] += m.B(k, a);
      acc[10 + a] += (double)m.U[a];
    }
    acc[7] += (double)uu;
    acc[8] += (double)(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    acc[9] += (double)(m.U[0] * b[0] + m.U[1] * b[1] + m.U[2] * b[2]);
    acc[13] += (double)(m.J[0] * m.J[0] + m.J[1] * m.J[1] + m.J[2] * m.J[2]);
    acc[14] = fmax(acc[14], sqrt((double)uu));
    acc[15] += (double)(dv * dv);
  }
  // warp, then block
  __shared__ double sh[32][kRedVals];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < kRedVals; ++v) {
    double a = acc[v];
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_down_sync(0xffffffffu, a, o);
      a = (v == 14) ? fmax(a, t) : a + t;
    }
    if (lane == 0) sh[warp][v] = a;
  }
  __syncthreads();
  if (threadIdx.x < kRedVals) {
    const int v = threadIdx.x;
    double a = sh[0][v];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) a = (v == 14) ? fmax(a, sh[w][v]) : a + sh[w][v];
    partials[(long long)blockIdx.x * kRedVals + v] = a;
  }
}

__global__ void reduce_final_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  const int v = threadIdx.x;
  if (v >= kRedVals) return;
  double a = partials[v];
  for (int bk = 1; bk < nblocks; ++bk) a = (v == 14) ? fmax(a, partials[(long long)bk * kRedVals + v]) : a + partials[(long long)bk * kRedVals + v];
  out[v] = a;
}

// Block of `threads` threads: x-rows of up to `threads` sites, several
// rows per block when nx is small.

template <class T, class O>
cudaError_t moments_t(int odd, const void* pop, Grid g, const StepConsts& k, O* rho, O* u, O* B, O* J,
                      long long os, cudaStream_t s) {
  const dim3 b = site_block(g), gr = site_grid(g, b);
  if (odd)
    moments_kernel<T, true, O><<<gr, b, 0, s>>>(static_cast<const T*>(pop), g, k, rho, u, B, J, os);
  else
    moments_kernel<T, false, O><<<gr, b, 0, s>>>(static_cast<const T*>(pop), g, k, rho, u, B, J, os);
  return cudaGetLastError();
}

template <class F>
cudaError_t init_t(int storage, void* pop, Grid g, const StepConsts& k, int noneq, const F* rho, const F* u,
                   const F* B, const F* gu, const F* gB, unsigned* speed_bits, cudaStream_t s) {
  const dim3 b = site_block(g), gr = site_grid(g, b);
  switch (storage) {
    case 1:
      init_kernel<float, double, F><<<gr, b, 0, s>>>(static_cast<float*>(pop), g, k, noneq, rho, u, B, gu, gB,
                                                      speed_bits);
      break;
    case 2:
      init_kernel<__half, float, F><<<gr, b, 0, s>>>(static_cast<__half*>(pop), g, k, noneq, rho, u, B, gu, gB,
                                                      speed_bits);
      break;
    case 3:
      init_kernel<__nv_bfloat16, float, F><<<gr, b, 0, s>>>(static_cast<__nv_bfloat16*>(pop), g, k, noneq, rho, u,
                                                             B, gu, gB, speed_bits);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class O>
cudaError_t moments_any(int storage, int odd, const void* pop, Grid g, const StepConsts& k, O* rho, O* u, O* B,
                        O* J, long long os, cudaStream_t s) {
  if (os == 0) os = g.n3i;
  switch (storage) {
    case 1: return moments_t<float, O>(odd, pop, g, k, rho, u, B, J, os, s);
    case 2: return moments_t<__half, O>(odd, pop, g, k, rho, u, B, J, os, s);
    case 3: return moments_t<__nv_bfloat16, O>(odd, pop, g, k, rho, u, B, J, os, s);
  }
  return cudaErrorInvalidValue;
}

template <class T>
cudaError_t populations_t(int odd, const void* pop, Grid g, const StepConsts& k, double* f, cudaStream_t s) {
  const dim3 b = site_block(g), gr = site_grid(g, b);
  if (odd)
    populations_kernel<T, true><<<gr, b, 0, s>>>(static_cast<const T*>(pop), g, k, f);
  else
    populations_kernel<T, false><<<gr, b, 0, s>>>(static_cast<const T*>(pop), g, k, f);
  return cudaGetLastError();
}

template <class T>
cudaError_t reduce_t(int odd, const void* pop, Grid g, const StepConsts& k, int nblocks, double* partials,
                     double* out, cudaStream_t s) {
  if (odd)
    reduce_kernel<T, true><<<nblocks, 256, 0, s>>>(static_cast<const T*>(pop), g, k, partials);
  else
    reduce_kernel<T, false><<<nblocks, 256, 0, s>>>(static_cast<const T*>(pop), g, k, partials);
  reduce_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}


}  // namespace

cudaError_t launch_init(int storage, void* pop, Grid g, const StepConsts& k, int noneq, const double* rho,
                        const double* u, const double* B, const double* gu, const double* gB,
                        unsigned* speed_bits, cudaStream_t s) {
  return init_t<double>(storage, pop, g, k, noneq, rho, u, B, gu, gB, speed_bits, s);
}

cudaError_t launch_init_f32(int storage, void* pop, Grid g, const StepConsts& k, int noneq, const float* rho,
                            const float* u, const float* B, const float* gu, const float* gB,
                            unsigned* speed_bits, cudaStream_t s) {
  return init_t<float>(storage, pop, g, k, noneq, rho, u, B, gu, gB, speed_bits, s);
}

cudaError_t launch_moments(int storage, int odd, const void* pop, Grid g, const StepConsts& k, double* rho,
                           double* u, double* B, double* J, cudaStream_t s, long long ostride) {
  return moments_any<double>(storage, odd, pop, g, k, rho, u, B, J, ostride, s);
}

cudaError_t launch_moments_f32(int storage, int odd, const void* pop, Grid g, const StepConsts& k, float* rho,
                               float* u, float* B, float* J, cudaStream_t s, long long ostride) {
  return moments_any<float>(storage, odd, pop, g, k, rho, u, B, J, ostride, s);
}

cudaError_t launch_populations(int storage, int odd, const void* pop, Grid g, const StepConsts& k, double* f,
                               cudaStream_t s) {
  switch (storage) {
    case 1: return populations_t<float>(odd, pop, g, k, f, s);
    case 2: return populations_t<__half>(odd, pop, g, k, f, s);
    case 3: return populations_t<__nv_bfloat16>(odd, pop, g, k, f, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_probe(int storage, int odd, const void* pop, Grid g, const StepConsts& k, int n,
                         const long long* sites, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  switch (storage) {
    case 1: return probe_t<float>(odd, pop, g, k, n, sites, out, s);
    case 2: return probe_t<__half>(odd, pop, g, k, n, sites, out, s);
    case 3: return probe_t<__nv_bfloat16>(odd, pop, g, k, n, sites, out, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_reduce_partials(int storage, int odd, const void* pop, Grid g, const StepConsts& k, int nblocks,
                                   double* partials, cudaStream_t s) {
  if (nblocks < 1) return cudaErrorInvalidValue;
  switch (storage) {
    case 1:
      if (odd) reduce_kernel<float, true><<<nblocks, 256, 0, s>>>(static_cast<const float*>(pop), g, k, partials);
      else reduce_kernel<float, false><<<nblocks, 256, 0, s>>>(static_cast<const float*>(pop), g, k, partials);
      break;
    case 2:
      if (odd) reduce_kernel<__half, true><<<nblocks, 256, 0, s>>>(static_cast<const __half*>(pop), g, k, partials);
      else reduce_kernel<__half, false><<<nblocks, 256, 0, s>>>(static_cast<const __half*>(pop), g, k, partials);
      break;
    case 3:
      if (odd) reduce_kernel<__nv_bfloat16, true><<<nblocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(pop), g, k, partials);
      else reduce_kernel<__nv_bfloat16, false><<<nblocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(pop), g, k, partials);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce(int storage, int odd, const void* pop, Grid g, const StepConsts& k, int nblocks,
                          double* partials, double* out, cudaStream_t s) {
  if (nblocks < 1 || nblocks > kRedBlocksMax) return cudaErrorInvalidValue;
  switch (storage) {
    case 1: return reduce_t<float>(odd, pop, g, k, nblocks, partials, out, s);
    case 2: return reduce_t<__half>(odd, pop, g, k, nblocks, partials, out, s);
    case 3: return reduce_t<__nv_bfloat16>(odd, pop, g, k, nblocks, partials, out, s);
  }
  return cudaErrorInvalidValue;
}


}  // namespace flame
