// adjoint.cu -- hand-written vector-Jacobian products of the FLAME step and
// of the initialisation, for gradients of a loss of the final state with
// respect to the initial fields and the Hall length d_i.
//
// Step.  With lambda_{t+1} = dL/df(t+1) (pre-collision populations, natural
// slot order), streaming f(x, q, t+1) = f*(x - c_q, q, t) gives
// dL/df*(x, q) = lambda_{t+1}(x + c_q, q), and the per-site collision's
// transpose Jacobian maps it to lambda_t.  The forward quantities of the
// site (rho, U, Pi, B, Lambda, J, V, D) are recomputed from the state at t.
// Reverse sweep per site (physical populations f, g; gamma = omega_B/C^2,
// s = 2 gamma alpha_H, M = I + s [. x B]):
//   g*  = (1-wB) g + wB g^eq(B, V):   gbar = (1-wB) gbar*; mu = wB W_i gbar*;
//        Bbar += m0 + 4 Q^T V - 4 Q V, Vbar = 4 Q B - 4 Q^T B with
//        m0_b = sum_i mu_bi, Q_ab = sum_i mu_bi xi_ia;
//   V = U - alpha J:  Ubar += Vbar, Jbar = -alpha Vbar, abar -= Vbar.J;
//   J = M^-1 y:       lJ = M^-T Jbar (same closed form with s -> -s),
//        ybar = lJ, sbar = -lJ.(J x B), Bbar -= s lJ x J;
//   s = 2 gamma alpha: abar += 2 gamma sbar;
//   y = -gamma (A - 2 U x B): Abar = -gamma ybar, Ubar += 2 gamma B x ybar,
//        Bbar += 2 gamma ybar x U; Lambdabar_ab = eps_cab Abar_c;
//   f* = rho prod psi(U) + Lorentz(B) + P(D, U), D = (1-w) dev(Pi - rho U U - M(B)):
//        contractions of fbar* with the products of 1-D functions and their
//        U derivatives give rhobar, Ubar, Dbar; Lorentz gives
//        Bbar += 4.5 (tr H B - 2 H B), H = sum_i fbar*_i w_i H2_i;
//        Dbar -> Sbar -> (Pibar, rhobar, Ubar, Bbar);
//   U = j/rho: jbar = Ubar/rho, rhobar -= Ubar.U/rho;
//   moments: fbar_i = rhobar + jbar.c_i + Pibar : c_i c_i,
//            gbar_bi += Bbar_b + sum_a xi_ia Lambdabar_ab.
#include <type_traits>

#include "aa.cuh"

namespace flame {
namespace {

// 96 registers without spills: 64-thread blocks, ten per SM, for FP32
// storage; 128-thread blocks, five per SM, for 16-bit storage.  The lambda gather
// goes into shared memory by asynchronous copies (cp.async) that are in
// flight during the forward recompute, and lambda is read from there where
// it is used rather than held in registers; for 16-bit storage the state
// loads are issued before the copies, for FP32 after them; both carry a
// 256-byte L2 prefetch hint.  The d_i
// contributions are summed per warp in FP64 (no block barrier) and the
// partials added in a fixed order by two small kernels.  Timed at
// 256^3 (GLUPS FP32 / FP16 storage): one 256-thread block of 185 registers
// per SM with per-velocity sums 5.6 / 5.3; 1-D passes, 128 x 3 (168
// registers) 8.30 / 8.53; lambda gathered into registers after the
// recompute, 128 x 4, 9.37 / 10.1; gathered by cp.async 9.71 / 10.1; lambda
// read from shared memory where used, 128 x 5, 9.71 / 10.39 (128 x 6, 80
// registers with spills: 9.26 / 9.85); the partials summed by one block had
// cost ~5 %: 10.23 / 10.91 with the two-level sum, 10.27 / 11.0 with the
// per-storage load order and 64 x 10, 10.51 / 11.16 with read-only state
// loads and 256-byte L2 prefetch hints on them and on the lambda copies
// (10.46 / 11.06 for the state loads alone; f32x2 pairs inside the 1-D
// passes: 10.35 / 11.04, not kept); with the hints, 128 x 5 10.52 / 11.31
// against 64 x 10 10.57 / 11.23, hence the block per storage (128-byte
// state prefetch: 10.51 / 11.18).  (Per-warp sums in FP32 gained 0.7 %
// but, where the sites' terms cancel -- a random lambda: sum |a| / |sum a|
// ~ 5000 -- they added ~5x the rounding of the per-site arithmetic to d_i.)
template <class T>
constexpr int kAdjThreads = sizeof(T) == 2 ? 128 : 64;
template <class T>
constexpr int kAdjMinBlocks = sizeof(T) == 2 ? 5 : 10;

// 1-D functions of the undivided equilibrium and inverse-moment maps, and
// their derivatives in u, at velocity component c (index p = c + 1).
// (The u derivative of F0 equals F1.)
struct Axis {
  float psi[3], dpsi[3], F0[3], F1[3];
  __device__ __forceinline__ explicit Axis(float u) {
    const float uu = u * u;
    psi[1] = 2.f / 3.f - uu;
    dpsi[1] = -2.f * u;
    F0[1] = 1.f - uu;
    F1[1] = -2.f * u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float c = h == 0 ? -1.f : 1.f;
      const int p = h == 0 ? 0 : 2;
      psi[p] = 0.5f * (1.f / 3.f + uu + c * u);
      dpsi[p] = u + 0.5f * c;
      F0[p] = 0.5f * (uu + c * u);
      F1[p] = u + 0.5f * c;
    }
  }
};

// Separable sums over the velocity cube, sum_p t[pz][py][px] fx(px) fy(py)
// fz(pz), as three 1-D passes (x, then y, then z), so that the partial sums
// are shared between the many products the adjoint needs.  A 1-D function
// of p = c + 1 is a table of values (Fv: the U-dependent factors) or one of
// the constant tables (Fc) written out, so that their zero entries cost
// nothing: F2 = (1/2, -1, 1/2) (the second-order inverse map), dF1 =
// (1, -2, 1) (u derivative of F1), the 1-D weights w = (1/6, 2/3, 1/6), w c,
// w c^2, and (1, 4, 1), c, c^2 (moments of the 216-scaled weights).
enum : int { kFnF2, kFnDF1, kFnW, kFnWC, kFnWC2, kFnM0, kFnM1, kFnM2 };
template <int K>
struct Fc {};
struct Fv {
  const float* f;
};
__device__ __forceinline__ float app(Fv F, float a0, float a1, float a2) {
  return fmaf(a2, F.f[2], fmaf(a1, F.f[1], a0 * F.f[0]));
}
template <int K>
__device__ __forceinline__ float app(Fc<K>, float a0, float a1, float a2) {
  if constexpr (K == kFnF2) return fmaf(0.5f, a0 + a2, -a1);
  else if constexpr (K == kFnDF1) return fmaf(-2.f, a1, a0 + a2);
  else if constexpr (K == kFnW) return fmaf(2.f / 3.f, a1, (1.f / 6.f) * (a0 + a2));
  else if constexpr (K == kFnWC) return (1.f / 6.f) * (a2 - a0);
  else if constexpr (K == kFnWC2) return (1.f / 6.f) * (a0 + a2);
  else if constexpr (K == kFnM0) return fmaf(4.f, a1, a0 + a2);
  else if constexpr (K == kFnM1) return a2 - a0;
  else return a0 + a2;
}
template <class F>
__device__ __forceinline__ void xpass(const float (&t)[3][3][3], F f, float (&o)[3][3]) {
#pragma unroll
  for (int pz = 0; pz < 3; ++pz)
#pragma unroll
    for (int py = 0; py < 3; ++py) o[pz][py] = app(f, t[pz][py][0], t[pz][py][1], t[pz][py][2]);
}
template <class F>
__device__ __forceinline__ void ypass(const float (&x)[3][3], F f, float (&o)[3]) {
#pragma unroll
  for (int pz = 0; pz < 3; ++pz) o[pz] = app(f, x[pz][0], x[pz][1], x[pz][2]);
}
template <class F>
__device__ __forceinline__ float zpass(const float (&y)[3], F f) {
  return app(f, y[0], y[1], y[2]);
}

// Per-warp partial sums (no block barrier at the end of the step kernel);
// blocks are whole warps (site_block rounds x to 32).
__device__ __forceinline__ void warp_sum_to(double v, double* out) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) *out = v;
}

__device__ __forceinline__ void block_sum_to(double v, double* out) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double a = 0.0;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    for (int w = 0; w < nw; ++w) a += sh[w];
    *out = a;
  }
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global.L2::256B [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ float lds(const float* p) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Read-only state loads with an L2 prefetch-size hint (the neighbouring
// warps' segments of the same rows arrive with the first request).
template <class T>
__device__ __forceinline__ float ld_state(const T* p) {
  if constexpr (sizeof(T) == 4) {
    float v;
    asm volatile("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
  } else {
    unsigned short h;
    asm volatile("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(h) : "l"(p));
    if constexpr (std::is_same_v<T, __half>) return __half2float(__ushort_as_half(h));
    else return __bfloat162float(__ushort_as_bfloat16(h));
  }
}

// Base pointers of lambda_{t+1} (in) and lambda_t (out) per natural slot,
// passed as kernel parameters (as the state's Slots are), so that each of a
// site's 96 lambda accesses is one index computation on a parameter.
struct LamSlots {
  const float* in[kPop];
  float* out[kPop];
};

template <class T, bool ODD>
__global__ void __launch_bounds__(kAdjThreads<T>, kAdjMinBlocks<T>)
    adjoint_step_kernel(Slots<T> P, Grid g, StepConsts k, const __grid_constant__ LamSlots L,
                        double* __restrict__ partials) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  const bool live = x < g.nx && y < g.ny;
  __shared__ float lsm[kPop][kAdjThreads<T>];
  double abar_site = 0.0;
  if (live) {
    const int site = (z * g.ny + y) * g.nx + x;
    const Nbr nb = make_nbr(x, y, z, g);

    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    auto lgv = [&](int b, int i) { return lds(&lsm[kQ + kM * b + i][tid]); };
    auto issue_gather = [&]() {
      // ---- gather dL/df* (streaming transpose: from x + c_q) as asynchronous
      // copies into shared memory, in flight during the forward recompute
#pragma unroll
      for (int i = 0; i < kQ; ++i) cp_async4(&lsm[i][tid], L.in[i] + site + nb(cx27(i), cy27(i), cz27(i)));
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int i = 0; i < kM; ++i)
          cp_async4(&lsm[kQ + kM * b + i][tid], L.in[mslot(b, i)] + site + nb(mx7(i), my7(i), mz7(i)));
      cp_async_commit();
    };
    // 16-bit storage: the state loads first; FP32: the lambda copies first
    // (each measured faster)
    constexpr bool kStateFirst = sizeof(T) == 2;
    if (!kStateFirst) issue_gather();

    // ---- forward recompute (deviation variables, as in the step kernel)
    float sf[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int slot = ODD ? opp27(i) : i;
      sf[i] = ld_state<T>(P.p[slot] + site + src_off<ODD>(nb, cx27(i), cy27(i), cz27(i)));
    }
    float sg[3][kM];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int i = 0; i < kM; ++i)
        sg[b][i] = ld_state<T>(P.p[mslot(b, ODD ? opp7(i) : i)] + site + src_off<ODD>(nb, mx7(i), my7(i), mz7(i)));
    if (kStateFirst) issue_gather();
    // sums of 216 w_i f_i times 1, c_a and c_a c_b, by 1-D passes with (1, 4, 1)
    float drho, jv[3], pv[3][3];
    {
      float tc[3][3][3];
#pragma unroll
      for (int i = 0; i < kQ; ++i) tc[cz27(i) + 1][cy27(i) + 1][cx27(i) + 1] = sf[i];
      const Fc<kFnM0> m0;
      const Fc<kFnM1> m1;
      const Fc<kFnM2> m2;
      float X0[3][3], X1[3][3], X2[3][3], Y[3];
      xpass(tc, m0, X0);
      xpass(tc, m1, X1);
      xpass(tc, m2, X2);
      ypass(X0, m0, Y);
      drho = zpass(Y, m0) / 216.f;
      jv[2] = zpass(Y, m1);
      pv[2][2] = zpass(Y, m2);
      ypass(X0, m1, Y);
      jv[1] = zpass(Y, m0);
      pv[1][2] = zpass(Y, m1);
      ypass(X0, m2, Y);
      pv[1][1] = zpass(Y, m0);
      ypass(X1, m0, Y);
      jv[0] = zpass(Y, m0);
      pv[0][2] = zpass(Y, m1);
      ypass(X1, m1, Y);
      pv[0][1] = zpass(Y, m0);
      ypass(X2, m0, Y);
      pv[0][0] = zpass(Y, m0);
    }
    const float rho = k.rho0 + drho;
    const float U[3] = {jv[0] / (216.f * rho), jv[1] / (216.f * rho), jv[2] / (216.f * rho)};
    float dB[3], lam[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      dB[b] = 0.25f * sg[b][0] + 0.125f * (sg[b][1] + sg[b][2] + sg[b][3] + sg[b][4] + sg[b][5] + sg[b][6]);
      lam[0][b] = 0.125f * (sg[b][1] - sg[b][2]);
      lam[1][b] = 0.125f * (sg[b][3] - sg[b][4]);
      lam[2][b] = 0.125f * (sg[b][5] - sg[b][6]);
    }
    const float B[3] = {k.Bref[0] + dB[0], k.Bref[1] + dB[1], k.Bref[2] + dB[2]};
    const float gam = 4.f * k.omegaB, al = k.alphaH;
    const float Av[3] = {lam[1][2] - lam[2][1], lam[2][0] - lam[0][2], lam[0][1] - lam[1][0]};
    float yv[3];
    {
      const float uxb[3] = {U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2], U[0] * B[1] - U[1] * B[0]};
#pragma unroll
      for (int a = 0; a < 3; ++a) yv[a] = -gam * (Av[a] - 2.f * uxb[a]);
    }
    const float s = 2.f * gam * al;
    const float b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const float iden = 1.f / (1.f + s * s * b2);
    float J[3], V[3];
    {
      const float yxb[3] = {yv[1] * B[2] - yv[2] * B[1], yv[2] * B[0] - yv[0] * B[2], yv[0] * B[1] - yv[1] * B[0]};
      const float yb = yv[0] * B[0] + yv[1] * B[1] + yv[2] * B[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        J[a] = (yv[a] - s * yxb[a] + s * s * yb * B[a]) * iden;
        V[a] = U[a] - al * J[a];
      }
    }
    // D = (1 - w) dev(Pi - rho U U - M(B)); in deviations dev(Pi~ - rho U U + N)
    float D[3][3];
    {
      const float Br[3] = {k.Bref[0], k.Bref[1], k.Bref[2]};
      float S[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
          const float N = Br[a] * dB[b] + dB[a] * Br[b] + dB[a] * dB[b];
          S[a][b] = pv[a][b] / 216.f - rho * U[a] * U[b] + N;
        }
      const float r = 1.f - k.omega;
      const float tr3 = (S[0][0] + S[1][1] + S[2][2]) / 3.f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) D[a][b] = r * (a == b ? S[a][b] - tr3 : S[a][b]);
    }

    cp_async_wait_all();

    // ---- magnetic collision
    const float omB = k.omegaB;
    float Bb[3], Vb[3], Q[3][3];  // Q[a][b] = sum_i mu_bi xi_ia
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float l[kM];
#pragma unroll
      for (int i = 0; i < kM; ++i) l[i] = lgv(b, i);
      float m0 = 0.25f * l[0];
#pragma unroll
      for (int i = 1; i < kM; ++i) m0 += 0.125f * l[i];
      Bb[b] = omB * m0;
#pragma unroll
      for (int a = 0; a < 3; ++a) Q[a][b] = omB * 0.125f * (l[2 * a + 1] - l[2 * a + 2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float qtv = 0.f, qv = 0.f, qb = 0.f, qtb = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        qtv += Q[a][c] * V[a];
        qv += Q[c][a] * V[a];
        qb += Q[c][a] * B[a];
        qtb += Q[a][c] * B[a];
      }
      Bb[c] += 4.f * (qtv - qv);
      Vb[c] = 4.f * (qb - qtb);
    }
    float Ub[3] = {Vb[0], Vb[1], Vb[2]};
    float Jb[3] = {-al * Vb[0], -al * Vb[1], -al * Vb[2]};
    float abar = -(Vb[0] * J[0] + Vb[1] * J[1] + Vb[2] * J[2]);
    // J = M^-1 y
    float lJ[3];
    {
      const float jxb[3] = {Jb[1] * B[2] - Jb[2] * B[1], Jb[2] * B[0] - Jb[0] * B[2], Jb[0] * B[1] - Jb[1] * B[0]};
      const float jb = Jb[0] * B[0] + Jb[1] * B[1] + Jb[2] * B[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) lJ[a] = (Jb[a] + s * jxb[a] + s * s * jb * B[a]) * iden;
    }
    {
      const float JxB[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2], J[0] * B[1] - J[1] * B[0]};
      const float sbar = -(lJ[0] * JxB[0] + lJ[1] * JxB[1] + lJ[2] * JxB[2]);
      abar += 2.f * gam * sbar;
      const float lxj[3] = {lJ[1] * J[2] - lJ[2] * J[1], lJ[2] * J[0] - lJ[0] * J[2], lJ[0] * J[1] - lJ[1] * J[0]};
#pragma unroll
      for (int a = 0; a < 3; ++a) Bb[a] -= s * lxj[a];
    }
    // y = -gamma (A - 2 U x B)
    float Lb[3][3];
    {
      const float* yb = lJ;
      const float bxy[3] = {B[1] * yb[2] - B[2] * yb[1], B[2] * yb[0] - B[0] * yb[2], B[0] * yb[1] - B[1] * yb[0]};
      const float yxu[3] = {yb[1] * U[2] - yb[2] * U[1], yb[2] * U[0] - yb[0] * U[2], yb[0] * U[1] - yb[1] * U[0]};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Ub[a] += 2.f * gam * bxy[a];
        Bb[a] += 2.f * gam * yxu[a];
      }
      const float Ab[3] = {-gam * yb[0], -gam * yb[1], -gam * yb[2]};
      Lb[0][0] = Lb[1][1] = Lb[2][2] = 0.f;
      Lb[1][2] = Ab[0];
      Lb[2][1] = -Ab[0];
      Lb[2][0] = Ab[1];
      Lb[0][2] = -Ab[1];
      Lb[0][1] = Ab[2];
      Lb[1][0] = -Ab[2];
    }

    // ---- fluid collision: contractions of fbar* = lf with products of 1-D
    // functions (grouped by the x function, 1-D passes)
    const Axis ax(U[0]), ay(U[1]), az(U[2]);
    const float Dxx = D[0][0], Dyy = D[1][1], Dzz = D[2][2], Dxy = D[0][1], Dxz = D[0][2], Dyz = D[1][2];
    float rb, Ueq[3], UP[3] = {0.f, 0.f, 0.f};
    float Dbxx, Dbyy, Dbzz, Dbxy, Dbxz, Dbyz;
    float r0, R[3][3];
    {
      float tl[3][3][3];
#pragma unroll
      for (int i = 0; i < kQ; ++i) tl[cz27(i) + 1][cy27(i) + 1][cx27(i) + 1] = lds(&lsm[i][tid]);
      const Fv Px{ax.psi}, Py{ay.psi}, Pz{az.psi}, DPx{ax.dpsi}, DPy{ay.dpsi}, DPz{az.dpsi};
      const Fv F0x{ax.F0}, F0y{ay.F0}, F0z{az.F0}, F1x{ax.F1}, F1y{ay.F1}, F1z{az.F1};
      const Fc<kFnF2> F2c;
      const Fc<kFnDF1> dF1c;
      const Fc<kFnW> Wc;
      const Fc<kFnWC> WCc;
      const Fc<kFnWC2> WC2c;
      float X[3][3], Y[3];
      // equilibrium: rho prod psi and its U derivatives
      xpass(tl, Px, X);
      ypass(X, Py, Y);
      rb = zpass(Y, Pz);
      Ueq[2] = zpass(Y, DPz);
      ypass(X, DPy, Y);
      Ueq[1] = zpass(Y, Pz);
      xpass(tl, DPx, X);
      ypass(X, Py, Y);
      Ueq[0] = zpass(Y, Pz);
      // P(D, U): Dbar and the U derivatives (dF0 = F1)
      xpass(tl, F0x, X);
      ypass(X, F2c, Y);
      Dbyy = zpass(Y, F0z);
      UP[2] = fmaf(Dyy, zpass(Y, F1z), UP[2]);
      ypass(X, F0y, Y);
      Dbzz = zpass(Y, F2c);
      ypass(X, F1y, Y);
      Dbyz = zpass(Y, F1z);
      UP[1] = fmaf(Dzz, zpass(Y, F2c), UP[1]);
      UP[2] = fmaf(Dyz, zpass(Y, dF1c), UP[2]);
      ypass(X, dF1c, Y);
      UP[1] = fmaf(Dyz, zpass(Y, F1z), UP[1]);
      xpass(tl, F1x, X);
      ypass(X, F1y, Y);
      Dbxy = zpass(Y, F0z);
      {
        const float t111 = zpass(Y, F1z);
        UP[0] = fmaf(Dyz, t111, UP[0]);
        UP[1] = fmaf(Dxz, t111, UP[1]);
        UP[2] = fmaf(Dxy, t111, UP[2]);
      }
      ypass(X, F0y, Y);
      Dbxz = zpass(Y, F1z);
      UP[0] = fmaf(Dzz, zpass(Y, F2c), UP[0]);
      UP[2] = fmaf(Dxz, zpass(Y, dF1c), UP[2]);
      ypass(X, F2c, Y);
      UP[0] = fmaf(Dyy, zpass(Y, F0z), UP[0]);
      ypass(X, dF1c, Y);
      UP[1] = fmaf(Dxy, zpass(Y, F0z), UP[1]);
      xpass(tl, F2c, X);
      ypass(X, F0y, Y);
      Dbxx = zpass(Y, F0z);
      UP[2] = fmaf(Dxx, zpass(Y, F1z), UP[2]);
      ypass(X, F1y, Y);
      UP[1] = fmaf(Dxx, zpass(Y, F0z), UP[1]);
      xpass(tl, dF1c, X);
      ypass(X, F1y, Y);
      UP[0] = fmaf(Dxy, zpass(Y, F0z), UP[0]);
      ypass(X, F0y, Y);
      UP[0] = fmaf(Dxz, zpass(Y, F1z), UP[0]);
      // Lorentz term: r0 = sum w_i fbar_i, R_ab = sum w_i fbar_i c_a c_b
      xpass(tl, Wc, X);
      ypass(X, Wc, Y);
      r0 = zpass(Y, Wc);
      R[2][2] = zpass(Y, WC2c);
      ypass(X, WC2c, Y);
      R[1][1] = zpass(Y, Wc);
      ypass(X, WCc, Y);
      R[1][2] = zpass(Y, WCc);
      xpass(tl, WC2c, X);
      ypass(X, Wc, Y);
      R[0][0] = zpass(Y, Wc);
      xpass(tl, WCc, X);
      ypass(X, WCc, Y);
      R[0][1] = zpass(Y, Wc);
      ypass(X, Wc, Y);
      R[0][2] = zpass(Y, WCc);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) Ub[a] += rho * Ueq[a] + UP[a];
    // Lorentz: H = R - r0 I / 3
    {
      const float H[3][3] = {{R[0][0] - r0 / 3.f, R[0][1], R[0][2]},
                             {R[0][1], R[1][1] - r0 / 3.f, R[1][2]},
                             {R[0][2], R[1][2], R[2][2] - r0 / 3.f}};
      const float trH = H[0][0] + H[1][1] + H[2][2];
#pragma unroll
      for (int a = 0; a < 3; ++a) Bb[a] += 4.5f * (trH * B[a] - 2.f * (H[a][0] * B[0] + H[a][1] * B[1] + H[a][2] * B[2]));
    }
    // D -> S -> (Pi, rho, U, B)
    const float r = 1.f - k.omega;
    const float trD3 = (Dbxx + Dbyy + Dbzz) / 3.f;
    const float Sb[3][3] = {{r * (Dbxx - trD3), r * Dbxy, r * Dbxz},
                            {r * Dbxy, r * (Dbyy - trD3), r * Dbyz},
                            {r * Dbxz, r * Dbyz, r * (Dbzz - trD3)}};
    {
      const float trS = Sb[0][0] + Sb[1][1] + Sb[2][2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        rb -= Sb[a][a] * U[a] * U[a];
        Ub[a] -= 2.f * rho * Sb[a][a] * U[a];
        Bb[a] += -trS * B[a] + 2.f * Sb[a][a] * B[a];
      }
      const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int a = pa[p], b = pb[p];
        rb -= Sb[a][b] * U[a] * U[b];
        Ub[a] -= rho * Sb[a][b] * U[b];
        Ub[b] -= rho * Sb[a][b] * U[a];
        Bb[a] += Sb[a][b] * B[b];
        Bb[b] += Sb[a][b] * B[a];
      }
    }
    // U = j / rho
    const float jb[3] = {Ub[0] / rho, Ub[1] / rho, Ub[2] / rho};
    rb -= (Ub[0] * U[0] + Ub[1] * U[1] + Ub[2] * U[2]) / rho;

    // ---- moments -> populations: fbar_i = rhobar + jbar.c_i + Pibar : c_i c_i,
    // per (c_x, c_y) column as base + lin c_z + Pibar_zz c_z^2
#pragma unroll
    for (int py = 0; py < 3; ++py)
#pragma unroll
      for (int px = 0; px < 3; ++px) {
        const int cx = px - 1, cy = py - 1;
        float base = rb, lin = jb[2];
        if (cx != 0) {
          base += (cx > 0 ? jb[0] : -jb[0]) + Sb[0][0];
          lin += cx > 0 ? Sb[0][2] : -Sb[0][2];
        }
        if (cy != 0) {
          base += (cy > 0 ? jb[1] : -jb[1]) + Sb[1][1];
          lin += cy > 0 ? Sb[1][2] : -Sb[1][2];
        }
        if (cx * cy != 0) base += cx * cy > 0 ? Sb[0][1] : -Sb[0][1];
        const float side = base + Sb[2][2];
        L.out[idx27(px, py, 0)][site] = side - lin;
        L.out[idx27(px, py, 1)][site] = base;
        L.out[idx27(px, py, 2)][site] = side + lin;
      }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int i = 0; i < kM; ++i) {
        float v = (1.f - omB) * lgv(b, i) + Bb[b];
        if (i > 0) {
          const int a = (i - 1) >> 1;
          v += (i & 1) ? Lb[a][b] : -Lb[a][b];
        }
        L.out[mslot(b, i)][site] = v;
      }
    abar_site = (double)abar;
  }
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int warp = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
  warp_sum_to(abar_site, partials + blk * ((blockDim.x * blockDim.y) >> 5) + warp);
}

// ---------------------------------------------------------------------------
// Initialisation adjoint (FP64), local part: per site the contributions to
// u_bar and B_bar that do not go through a gradient, and the adjoints of the
// central-difference gradients (d_a u_b, d_a B_b at [3a+b]).
__global__ void init_adjoint_local_kernel(Grid g, StepConsts k, const double* __restrict__ u,
                                          const double* __restrict__ Bf, const float* __restrict__ lam,
                                          double* __restrict__ ubl, double* __restrict__ Bbl,
                                          double* __restrict__ dub, double* __restrict__ dBb,
                                          double* __restrict__ partials) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  double abar = 0.0;
  if (x < g.nx && y < g.ny) {
    const long long n3 = g.n3;
    const long long site = ((long long)z * g.ny + y) * g.nx + x;
    const double U[3] = {u[site], u[n3 + site], u[2 * n3 + site]};
    const double B[3] = {Bf[site], Bf[n3 + site], Bf[2 * n3 + site]};
    // central-difference gradient of B for J0 = curl B
    const int xp = x + 1 == g.nx ? 0 : x + 1, xm = x == 0 ? g.nx - 1 : x - 1;
    const int yp = y + 1 == g.ny ? 0 : y + 1, ym = y == 0 ? g.ny - 1 : y - 1;
    const int zp = z + 1 == g.nz ? 0 : z + 1, zm = z == 0 ? g.nz - 1 : z - 1;
    auto at = [&](int xx, int yy, int zz) { return ((long long)zz * g.ny + yy) * g.nx + xx; };
    double dB[3][3];
    for (int b = 0; b < 3; ++b) {
      const double* F = Bf + b * n3;
      dB[0][b] = 0.5 * (F[at(xp, y, z)] - F[at(xm, y, z)]);
      dB[1][b] = 0.5 * (F[at(x, yp, z)] - F[at(x, ym, z)]);
      dB[2][b] = 0.5 * (F[at(x, y, zp)] - F[at(x, y, zm)]);
    }
    const double al = (double)k.alphaH, omB = (double)k.omegaB, om = (double)k.omega;
    const double J0[3] = {dB[1][2] - dB[2][1], dB[2][0] - dB[0][2], dB[0][1] - dB[1][0]};
    const double V[3] = {U[0] - al * J0[0], U[1] - al * J0[1], U[2] - al * J0[2]};
    double lf[kQ], lg[3][kM];
    for (int i = 0; i < kQ; ++i) lf[i] = (double)lam[(long long)i * n3 + site];
    for (int b = 0; b < 3; ++b)
      for (int i = 0; i < kM; ++i) lg[b][i] = (double)lam[(long long)mslot(b, i) * n3 + site];
    // H = sum_i lf w H2; Lorentz part of B_bar; equilibrium part of u_bar
    double r0 = 0.0, R[3][3] = {{0.0}}, Ub[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < kQ; ++i) {
      const int c[3] = {cx27(i), cy27(i), cz27(i)};
      const double wt = w27d(i) * lf[i];
      r0 += wt;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R[a][b] += wt * c[a] * c[b];
      double ps[3], dps[3];
      for (int a = 0; a < 3; ++a) {
        const double uu = U[a] * U[a];
        ps[a] = c[a] == 0 ? 2.0 / 3.0 - uu : 0.5 * (1.0 / 3.0 + uu + c[a] * U[a]);
        dps[a] = c[a] == 0 ? -2.0 * U[a] : U[a] + 0.5 * c[a];
      }
      Ub[0] += lf[i] * dps[0] * ps[1] * ps[2];
      Ub[1] += lf[i] * ps[0] * dps[1] * ps[2];
      Ub[2] += lf[i] * ps[0] * ps[1] * dps[2];
    }
    double H[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) H[a][b] = R[a][b] - (a == b ? r0 / 3.0 : 0.0);
    const double trH = H[0][0] + H[1][1] + H[2][2];
    double Bb[3];
    for (int a = 0; a < 3; ++a) Bb[a] = 4.5 * (trH * B[a] - 2.0 * (H[a][0] * B[0] + H[a][1] * B[1] + H[a][2] * B[2]));
    // Hall equilibrium: mu = W lg, m0, Q[a][b] = sum_i mu_bi xi_ia
    double Q[3][3], Vb[3];
    for (int b = 0; b < 3; ++b) {
      double m0 = 0.25 * lg[b][0];
      for (int i = 1; i < kM; ++i) m0 += 0.125 * lg[b][i];
      Bb[b] += m0;
      for (int a = 0; a < 3; ++a) Q[a][b] = 0.125 * (lg[b][2 * a + 1] - lg[b][2 * a + 2]);
    }
    for (int c = 0; c < 3; ++c) {
      double qtv = 0.0, qv = 0.0, qb = 0.0, qtb = 0.0;
      for (int a = 0; a < 3; ++a) {
        qtv += Q[a][c] * V[a];
        qv += Q[c][a] * V[a];
        qb += Q[c][a] * B[a];
        qtb += Q[a][c] * B[a];
      }
      Bb[c] += 4.0 * (qtv - qv);
      Vb[c] = 4.0 * (qb - qtb);
    }
    for (int a = 0; a < 3; ++a) Ub[a] += Vb[a];
    const double J0b[3] = {-al * Vb[0], -al * Vb[1], -al * Vb[2]};
    abar = -(Vb[0] * J0[0] + Vb[1] * J0[1] + Vb[2] * J0[2]);
    double db[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) db[a][b] = -Q[a][b] / omB;
    db[1][2] += J0b[0];
    db[2][1] -= J0b[0];
    db[2][0] += J0b[1];
    db[0][2] -= J0b[1];
    db[0][1] += J0b[2];
    db[1][0] -= J0b[2];
    for (int a = 0; a < 3; ++a) {
      ubl[a * n3 + site] = Ub[a];
      Bbl[a * n3 + site] = Bb[a];
      for (int b = 0; b < 3; ++b) {
        dBb[(3 * a + b) * n3 + site] = db[a][b];
        dub[(3 * a + b) * n3 + site] = -(3.0 / om) * H[a][b];  // rho = 1 initial density
      }
    }
  }
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  block_sum_to(abar, partials + blk);
}

// Transpose of the periodic central difference: F_bar(y) += 1/2 (G(y - e_a) - G(y + e_a)).
__global__ void init_adjoint_stencil_kernel(Grid g, const double* __restrict__ ubl, const double* __restrict__ Bbl,
                                            const double* __restrict__ dub, const double* __restrict__ dBb,
                                            double* __restrict__ ubar, double* __restrict__ Bbar) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  if (x >= g.nx || y >= g.ny) return;
  const long long n3 = g.n3;
  const long long site = ((long long)z * g.ny + y) * g.nx + x;
  const int xp = x + 1 == g.nx ? 0 : x + 1, xm = x == 0 ? g.nx - 1 : x - 1;
  const int yp = y + 1 == g.ny ? 0 : y + 1, ym = y == 0 ? g.ny - 1 : y - 1;
  const int zp = z + 1 == g.nz ? 0 : z + 1, zm = z == 0 ? g.nz - 1 : z - 1;
  const long long m[3] = {((long long)z * g.ny + y) * g.nx + xm, ((long long)z * g.ny + ym) * g.nx + x,
                          ((long long)zm * g.ny + y) * g.nx + x};
  const long long p[3] = {((long long)z * g.ny + y) * g.nx + xp, ((long long)z * g.ny + yp) * g.nx + x,
                          ((long long)zp * g.ny + y) * g.nx + x};
  for (int b = 0; b < 3; ++b) {
    double vb = Bbl[b * n3 + site], vu = ubl[b * n3 + site];
    for (int a = 0; a < 3; ++a) {
      const double* G = dBb + (3 * a + b) * n3;
      const double* Gu = dub + (3 * a + b) * n3;
      vb += 0.5 * (G[m[a]] - G[p[a]]);
      vu += 0.5 * (Gu[m[a]] - Gu[p[a]]);
    }
    if (Bbar) Bbar[b * n3 + site] = vb;
    if (ubar) ubar[b * n3 + site] = vu;
  }
}

// Deterministic two-level sum of n partials: kSumBlocks blocks sum fixed
// chunks into stage[], then one block sums the stage.
constexpr int kSumBlocks = 256;
__global__ void sum_chunks_kernel(const double* __restrict__ partials, long long n, double* __restrict__ stage) {
  __shared__ double sh[256];
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = per * blockIdx.x, hi = lo + per < n ? lo + per : n;
  double a = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) a += partials[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) stage[blockIdx.x] = sh[0];
}
__global__ void sum_partials_kernel(const double* __restrict__ partials, long long n, double* __restrict__ out) {
  __shared__ double sh[256];
  double a = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) a += partials[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}
// Sum of n partials (the buffer holds n + kSumBlocks doubles) into *out.
inline void sum_partials(double* partials, long long n, double* out, cudaStream_t s) {
  sum_chunks_kernel<<<kSumBlocks, 256, 0, s>>>(partials, n, partials + n);
  sum_partials_kernel<<<1, 256, 0, s>>>(partials + n, kSumBlocks, out);
}

template <class T>
cudaError_t adjoint_t(int odd, const void* pop, Grid g, const StepConsts& k, const float* lin, float* lout,
                      double* partials, double* ddi, cudaStream_t s) {
  const dim3 b = site_block(g, kAdjThreads<T>), gr = site_grid(g, b);
  const long long nblk = (long long)gr.x * gr.y * gr.z;
  const Slots<T> P = make_slots<T>(pop, g);
  LamSlots L;
  for (int q = 0; q < kPop; ++q) {
    L.in[q] = lin + (size_t)q * (size_t)g.n3;
    L.out[q] = lout + (size_t)q * (size_t)g.n3;
  }
  if (odd)
    adjoint_step_kernel<T, true><<<gr, b, 0, s>>>(P, g, k, L, partials);
  else
    adjoint_step_kernel<T, false><<<gr, b, 0, s>>>(P, g, k, L, partials);
  sum_partials(partials, nblk * ((b.x * b.y) >> 5), ddi, s);
  return cudaGetLastError();
}

}  // namespace

long long adjoint_partials_needed(Grid g) {
  // per warp of the step kernel (either block shape), per block of the
  // initialisation adjoint
  long long need = 0;
  for (int threads : {kAdjThreads<float>, kAdjThreads<__half>}) {
    const dim3 b = site_block(g, threads), gr = site_grid(g, b);
    const long long a = (long long)gr.x * gr.y * gr.z * ((b.x * b.y) >> 5);
    if (a > need) need = a;
  }
  const dim3 bi = site_block(g, 128), gi = site_grid(g, bi);
  const long long c = (long long)gi.x * gi.y * gi.z;
  return (need > c ? need : c) + kSumBlocks;
}

cudaError_t launch_step_adjoint(int storage, int odd, const void* pop, Grid g, const StepConsts& k, const float* lin,
                                float* lout, double* partials, double* ddi, cudaStream_t s) {
  switch (storage) {
    case 1: return adjoint_t<float>(odd, pop, g, k, lin, lout, partials, ddi, s);
    case 2: return adjoint_t<__half>(odd, pop, g, k, lin, lout, partials, ddi, s);
    case 3: return adjoint_t<__nv_bfloat16>(odd, pop, g, k, lin, lout, partials, ddi, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_init_adjoint(Grid g, const StepConsts& k, const double* u, const double* B, const float* lam,
                                double* ws, double* partials, double* ubar, double* Bbar, double* ddi,
                                cudaStream_t s) {
  const dim3 b = site_block(g, 128), gr = site_grid(g, b);
  const long long n3 = g.n3;
  double* ubl = ws;
  double* Bbl = ws + 3 * n3;
  double* dub = ws + 6 * n3;
  double* dBb = ws + 15 * n3;
  init_adjoint_local_kernel<<<gr, b, 0, s>>>(g, k, u, B, lam, ubl, Bbl, dub, dBb, partials);
  init_adjoint_stencil_kernel<<<gr, b, 0, s>>>(g, ubl, Bbl, dub, dBb, ubar, Bbar);
  sum_partials(partials, (long long)gr.x * gr.y * gr.z, ddi, s);
  return cudaGetLastError();
}

}  // namespace flame
