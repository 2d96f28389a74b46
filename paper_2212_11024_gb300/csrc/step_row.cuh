// step_row.cuh -- the row kernel: the fused FLAME collide-and-stream step for
// 16-bit storage as a persistent kernel over x rows, two sites per thread,
// with the per-site FP32 arithmetic in packed pairs (one Blackwell f32x2 add /
// multiply / fused multiply-add does the same operation for both sites).
//
// Algebra and order of the steps (Sec. 3: a1 load + decode, a2 rho and U,
// a3 B and Lambda, a4 J, a6 Hall BGK, a5 central-moment fluid collision, a7
// encode and AA store) are those of the one-site kernel in step.cu, and so
// is the layout of the state.  What differs is the data movement:
//  - For each tile (one x row (y, z)) warp 0 stages the 48 source rows of
//    the AA pattern in shared memory with TMA copies completed on an
//    mbarrier: the row (y, z) of every slot on even steps (one tensor-map
//    box), the row (y, z) - (c_y, c_z) of the opposite slot on odd steps
//    (16 boxes of three consecutive storage slots, see phys()).  Two or
//    three stages: the copies of the next tiles overlap the arithmetic of
//    this one.
//  - The x shift of the odd step becomes a wrap-around index into the
//    staged row.  Thread t takes the sites (2t, 2t + 1); unshifted values
//    are read and written as one 32-bit pair.
//  - The collision writes its results in place into the staged rows (under
//    the AA pattern each result lands where the same thread read), and warp
//    0 writes the tile back with TMA stores to the rows it was loaded from.
//    Rows longer than 256 sites write their results straight to HBM instead
//    (their two stages are then refilled without waiting for a store).
//  - The packed arithmetic halves the FP32 instruction count per site,
//    which is what limited the one-site kernel with 16-bit storage.
// The scheme variants are instantiations of the same kernel (template
// parameter VAR): the BGK fluid collision (Sec. 3.1.1), the electron-MHD
// magnetic equilibrium (Sec. 5) and the current from the central-difference
// curl of B (read from the field that step.cu's pre-pass writes in the
// storage's type).  Each
// variant is instantiated in a translation unit of its own (step_row.cu,
// step_row_bgk.cu, step_row_emhd.cu, step_row_fd.cu), so they compile in
// parallel.
// Requirements: 16-bit storage, 64 <= nx <= 1024 with nx a multiple of 8
// (rows of whole 16-byte units; half rows per tile: of 16), a 16-byte
// aligned state.  Rows of up to 256 sites are staged by tensor-map boxes of
// runs of three rows (or one box of all 48 when the runs are dense), each
// run at a 128-byte aligned place in shared memory (run_stride); longer rows
// by one bulk copy per storage slot.  Warp 0, which issues the copies, is always
// whole (nx / 2 >= 32 threads); the last warp of a block may be partial.
// The same packed collision also runs unstaged (step_pair_kernel: loads and
// stores straight from HBM, any even row length).  flame_step picks among
// whole rows, half rows and the pair kernel by row length
// (row_auto_segments).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "aa.cuh"

namespace flame {

// Tensor maps of the state as [48][nz][ny][nx]: one box of a row of all 48
// slots (even steps) and one of a row of 3 consecutive slots (odd steps).
struct RowMaps {
  CUtensorMap all, run;
};

// Wait limit and the failure-path test of the waits: with stall set, every
// stage's barrier is armed for its bytes but no copy is issued, so each wait
// runs out after `tries` polls (and no copy is ever in flight).
struct RowWait {
  unsigned tries;
  int stall;
};

// One step of the row kernel: storage 2 FP16 / 3 BF16, AA parity odd; Bfd
// the pre-collision B - B_ref ([3][N3], storage type) for the finite-difference
// current, else unused; launch false only settles the launch configuration.
struct RowCall {
  int storage, odd;
  int segments;  // 1: a tile is a whole row; 2: half a row (rows of more than 256 sites);
                 // 0: no staging (the pair kernel)
  void* pop;
  Grid g;
  StepConsts k;
  unsigned* flag;
  const void* Bfd;
  cudaStream_t s;
  bool launch;
  RowWait wt;
};

// Tensor maps of a state (step_row.cu), cached per host thread.
cudaError_t row_maps(const void* pop, const Grid& g, RowMaps* out);

// The step per scheme variant, one translation unit each.
cudaError_t step_row_flame(const RowCall& c);  // step_row.cu
cudaError_t step_row_bgk(const RowCall& c);    // step_row_bgk.cu
cudaError_t step_row_emhd(const RowCall& c);   // step_row_emhd.cu
cudaError_t step_row_fd(const RowCall& c);     // step_row_fd.cu

namespace {

// ----------------------------------------------------------- packed FP32
struct f2 {
  float2 v;
};
__device__ __forceinline__ f2 splat(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ f2 pack(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator*(float s, f2 b) { return {__fmul2_rn(make_float2(s, s), b.v)}; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ f2 fma2(float s, f2 b, f2 c) { return {__ffma2_rn(make_float2(s, s), b.v, c.v)}; }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  f2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.v.x), "=f"(d.v.y)
      : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
  return d;
}

// Two adjacent 16-bit values as one 32-bit word.
template <class T>
struct Codec2;
template <>
struct Codec2<__half> {
  static __device__ __forceinline__ f2 dec(const __half* p) { return {__half22float2(*reinterpret_cast<const __half2*>(p))}; }
  static __device__ __forceinline__ void enc(__half* p, f2 v) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.v.x, v.v.y);
  }
};
template <>
struct Codec2<__nv_bfloat16> {
  static __device__ __forceinline__ f2 dec(const __nv_bfloat16* p) {
    return {__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p))};
  }
  static __device__ __forceinline__ void enc(__nv_bfloat16* p, f2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.v.x, v.v.y);
  }
};

// --------------------------------------------------- per-pair arithmetic
// One collision of two sites.  ldf(px, py, pz) returns the decoded
// pre-collision fluid population of velocity (px-1, py-1, pz-1), ldg(c, i)
// the magnetic one of component c and D3Q7 velocity i; stf(px, py, pz, v)
// and stg(c, i, v) take the post-collision values of the same velocities.
// VAR is the scheme variant; curl_b(J) gives the central-difference curl of
// the pre-collision B at both sites (used by kVarFdCurrent only); mid() runs
// between the magnetic and the fluid collision (the pipeline's hook).
template <int VAR, class LdF, class LdG, class StF, class StG, class CurlB, class Mid>
__device__ __forceinline__ void collide_pair(const LdF& ldf, const LdG& ldg, const StF& stf, const StG& stg,
                                             const CurlB& curl_b, const Mid& mid, const StepConsts& k,
                                             unsigned* __restrict__ flag) {
  // a2: 1-D passes with the weights (1, 4, 1) / 6 (x, then y, then z).
  f2 m0[9], m1[9], m2[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int py = q % 3, pz = q / 3;
    const f2 sm = ldf(0, py, pz), s0 = ldf(1, py, pz), sp = ldf(2, py, pz);
    const f2 t = sp + sm;
    m0[q] = fma2(4.f, s0, t);
    m1[q] = sp - sm;
    m2[q] = t;
  }
  f2 M00[3], M10[3], M20[3], M01[3], M11[3], M02[3];
#pragma unroll
  for (int pz = 0; pz < 3; ++pz) {
    const int q = 3 * pz;
    const f2 t0 = m0[q + 2] + m0[q];
    M00[pz] = fma2(4.f, m0[q + 1], t0);
    M02[pz] = t0;
    M01[pz] = m0[q + 2] - m0[q];
    M10[pz] = fma2(4.f, m1[q + 1], m1[q + 2] + m1[q]);
    M11[pz] = m1[q + 2] - m1[q];
    M20[pz] = fma2(4.f, m2[q + 1], m2[q + 2] + m2[q]);
  }
  // The density deviation is divided exactly (mass stays unbiased); U and
  // Pi use the reciprocals of 216 rho and of 216.
  const f2 t00 = M00[2] + M00[0];
  const f2 r216 = fma2(4.f, M00[1], t00);
  const f2 drho = pack(r216.v.x / 216.f, r216.v.y / 216.f);
  const f2 rho = splat(k.rho0) + drho;
  const f2 irho216 = pack(1.f / (216.f * rho.v.x), 1.f / (216.f * rho.v.y));
  const f2 U[3] = {fma2(4.f, M10[1], M10[2] + M10[0]) * irho216, fma2(4.f, M01[1], M01[2] + M01[0]) * irho216,
                   (M00[2] - M00[0]) * irho216};
  constexpr float k216 = 1.f / 216.f;
  const f2 pxx = k216 * fma2(4.f, M20[1], M20[2] + M20[0]);
  const f2 pyy = k216 * fma2(4.f, M02[1], M02[2] + M02[0]);
  const f2 pzz = k216 * t00;
  const f2 pxy = k216 * fma2(4.f, M11[1], M11[2] + M11[0]);
  const f2 pxz = k216 * (M10[2] - M10[0]);
  const f2 pyz = k216 * (M01[2] - M01[0]);

  // a3: B = sum_i g_i, Lambda_ab = sum_i xi_ia g_ib (deviations from rest).
  f2 sg[3][kM], dB[3], lam[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int i = 0; i < kM; ++i) sg[c][i] = ldg(c, i);
    dB[c] = fma2(0.25f, sg[c][0], 0.125f * (((sg[c][1] + sg[c][2]) + (sg[c][3] + sg[c][4])) + (sg[c][5] + sg[c][6])));
    lam[0][c] = 0.125f * (sg[c][1] - sg[c][2]);
    lam[1][c] = 0.125f * (sg[c][3] - sg[c][4]);
    lam[2][c] = 0.125f * (sg[c][5] - sg[c][6]);
  }
  const f2 B[3] = {splat(k.Bref[0]) + dB[0], splat(k.Bref[1]) + dB[1], splat(k.Bref[2]) + dB[2]};

  {
    const f2 chk = ((drho + U[0]) + (U[1] + U[2])) + ((dB[0] + dB[1]) + dB[2]);
    if (!isfinite(chk.v.x + chk.v.y)) {
      if (*((volatile unsigned*)flag) == 0u) atomicOr(flag, 1u);
    }
  }

  // a4: J from J + s J x B = y (closed form), V = U - alpha_H J.  Electron
  // MHD drops U here and in g^Hall(0); the finite-difference variant takes J
  // from the curl of the pre-collision field.
  f2 V[3];
  if constexpr (VAR == kVarFdCurrent) {
    f2 J[3];
    curl_b(J);
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a] = fma2(-k.alphaH, J[a], U[a]);
  } else {
    const float gq = 4.f * k.omegaB, sH = 2.f * k.alphaH * gq;
    const f2 A[3] = {lam[1][2] - lam[2][1], lam[2][0] - lam[0][2], lam[0][1] - lam[1][0]};
    f2 yv[3];
    if constexpr (VAR == kVarEmhd) {
#pragma unroll
      for (int a = 0; a < 3; ++a) yv[a] = (-gq) * A[a];
    } else {
      const f2 uxb[3] = {U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2], U[0] * B[1] - U[1] * B[0]};
      // y = -gq (A - 2 U x B) = 2 gq (U x B) - gq A
#pragma unroll
      for (int a = 0; a < 3; ++a) yv[a] = fma2(2.f * gq, uxb[a], (-gq) * A[a]);
    }
    const f2 yxb[3] = {yv[1] * B[2] - yv[2] * B[1], yv[2] * B[0] - yv[0] * B[2], yv[0] * B[1] - yv[1] * B[0]};
    const f2 yb = fma2(yv[0], B[0], fma2(yv[1], B[1], yv[2] * B[2]));
    const f2 b2 = fma2(B[0], B[0], fma2(B[1], B[1], B[2] * B[2]));
    const f2 den = fma2(sH * sH, b2, splat(1.f));
    const f2 iden = pack(1.f / den.v.x, 1.f / den.v.y);
    const f2 t = (sH * sH) * yb;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const f2 J = fma2(t, B[a], fma2(-sH, yxb[a], yv[a])) * iden;
      V[a] = VAR == kVarEmhd ? (-k.alphaH) * J : fma2(-k.alphaH, J, U[a]);
    }
  }

  // a6: magnetic BGK towards g^Hall(0): rest dB_b, face (axis a, sign +-)
  // dB_b +- 4 (V_a B_b - B_a V_b); the bracket is antisymmetric in (a, b).
  {
    const float om = k.omegaB, cm = 1.f - k.omegaB;
    const f2 W01 = (4.f * om) * (V[0] * B[1] - B[0] * V[1]);
    const f2 W02 = (4.f * om) * (V[0] * B[2] - B[0] * V[2]);
    const f2 W12 = (4.f * om) * (V[1] * B[2] - B[1] * V[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const f2 omdB = om * dB[c];
      stg(c, 0, fma2(cm, sg[c][0], omdB));
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const f2 W = (a == c) ? splat(0.f) : (a + c == 1 ? W01 : (a + c == 2 ? W02 : W12));
        const bool pos = a < c;
#pragma unroll
        for (int h = 1; h <= 2; ++h) {
          const int i = 2 * a + h;
          const f2 rhs = (a == c) ? omdB : ((h == 1) == pos ? omdB + W : omdB - W);
          stg(c, i, fma2(cm, sg[c][i], rhs));
        }
      }
    }
  }

  mid();

  // a5: fluid.  N = Bref b + b Bref + b b, miso = Bref.b + |b|^2 / 2.
  const f2 bx = dB[0], by = dB[1], bz = dB[2];
  const float Brx = k.Bref[0], Bry = k.Bref[1], Brz = k.Bref[2];
  const f2 Nxx = fma2(2.f * Brx, bx, bx * bx), Nyy = fma2(2.f * Bry, by, by * by), Nzz = fma2(2.f * Brz, bz, bz * bz);
  const f2 Nxy = fma2(Brx, by, fma2(Bry, bx, bx * by));
  const f2 Nxz = fma2(Brx, bz, fma2(Brz, bx, bx * bz));
  const f2 Nyz = fma2(Bry, bz, fma2(Brz, by, by * bz));
  const f2 miso = fma2(Brx, bx, fma2(Bry, by, fma2(Brz, bz, 0.5f * fma2(bx, bx, fma2(by, by, bz * bz)))));
  // (1 - w) dev(Pi - rho U U + N), with nrU = -rho U.
  const f2 nrho = splat(-k.rho0) - drho;
  const f2 nrU[3] = {nrho * U[0], nrho * U[1], nrho * U[2]};
  const f2 Sxx = fma2(nrU[0], U[0], pxx + Nxx), Syy = fma2(nrU[1], U[1], pyy + Nyy),
           Szz = fma2(nrU[2], U[2], pzz + Nzz);
  const float r = 1.f - k.omega;
  const f2 tr3 = (1.f / 3.f) * ((Sxx + Syy) + Szz);
  const f2 Dxx = r * (Sxx - tr3), Dyy = r * (Syy - tr3), Dzz = r * (Szz - tr3);
  const f2 Dxy = r * fma2(nrU[0], U[1], pxy + Nxy);
  const f2 Dxz = r * fma2(nrU[0], U[2], pxz + Nxz);
  const f2 Dyz = r * fma2(nrU[1], U[2], pyz + Nyz);

  // 1-D factors over x and y (divided by the 1-D weight): e = psi/w1 - 1,
  // p0 and p1 the inverse-moment maps of m0 and m1 (p0 = e except at 0).
  f2 ex[3], ey[3], p1x[3], p1y[3];
  {
    const f2 u = U[0], uu = u * u, u3 = 3.f * u, nu3 = -3.f * u;
    ex[0] = fma2(3.f, uu, nu3), ex[1] = -1.5f * uu, ex[2] = fma2(3.f, uu, u3);
    p1x[0] = fma2(6.f, u, splat(-3.f)), p1x[1] = nu3, p1x[2] = fma2(6.f, u, splat(3.f));
  }
  {
    const f2 u = U[1], uu = u * u, u3 = 3.f * u, nu3 = -3.f * u;
    ey[0] = fma2(3.f, uu, nu3), ey[1] = -1.5f * uu, ey[2] = fma2(3.f, uu, u3);
    p1y[0] = fma2(6.f, u, splat(-3.f)), p1y[1] = nu3, p1y[2] = fma2(6.f, u, splat(3.f));
  }
  const f2 p0x[3] = {ex[0], ex[1] + splat(1.5f), ex[2]};
  const f2 p0y[3] = {ey[0], ey[1] + splat(1.5f), ey[2]};
  // along z: ez(c) = e0z + e1z c + e2z c^2, p0z(c) = q00 + e1z c + q20 c^2,
  // p1z(c) = q01 + 3 c + q21 c^2, p2z(c) = -1.5 + 4.5 c^2.
  const f2 uz = U[2], uzz = uz * uz;
  const f2 e0z = -1.5f * uzz, e1z = 3.f * uz, e2z = 4.5f * uzz;
  const f2 q00 = e0z + splat(1.5f), q20 = e2z + splat(-1.5f);
  const f2 q01 = -3.f * uz, q21 = 9.f * uz;
  // Lorentz term 4.5 (miso (|c|^2 - 1) - c.N.c) + 1.5 tr N = Lxy + Lz1 cz + LZ cz^2.
  const f2 Lbase = fma2(1.5f, (Nxx + Nyy) + Nzz, -4.5f * miso);
  const f2 LA = 4.5f * (miso - Nxx), LB = 4.5f * (miso - Nyy), LC = 9.f * Nxy;
  const f2 LZ = 4.5f * (miso - Nzz);
  // drho + Lxy for the classes cx = cy = 0; cx only; cy only; cx cy > 0; cx cy < 0
  const f2 base0 = drho + Lbase, baseA = base0 + LA, baseB = base0 + LB, baseAB = baseA + LB;
  const f2 basePP = baseAB - LC, basePM = baseAB + LC;
  // Lz1 = -9 (cx Nxz + cy Nyz) for cx, cy in {-1, 0, 1}
  const f2 NX = -9.f * Nxz, NY = -9.f * Nyz, mNX = 9.f * Nxz, mNY = 9.f * Nyz;
  const f2 Lpp = NX + NY, Lmm = mNX + mNY, Lpm = NX + mNY, Lmp = mNX + NY;

  // a7: for each (cx, cy) the outputs are Z0 + Z1 cz + Z2 cz^2 (the BGK
  // fluid collision has no projected non-equilibrium part).
  auto column = [&](int px, int py, f2 (&v)[3]) {
    const int cx = px - 1, cy = py - 1;
    const f2 exy = fma2(ex[px], ey[py], ex[px] + ey[py]);
    const f2 gg = fma2(rho, exy, rho);
    const float p2x = px == 1 ? -1.5f : 3.f, p2y = py == 1 ? -1.5f : 3.f;
    const bool bgk = VAR == kVarBgkFluid;
    const f2 A0 = bgk ? splat(0.f) : fma2(p2x * Dxx, p0y[py], fma2(p2y * Dyy, p0x[px], (Dxy * p1x[px]) * p1y[py]));
    const f2 A1 = bgk ? splat(0.f) : fma2(Dxz * p1x[px], p0y[py], (Dyz * p1y[py]) * p0x[px]);
    const f2 A2 = bgk ? splat(0.f) : (Dzz * p0x[px]) * p0y[py];
    const f2 b0 = cx == 0 ? (cy == 0 ? base0 : baseB) : (cy == 0 ? baseA : (cx == cy ? basePP : basePM));
    const f2 Lz1 = cx == 0 ? (cy == 0 ? splat(0.f) : (cy > 0 ? NY : mNY))
                           : (cy == 0 ? (cx > 0 ? NX : mNX)
                                      : (cx > 0 ? (cy > 0 ? Lpp : Lpm) : (cy > 0 ? Lmp : Lmm)));
    const f2 Z0 = fma2(gg, e0z, fma2(A0, q00, fma2(A1, q01, fma2(-1.5f, A2, fma2(rho, exy, b0)))));
    const f2 Z1 = fma2(gg, e1z, fma2(A0, e1z, cx == 0 && cy == 0 ? 3.f * A1 : fma2(3.f, A1, Lz1)));
    const f2 Z2 = fma2(gg, e2z, fma2(A0, q20, fma2(A1, q21, fma2(4.5f, A2, LZ))));
    const f2 tz = Z0 + Z2;
    v[0] = tz - Z1;
    v[1] = Z0;
    v[2] = tz + Z1;
  };
  if constexpr (VAR != kVarBgkFluid) {
#pragma unroll
    for (int py = 0; py < 3; ++py)
#pragma unroll
      for (int px = 0; px < 3; ++px) {
        f2 v[3];
        column(px, py, v);
        stf(px, py, 0, v[0]);
        stf(px, py, 1, v[1]);
        stf(px, py, 2, v[2]);
      }
  } else {
    // f* = (1 - w) f + w f^mhd(0).  The results of column (px, py) go where
    // the mirror column (2 - px, 2 - py) was read, so the pre-collision
    // values of both are read before either is written.  They are read again
    // from shared memory (the compiler barrier keeps the values of a2 from
    // being held in registers through the whole collision).
    asm volatile("" ::: "memory");
    const float om = k.omega, cm = 1.f - k.omega;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int px = c % 3, py = c / 3, qx = 2 - px, qy = 2 - py;
      f2 a[3], b[3], v[3], w[3];
#pragma unroll
      for (int pz = 0; pz < 3; ++pz) {
        a[pz] = ldf(px, py, pz);
        b[pz] = ldf(qx, qy, pz);
      }
      column(px, py, v);
#pragma unroll
      for (int pz = 0; pz < 3; ++pz) stf(px, py, pz, fma2(cm, a[pz], om * v[pz]));
      if (c < 4) {
        column(qx, qy, w);
#pragma unroll
        for (int pz = 0; pz < 3; ++pz) stf(qx, qy, pz, fma2(cm, b[pz], om * w[pz]));
      }
    }
  }
}

// ------------------------------------------- rows staged by TMA, persistent
// At most 512 threads per block (nx <= 1024); launch bounds per instantiation
// (row_bound_threads / row_bound_blocks below); stages: row_stages().
constexpr int kRowMaxThreads = 512;
// Rows up to this length are staged by tensor-map copies (a box is at most
// 256 elements wide), longer ones by one bulk copy per row.
constexpr int kBoxMaxX = 256;
// mbarrier.try_wait returns after a bounded, hardware-defined time; this
// many tries (far longer than any copy takes) end a wait with an error.
constexpr unsigned kWaitTries = 1u << 22;

// Storage slots come in 16 runs of three (see phys()).  On an odd step run r
// is staged from the row (y, z) + (dy, dz): the fluid run r = (cy+1) + 3(cz+1)
// from (cy, cz), the magnetic run 9 + i from the D3Q7 velocity i.
constexpr int kRuns = 16;
__host__ __device__ constexpr int run_dy(int r) { return r < 9 ? r % 3 - 1 : my7(r - 9); }
__host__ __device__ constexpr int run_dz(int r) { return r < 9 ? r / 3 - 1 : mz7(r - 9); }

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
// The finite-difference current's B values of a pair (the curl's face
// neighbours), prefetched into L1 before the collision, so that their
// latency passes during the moments (256^3 FP16: 23.3 -> 24.1 GLUPS with
// the pre-pass).
template <class T>
__device__ __forceinline__ void prefetch_curl(const T* Bfd, long long n3, long long r0, long long ryp, long long rym,
                                              long long rzp, long long rzm, int gx0, int gxm0, int gxp1) {
  const T *Bx = Bfd, *By = Bfd + n3, *Bz = Bfd + 2 * n3;
  prefetch_l1(By + r0 + gx0);
  prefetch_l1(Bz + r0 + gx0);
  prefetch_l1(By + r0 + gxm0);
  prefetch_l1(By + r0 + gxp1);
  prefetch_l1(Bz + ryp + gx0);
  prefetch_l1(Bz + rym + gx0);
  prefetch_l1(By + rzp + gx0);
  prefetch_l1(By + rzm + gx0);
  prefetch_l1(Bx + rzp + gx0);
  prefetch_l1(Bx + rzm + gx0);
  prefetch_l1(Bx + ryp + gx0);
  prefetch_l1(Bx + rym + gx0);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned tries) {
  for (unsigned n = 0; n < tries; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 1-D bulk copy global -> shared, completing bytes on the mbarrier.
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Tensor-map copy of the box at (x, y, z, slot) of the state viewed as
// [48][nz][ny][nx], completing bytes on the mbarrier.
__device__ __forceinline__ void tensor_load(unsigned dst, const CUtensorMap* map, int y, int z, int slot, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(y), "r"(z), "r"(slot), "r"(bar)
      : "memory");
}

// ... and back: shared -> global, in the bulk async-group of the thread.
__device__ __forceinline__ void tensor_store(const CUtensorMap* map, int y, int z, int slot, unsigned src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(0), "r"(y), "r"(z), "r"(slot), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, unsigned src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the thread's committed stores have read their shared-memory source / are complete
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_done() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's shared-memory writes before later TMA reads of them
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// A row split into H segments (H = 2 for long rows: a tile is half a row,
// so a block needs half the threads and half the shared memory) stages each
// segment with kHalo values of its neighbours on each side, so that the odd
// step's x shift stays inside the staged copy; kHalo 16-bit values are one
// 16-byte unit, the granule of the bulk copies.
constexpr int kHalo = 8;

// Width of a staged row: the row itself, or a segment with its halos.
__host__ __device__ constexpr int staged_width(int nx, int H) { return H == 1 ? nx : nx / H + 2 * kHalo; }

// Values between the starts of two runs of three staged rows.  A tensor
// copy's shared-memory destination must be 128-byte aligned, so for rows
// staged by boxes the run is padded to a multiple of 64 16-bit values (no
// padding when nx is a multiple of 64); bulk-copied rows are dense.
__host__ __device__ constexpr int run_stride(int nx, int H) {
  return H == 1 && nx <= kBoxMaxX ? (3 * nx + 63) / 64 * 64 : 3 * staged_width(nx, H);
}

// The site pair (2t, 2t + 1) of a staged tile: ld(s, d) reads staged
// storage slot s at the pair moved by d sites (d = -c_x reads velocity c on
// an odd step; d = 0 on even steps), st(s, d, v) writes it there.  NX > 0
// fixes the row length at compile time (shared-memory offsets become
// immediates); NX = 0 reads it from the grid.  Whole rows (H = 1) wrap the
// shift around the row; a segment (H > 1) reads its halo.
template <class T, bool ODD, int NX, int H = 1>
struct PairAccess {
  const T* R;
  int nx, rs, x0, x1, xm0, xp1;  // nx: the staged row width; rs: the run stride
  __device__ __forceinline__ PairAccess(const T* rows, int n)
      : R(rows), nx(staged_width(NX ? NX : n, H)), rs(run_stride(NX ? NX : n, H)) {
    if constexpr (H == 1) {
      x0 = 2 * threadIdx.x;
      x1 = x0 + 1;
      xm0 = x0 == 0 ? nx - 1 : x0 - 1;
      xp1 = x1 == nx - 1 ? 0 : x1 + 1;
    } else {
      x0 = kHalo + 2 * threadIdx.x;
      x1 = x0 + 1;
      xm0 = x0 - 1;
      xp1 = x1 + 1;
    }
  }
  __device__ __forceinline__ f2 ld(int s, int d) const {
    const T* r = R + (s / 3) * rs + (s % 3) * nx;
    if (!ODD || d == 0) return Codec2<T>::dec(r + x0);
    if (d < 0) return pack(Codec<T>::dec(r[xm0]), Codec<T>::dec(r[x0]));
    return pack(Codec<T>::dec(r[x1]), Codec<T>::dec(r[xp1]));
  }
  __device__ __forceinline__ void st(int s, int d, f2 v) const {
    T* r = const_cast<T*>(R) + (s / 3) * rs + (s % 3) * nx;
    if (!ODD || d == 0) {
      Codec2<T>::enc(r + x0, v);
    } else if (d < 0) {
      r[xm0] = Codec<T>::enc(v.v.x);
      r[x0] = Codec<T>::enc(v.v.y);
    } else {
      r[x1] = Codec<T>::enc(v.v.x);
      r[xp1] = Codec<T>::enc(v.v.y);
    }
  }
};

// Base of every storage slot's rows (slot s starts at state + s N3), a
// kernel parameter, for the direct stores of long rows.
template <class T>
struct SlotBases {
  T* p[kPop];
};

// Results of a pair written straight to HBM (rows longer than 256 sites):
// storage slot s was staged from the row (y, z) + (run_dy(s / 3),
// run_dz(s / 3)) on odd steps and from (y, z) on even steps, and a result
// goes to the position of that row it was read from (as st() above does in
// the staged copy).  off[dz + 1][dy + 1]: the offset of the row (y + dy,
// z + dz) (periodic) plus the pair's first site x0, so that a store is one
// address computation on the slot's base; dm = xm0 - x0 and dp = xp1 - x1
// are the shifted sites' offsets (the wrap at the row's ends).
template <class T, bool ODD>
struct PairGlobal {
  const SlotBases<T>* base;
  int off[3][3];
  int dm, dp;
  __device__ __forceinline__ f2 ld(int s, int d) const {
    const int r = s / 3;
    const int dy = ODD ? run_dy(r) : 0, dz = ODD ? run_dz(r) : 0;
    const T* row = base->p[s] + off[dz + 1][dy + 1];
    if (!ODD || d == 0) return Codec2<T>::dec(row);
    if (d < 0) return pack(Codec<T>::dec(row[dm]), Codec<T>::dec(row[0]));
    return pack(Codec<T>::dec(row[1]), Codec<T>::dec(row[1 + dp]));
  }
  __device__ __forceinline__ void st(int s, int d, f2 v) const {
    const int r = s / 3;
    const int dy = ODD ? run_dy(r) : 0, dz = ODD ? run_dz(r) : 0;
    T* row = base->p[s] + off[dz + 1][dy + 1];
    if (!ODD || d == 0) {
      Codec2<T>::enc(row, v);
    } else if (d < 0) {
      row[dm] = Codec<T>::enc(v.v.x);
      row[0] = Codec<T>::enc(v.v.y);
    } else {
      row[1] = Codec<T>::enc(v.v.x);
      row[1 + dp] = Codec<T>::enc(v.v.y);
    }
  }
};

// Warp 0 moves the 48 rows of tile (y, z) between HBM and stage st: the rows
// (y, z) of all storage slots on even steps, run r of three storage slots
// from the row (y, z) + (run_dy(r), run_dz(r)) on odd steps.  The store
// writes each row back to where it was loaded from.  With H = 2 segments a
// tile is the segment h = tile % 2 of row tile / 2 (sites h W .. h W + W - 1,
// W = nx / 2), staged with bulk copies at offset kHalo of a row of
// staged_width(nx, 2) values: on odd steps with its halos, the one at the
// row's end (periodic) by a copy of its own; its results are stored directly.
template <class T, bool ODD, int H = 1>
struct RowIO {
  T* state;
  T* rows;  // [stage][16 runs, run_stride(nx, H) apart][3 storage slots][staged_width(nx, H)]
  unsigned long long* bars;
  long long n3;
  int nx, ny, nz, z0;  // tile t is the row (y, z) = (r % ny, r / ny + z0), r = t / H
  unsigned rowbytes;   // bytes of a whole row
  int lane;
  bool boxed, stall;
  const RowMaps* maps;
  int rs;  // run_stride(nx, H)

  __device__ __forceinline__ void issue(int tile, int st) const {
    if constexpr (H > 1) {
      issue_segment(tile, st);
      return;
    }
    const int y = tile % ny, z = tile / ny + z0;
    const unsigned bar = smem_addr(&bars[st]);
    T* dst = rows + (size_t)st * kRuns * rs;
    if (lane == 0) mbar_expect_tx(bar, kPop * rowbytes);
    __syncwarp();
    if (stall) return;
    if (boxed) {
      if (!ODD && rs == 3 * nx) {
        // dense runs: one box of all 48 storage slots
        if (lane == 0) tensor_load(smem_addr(dst), &maps->all, y, z, 0, bar);
      } else if (lane < kRuns) {
        const int ys = ODD ? wrap(y + run_dy(lane), ny) : y, zs = ODD ? wrap(z + run_dz(lane), nz) : z;
        tensor_load(smem_addr(dst + lane * rs), &maps->run, ys, zs, 3 * lane, bar);
      }
    } else {
      for (int s = lane; s < kPop; s += 32) {
        const int r = s / 3;
        const int ys = ODD ? wrap(y + run_dy(r), ny) : y, zs = ODD ? wrap(z + run_dz(r), nz) : z;
        bulk_load(smem_addr(dst + s * nx), state + (size_t)s * n3 + ((long long)zs * ny + ys) * nx, rowbytes, bar);
      }
    }
  }

  // Half-row segments (H = 2): every staged row of the segment, by bulk
  // copies of whole 16-byte units (W and kHalo are multiples of 8 values).
  __device__ __forceinline__ void issue_segment(int tile, int st) const {
    const int row = tile / H, h = tile % H;
    const int y = row % ny, z = row / ny + z0;
    const int W = nx / H, ws = staged_width(nx, H);
    const unsigned bar = smem_addr(&bars[st]);
    T* dst = rows + (size_t)st * kPop * ws;
    const unsigned seg = (unsigned)W * sizeof(T), halo = (unsigned)kHalo * sizeof(T);
    if (lane == 0) mbar_expect_tx(bar, kPop * (ODD ? seg + 2 * halo : seg));
    __syncwarp();
    if (stall) return;
    if (!ODD) {
      for (int s = lane; s < kPop; s += 32)
        bulk_load(smem_addr(dst + s * ws + kHalo),
                  state + (size_t)s * n3 + ((long long)z * ny + y) * nx + (long long)h * W, seg, bar);
    } else {
      // two copies per storage slot: the segment with the halo inside the
      // row, and the halo across the row's end (the first segment's left
      // halo is the row's last kHalo values, the last segment's right halo
      // its first ones)
      for (int j = lane; j < 2 * kPop; j += 32) {
        const int s = j >> 1, r = s / 3;
        const int ys = wrap(y + run_dy(r), ny), zs = wrap(z + run_dz(r), nz);
        const T* src = state + (size_t)s * n3 + ((long long)zs * ny + ys) * nx;
        T* d = dst + s * ws;
        if (h == 0) {
          if (j & 1) bulk_load(smem_addr(d), src + (nx - kHalo), halo, bar);
          else bulk_load(smem_addr(d + kHalo), src, seg + halo, bar);
        } else {
          if (j & 1) bulk_load(smem_addr(d + kHalo + W), src, halo, bar);
          else bulk_load(smem_addr(d), src + (W - kHalo), seg + halo, bar);
        }
      }
    }
  }

  // Returns once the stage has been read out as far as its refill needs
  // (DEFER: the refill waits for it itself, later).
  template <int STAGES, bool DEFER>
  __device__ __forceinline__ void store(int tile, int st) const {
    const int y = tile % ny, z = tile / ny + z0;
    const T* src = rows + (size_t)st * kRuns * rs;
    if (boxed) {
      if (!ODD && rs == 3 * nx) {
        if (lane == 0) tensor_store(&maps->all, y, z, 0, smem_addr(src));
      } else if (lane < kRuns) {
        const int ys = ODD ? wrap(y + run_dy(lane), ny) : y, zs = ODD ? wrap(z + run_dz(lane), nz) : z;
        tensor_store(&maps->run, ys, zs, 3 * lane, smem_addr(src + lane * rs));
      }
    } else {
      for (int s = lane; s < kPop; s += 32) {
        const int r = s / 3;
        const int ys = ODD ? wrap(y + run_dy(r), ny) : y, zs = ODD ? wrap(z + run_dz(r), nz) : z;
        bulk_store(state + (size_t)s * n3 + ((long long)zs * ny + ys) * nx, smem_addr(src + s * nx), rowbytes);
      }
    }
    bulk_commit();
    // Two stages: this stage is refilled next, so its rows must have been
    // read out.  Three: the stage refilled next held the previous tile,
    // whose store is the older of the two groups in flight.
    if constexpr (!DEFER) {
      if (STAGES == 2) bulk_wait_read();
      else asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    }
    __syncwarp();
  }
};

// Launch bounds per instantiation: 128 registers per thread (512 threads'
// worth per SM); a block has nx / (2 H) threads.
constexpr int row_bound_threads(int nx, int H = 1) { return nx ? nx / (2 * H) : kRowMaxThreads; }
constexpr int row_bound_blocks(int nx, int H = 1) { return 512 / row_bound_threads(nx, H); }

// Bfd: the pre-collision B - B_ref ([3][N3], storage type), read by kVarFdCurrent only.
// H: segments per row (1: a tile is a whole row; 2: half a row, rows of
// more than 256 sites only).
template <class T, bool ODD, int NX, int kRowStages, int VAR, int H = 1>
__global__ void __launch_bounds__(row_bound_threads(NX, H), row_bound_blocks(NX, H))
    step_row_kernel(T* __restrict__ state, Grid g, StepConsts k, unsigned* __restrict__ flag,
                    const T* __restrict__ Bfd, const __grid_constant__ RowMaps maps,
                    const __grid_constant__ SlotBases<T> bases, RowWait wt) {
  static_assert(H == 1 || (H == 2 && kRowStages == 2 && (NX == 0 || NX > 256)), "half rows: long rows, two stages");
  extern __shared__ __align__(128) unsigned char smem[];
  const int nx = NX ? NX : g.nx, ny = g.ny, nz = g.nz;
  const unsigned rowbytes = static_cast<unsigned>(nx) * sizeof(T);
  const unsigned stagebytes = static_cast<unsigned>(kRuns * run_stride(nx, H) * sizeof(T));
  T* rows = reinterpret_cast<T*>(smem);  // [stage][16 runs][3 storage slots][staged_width(nx, H)]
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + kRowStages * stagebytes);
  const int ntiles = ny * g.nzi * H;  // rows (or row segments) of the updated planes
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool boxed = nx <= kBoxMaxX;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRowStages; ++s) mbar_init(smem_addr(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const RowIO<T, ODD, H> io{state, rows, bars, g.n3, nx, ny, nz, g.z0, rowbytes, lane, boxed && H == 1,
                           wt.stall != 0, &maps, run_stride(nx, H)};

  const int first = blockIdx.x, stride = gridDim.x;
  // Tiles staged before the loop: both stages with two; with three, two of
  // them (the third is filled once the first tile's store has drained).
  constexpr int kAhead = kRowStages == 2 ? 2 : kRowStages - 1;
  // Rows of up to 256 sites with two stages (stages of up to 24.6 KB, four
  // or more blocks per SM) refill the stage of the previous tile from inside
  // the collision of the next one, so warp 0 no longer waits for that store
  // to drain at the end of a tile (128^3: 29.9 -> 31.2 GLUPS; 256^3, where
  // it also beats three stages of three blocks: 32.15 -> 32.9; at 512-site
  // rows, where a stage is 48 KB and the refill needs its lead time, it was
  // slower: 29.4 -> 28.4).
  constexpr bool kMidRefill = kRowStages == 2 && NX != 0 && NX <= 256 && H == 1;
  // Rows longer than 256 sites (two stages of up to 96 KB): the results go
  // straight from registers to HBM and the staged rows are only read, so a
  // stage is refilled as soon as its tile's collision ends, with no store to
  // drain first (512^3: 29.4 -> 30.2 GLUPS; 960- and 1024-site rows +7 % /
  // +4 %; at 256-site rows the extra address arithmetic made it slower).  No
  // location is read or written by more than one tile, so the order of these
  // stores and of other tiles' loads does not matter.
  constexpr bool kDirect = kRowStages == 2 && (NX == 512 || NX == 0 || H > 1);
  if (warp == 0)
    for (int s = 0; s < kAhead; ++s)
      if (first + s * stride < ntiles) io.issue(first + s * stride, s);

  int it = 0;
  for (int tile = first; tile < ntiles; tile += stride, ++it) {
    const int st = it % kRowStages;
    const bool ok = mbar_wait(smem_addr(&bars[st]), (it / kRowStages) & 1, wt.tries);
    if (ok) {
      // Collide in place.  The post-collision value of velocity c belongs in
      // the staged slot of the opposite velocity (on odd steps: the slot of
      // c itself, staged from the row (y, z) + (c_y, c_z)) at the position
      // this pair read that slot from, so each thread writes only what it
      // has read, and every staged row is the new content of the HBM row it
      // was loaded from.
      const PairAccess<T, ODD, NX, H> A(rows + (size_t)st * (stagebytes / sizeof(T)), nx);
      // the pair's sites in the row (global x), for the direct stores and the
      // B field: the staged positions for whole rows, shifted by the
      // segment's first site for half rows
      int gx0 = A.x0, gx1 = A.x1, gxm0 = A.xm0, gxp1 = A.xp1;
      if constexpr (H > 1) {
        gx0 = (tile % H) * (nx / H) + 2 * (int)threadIdx.x;
        gx1 = gx0 + 1;
        gxm0 = gx0 == 0 ? nx - 1 : gx0 - 1;
        gxp1 = gx1 == nx - 1 ? 0 : gx1 + 1;
      }
      auto ldf = [&](int px, int py, int pz) {
        const int q = px + 3 * py + 9 * pz;
        return A.ld(ODD ? 26 - q : q, 1 - px);
      };
      auto ldg = [&](int c, int i) { return A.ld(kQ + 3 * (ODD ? opp7(i) : i) + c, -mx7(i)); };
      PairGlobal<T, ODD> G;
      if constexpr (kDirect) {
        const int y = (tile / H) % ny, z = (tile / H) / ny + g.z0;
        G.base = &bases;
        G.dm = gxm0 - gx0;
        G.dp = gxp1 - gx1;
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
            G.off[dz][dy] = (ODD || (dz == 1 && dy == 1))
                                ? (wrap(z + dz - 1, nz) * ny + wrap(y + dy - 1, ny)) * nx + gx0
                                : 0;
      }
      auto stf = [&](int px, int py, int pz, f2 v) {
        const int q = px + 3 * py + 9 * pz;
        if constexpr (kDirect) G.st(ODD ? q : 26 - q, px - 1, v);
        else A.st(ODD ? q : 26 - q, px - 1, v);
      };
      auto stg = [&](int c, int i, f2 v) {
        if constexpr (kDirect) G.st(kQ + 3 * (ODD ? i : opp7(i)) + c, mx7(i), v);
        else A.st(kQ + 3 * (ODD ? i : opp7(i)) + c, mx7(i), v);
      };
      // J = periodic central-difference curl of the pre-collision field at
      // the pair (the face neighbours in y and z are whole-pair loads).
      auto curl_b = [&](f2 (&J)[3]) {
        const int y = (tile / H) % ny, z = (tile / H) / ny + g.z0;
        const long long r0 = ((long long)z * ny + y) * nx;
        const long long ryp = ((long long)z * ny + wrap(y + 1, ny)) * nx;
        const long long rym = ((long long)z * ny + wrap(y - 1, ny)) * nx;
        const long long rzp = ((long long)wrap(z + 1, nz) * ny + y) * nx;
        const long long rzm = ((long long)wrap(z - 1, nz) * ny + y) * nx;
        const T *Bx = Bfd, *By = Bfd + g.n3, *Bz = Bfd + 2 * g.n3;
        // the pair (x0, x1) of a row as one 32-bit load, a single value as one 16-bit load
        auto at = [&](const T* b, long long r) { return f2{dec2(b + r + gx0)}; };
        auto one = [&](const T* b, long long i) { return Codec<T>::dec(b[i]); };
        const f2 by0 = at(By, r0), bz0 = at(Bz, r0);
        // B(x + 1) - B(x - 1) at x = x0, x1
        const f2 dxBy = pack(by0.v.y, one(By, r0 + gxp1)) - pack(one(By, r0 + gxm0), by0.v.x);
        const f2 dxBz = pack(bz0.v.y, one(Bz, r0 + gxp1)) - pack(one(Bz, r0 + gxm0), bz0.v.x);
        J[0] = 0.5f * ((at(Bz, ryp) - at(Bz, rym)) - (at(By, rzp) - at(By, rzm)));
        J[1] = 0.5f * ((at(Bx, rzp) - at(Bx, rzm)) - dxBz);
        J[2] = 0.5f * (dxBy - (at(Bx, ryp) - at(Bx, rym)));
      };
      auto mid = [&]() {
        if constexpr (kMidRefill) {
          if (warp == 0 && it > 0) {
            bulk_wait_read();  // the previous tile's store has read its stage
            __syncwarp();
            if (tile + stride < ntiles) io.issue(tile + stride, (it + 1) % 2);
          }
        }
      };
      if constexpr (VAR == kVarFdCurrent) {
        const int y = (tile / H) % ny, z = (tile / H) / ny + g.z0;
        prefetch_curl(Bfd, g.n3, ((long long)z * ny + y) * nx, ((long long)z * ny + wrap(y + 1, ny)) * nx,
                      ((long long)z * ny + wrap(y - 1, ny)) * nx, ((long long)wrap(z + 1, nz) * ny + y) * nx,
                      ((long long)wrap(z - 1, nz) * ny + y) * nx, gx0, gxm0, gxp1);
      }
      collide_pair<VAR>(ldf, ldg, stf, stg, curl_b, mid, k, flag);
      fence_proxy_async();
    }
    // Every thread is done with this stage before it is refilled.
    if (__syncthreads_or(!ok)) {
      // A copy did not complete in time: report it, let the copies still in
      // flight into or out of this block's shared memory finish (bounded),
      // and stop.
      if (threadIdx.x == 0) atomicOr(flag, 2u);
      if (warp == 0) bulk_wait_done();
      for (int j = it; j < it + kAhead + (kMidRefill ? 1 : 0); ++j)
        if (first + j * stride < ntiles)
          (void)mbar_wait(smem_addr(&bars[j % kRowStages]), (j / kRowStages) & 1, wt.tries);
      return;
    }
    if (warp == 0 && kDirect) {
      // the stage was only read: refill it with the tile two ahead
      if (tile + 2 * stride < ntiles) io.issue(tile + 2 * stride, st);
    } else if (warp == 0) {
      io.template store<kRowStages, kMidRefill>(tile, st);
      if constexpr (kMidRefill) {
        // refilled from inside the next tile's collision
      } else if constexpr (kRowStages == 2) {
        if (tile + 2 * stride < ntiles) io.issue(tile + 2 * stride, st);
      } else {
        const int next = tile + (kRowStages - 1) * stride;
        if (next < ntiles) io.issue(next, (it + kRowStages - 1) % kRowStages);
      }
    }
  }
  if (warp == 0) bulk_wait_done();
}

// The pair kernel: the row kernel's packed collision of the site pair
// (x0, x0 + 1) with its populations loaded from and stored to HBM directly,
// no staging -- any even row length.  Under the AA pattern a pair writes
// exactly the places it read (PairGlobal), and the collision reads all of
// its inputs before it writes (as in the staged rows, which it updates in
// place), so pairs need no synchronisation.  One pair per thread.
constexpr int kPairThreads = 128;
template <class T, bool ODD, int VAR>
__global__ void __launch_bounds__(kPairThreads, 4)
    step_pair_kernel(Grid g, StepConsts k, unsigned* __restrict__ flag, const T* __restrict__ Bfd,
                     const __grid_constant__ SlotBases<T> bases) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, pairs = nx / 2;
  const long long p = (long long)blockIdx.x * kPairThreads + threadIdx.x;
  if (p >= (long long)pairs * ny * g.nzi) return;
  const int xp = (int)(p % pairs);
  const long long rowi = p / pairs;
  const int y = (int)(rowi % ny), z = (int)(rowi / ny) + g.z0;
  const int gx0 = 2 * xp, gx1 = gx0 + 1;
  const int gxm0 = gx0 == 0 ? nx - 1 : gx0 - 1, gxp1 = gx1 == nx - 1 ? 0 : gx1 + 1;
  PairGlobal<T, ODD> G;
  G.base = &bases;
  G.dm = gxm0 - gx0;
  G.dp = gxp1 - gx1;
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
      G.off[dz][dy] =
          (ODD || (dz == 1 && dy == 1)) ? (wrap(z + dz - 1, nz) * ny + wrap(y + dy - 1, ny)) * nx + gx0 : 0;
  auto ldf = [&](int px, int py, int pz) {
    const int q = px + 3 * py + 9 * pz;
    return G.ld(ODD ? 26 - q : q, 1 - px);
  };
  auto ldg = [&](int c, int i) { return G.ld(kQ + 3 * (ODD ? opp7(i) : i) + c, -mx7(i)); };
  auto stf = [&](int px, int py, int pz, f2 v) {
    const int q = px + 3 * py + 9 * pz;
    G.st(ODD ? q : 26 - q, px - 1, v);
  };
  auto stg = [&](int c, int i, f2 v) { G.st(kQ + 3 * (ODD ? i : opp7(i)) + c, mx7(i), v); };
  auto curl_b = [&](f2 (&J)[3]) {
    const long long r0 = ((long long)z * ny + y) * nx;
    const long long ryp = ((long long)z * ny + wrap(y + 1, ny)) * nx;
    const long long rym = ((long long)z * ny + wrap(y - 1, ny)) * nx;
    const long long rzp = ((long long)wrap(z + 1, nz) * ny + y) * nx;
    const long long rzm = ((long long)wrap(z - 1, nz) * ny + y) * nx;
    const T *Bx = Bfd, *By = Bfd + g.n3, *Bz = Bfd + 2 * g.n3;
    auto at = [&](const T* b, long long r) { return f2{dec2(b + r + gx0)}; };
    auto one = [&](const T* b, long long i) { return Codec<T>::dec(b[i]); };
    const f2 by0 = at(By, r0), bz0 = at(Bz, r0);
    const f2 dxBy = pack(by0.v.y, one(By, r0 + gxp1)) - pack(one(By, r0 + gxm0), by0.v.x);
    const f2 dxBz = pack(bz0.v.y, one(Bz, r0 + gxp1)) - pack(one(Bz, r0 + gxm0), bz0.v.x);
    J[0] = 0.5f * ((at(Bz, ryp) - at(Bz, rym)) - (at(By, rzp) - at(By, rzm)));
    J[1] = 0.5f * ((at(Bx, rzp) - at(Bx, rzm)) - dxBz);
    J[2] = 0.5f * (dxBy - (at(Bx, ryp) - at(Bx, rym)));
  };
  auto mid = [] {};
  if constexpr (VAR == kVarFdCurrent)
    prefetch_curl(Bfd, g.n3, ((long long)z * ny + y) * nx, ((long long)z * ny + wrap(y + 1, ny)) * nx,
                  ((long long)z * ny + wrap(y - 1, ny)) * nx, ((long long)wrap(z + 1, nz) * ny + y) * nx,
                  ((long long)wrap(z - 1, nz) * ny + y) * nx, gx0, gxm0, gxp1);
  collide_pair<VAR>(ldf, ldg, stf, stg, curl_b, mid, k, flag);
}

template <class T, bool ODD, int VAR>
cudaError_t pair_launch(const RowCall& c) {
  if (c.g.nx % 2 != 0) return cudaErrorInvalidValue;
  if (!c.launch) return cudaSuccess;
  const long long npairs = (long long)(c.g.nx / 2) * c.g.ny * c.g.nzi;
  const long long blocks = (npairs + kPairThreads - 1) / kPairThreads;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  SlotBases<T> bases;
  for (int sl = 0; sl < kPop; ++sl) bases.p[sl] = static_cast<T*>(c.pop) + (size_t)sl * (size_t)c.g.n3;
  step_pair_kernel<T, ODD, VAR><<<(unsigned)blocks, kPairThreads, 0, c.s>>>(c.g, c.k, c.flag,
                                                                         static_cast<const T*>(c.Bfd), bases);
  return cudaGetLastError();
}

size_t row_smem_bytes(int nx, size_t elem, int stages, int H = 1) {
  return stages * (kRuns * (size_t)run_stride(nx, H) * elem + sizeof(unsigned long long));
}

// Stages per row length, from timings at 128^3, 256^3 and 512^3 (FP16).
// Two stages, with the refill issued inside the next tile's collision (up
// to 256 sites) or with direct stores (longer rows): four blocks per SM at
// 256-site rows (32.9 GLUPS against 32.15 for three stages of three
// blocks, where the store of a tile drains while the next one computes),
// and one block instead of two at 512-site rows with three (17.5 against
// 30.1).  The general instantiation: three stages with TMA stores from 129
// to 199 sites, two with direct stores from 200 (~4M-site lattices, GLUPS
// three / two stages: 136 21.2 / 20.7, 160 25.2 / 24.2, 200 23.9 / 26.5,
// 224 26.5 / 28.8, 248 28.8 / 28.6; 192: 29.4 with three).
constexpr int row_stages(int nx) { return nx > 128 && nx < 200 ? 3 : 2; }

// Launch configuration of one instantiation, cached per device (the
// shared-memory opt-in and the resident blocks per SM depend on the device
// and on nx only); a mutex makes concurrent host threads safe.
constexpr int kMaxDevices = 64;

template <class T, bool ODD, int NX, int S, int VAR, int H>
cudaError_t row_config(const Grid& g, int* grid, size_t* smem_out) {
  auto kern = step_row_kernel<T, ODD, NX, S, VAR, H>;
  const int threads = g.nx / (2 * H);
  const size_t smem = row_smem_bytes(g.nx, sizeof(T), S, H);
  struct Cache {
    size_t attr_smem, occ_smem;
    int occ, nsm;
  };
  static Cache cache[kMaxDevices];
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  Cache& c = cache[dev];
  if (smem > c.attr_smem) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    c.attr_smem = smem;
  }
  if (smem != c.occ_smem) {
    int per = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    c.occ = per;
    c.occ_smem = smem;
  }
  if (c.nsm == 0 && (e = cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long long ntiles = (long long)g.ny * g.nzi * H, slots = (long long)c.occ * c.nsm;
  *grid = (int)(ntiles < slots ? ntiles : slots);
  *smem_out = smem;
  return cudaSuccess;
}

template <class T, bool ODD, int NX, int S, int VAR, int H = 1>
cudaError_t row_launch(const RowCall& c) {
  int grid = 0;
  size_t smem = 0;
  cudaError_t e = row_config<T, ODD, NX, S, VAR, H>(c.g, &grid, &smem);
  RowMaps maps{};
  if (e == cudaSuccess && H == 1 && c.g.nx <= kBoxMaxX) e = row_maps(c.pop, c.g, &maps);
  if (e != cudaSuccess || !c.launch) return e;
  SlotBases<T> bases;
  for (int sl = 0; sl < kPop; ++sl) bases.p[sl] = static_cast<T*>(c.pop) + (size_t)sl * (size_t)c.g.n3;
  step_row_kernel<T, ODD, NX, S, VAR, H>
      <<<grid, c.g.nx / (2 * H), smem, c.s>>>(static_cast<T*>(c.pop), c.g, c.k, c.flag,
                                              static_cast<const T*>(c.Bfd), maps, bases, c.wt);
  return cudaGetLastError();
}

template <class T, bool ODD, int VAR>
cudaError_t row_nx(const RowCall& c) {
  if (c.segments == 0) return pair_launch<T, ODD, VAR>(c);
  // the alignment the staging copies need (see the requirements above)
  if (c.g.nx % 8 != 0) return cudaErrorInvalidValue;
  if (c.segments == 2) {
    if (c.g.nx <= kBoxMaxX || c.g.nx % 16 != 0) return cudaErrorInvalidValue;
    return c.g.nx == 512 ? row_launch<T, ODD, 512, 2, VAR, 2>(c) : row_launch<T, ODD, 0, 2, VAR, 2>(c);
  }
  switch (c.g.nx) {
    case 64: return row_launch<T, ODD, 64, row_stages(64), VAR>(c);
    case 128: return row_launch<T, ODD, 128, row_stages(128), VAR>(c);
    case 256: return row_launch<T, ODD, 256, row_stages(256), VAR>(c);
    case 512: return row_launch<T, ODD, 512, row_stages(512), VAR>(c);
    default:
      return row_stages(c.g.nx) == 3 ? row_launch<T, ODD, 0, 3, VAR>(c) : row_launch<T, ODD, 0, 2, VAR>(c);
  }
}

template <int VAR>
cudaError_t row_call(const RowCall& c) {
  if (VAR == kVarFdCurrent && !c.Bfd) return cudaErrorInvalidValue;
  switch (c.storage) {
    case 2: return c.odd ? row_nx<__half, true, VAR>(c) : row_nx<__half, false, VAR>(c);
    case 3: return c.odd ? row_nx<__nv_bfloat16, true, VAR>(c) : row_nx<__nv_bfloat16, false, VAR>(c);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace flame
