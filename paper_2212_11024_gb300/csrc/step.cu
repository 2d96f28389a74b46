// step.cu -- the fused FLAME collide-and-stream step, one thread per site,
// AA in-place streaming over the 48-slot population state: the kernel for
// FP32 storage, and for 16-bit storage where the row kernel of step_row.cuh
// (the same algebra and variants, two sites per thread) does not apply.
// launch_step chooses between the two; the finite-difference current's B
// pre-pass (bfield_kernel) serves both.
//
// Algebra of the fluid collision.  With S = diag[1,1,1,1,w,w,w,w,w,1,...,1]
// (eq. collision_matrix) every central moment except the five deviatoric
// second-order ones is set to its equilibrium value, so
//     f* = f^mhd(0) + (1 - w) P(f - f^mhd(0)),
// where P(D) is the population whose central moments are zero except the
// second-order ones, which equal dev(Pi_neq) with Pi_neq the raw second
// moment of f - f^mhd(0) (equal to its central moment since that difference
// carries no mass or momentum).  Any basis with the span of the corrected
// T of Sec. 3.1.2 gives this result.  In 1-D, the population with central
// moments (m0, m1, m2) at velocity shift u is
//     f_0 = m0 (1 - u^2) - 2 u m1 - m2,   f_+-1 = (m0 (u^2 +- u) + m1 (2u +- 1) + m2) / 2,
// and the 3-D map is the tensor product over the axes; the 6th-order Hermite
// equilibrium of App. A factors the same way (psi(0,u) = 2/3 - u^2,
// psi(+-1,u) = (1/3 + u^2 +- u)/2).  Everything is evaluated divided by the
// lattice weights w_i = w1(cx) w1(cy) w1(cz), w1 = (2/3, 1/6), and as a
// deviation from the rest equilibrium of (rho0, B_ref), so FP32 keeps the
// relative precision of the dynamic part.
//
// Collision step per site (Sec. 3): a1 load + decode, a2 rho and U
// (eq. LB_moments2), a3 B and Lambda (eqs. mag_field_LB, LB_density_current),
// a4 J from the Hall system (eq. soe_current_density, closed form of its
// 3x3 solve), a5 central-moment fluid collision (eq. cm_collision_step),
// a6 g^Hall(0) (eq. gHall_eq) and BGK (eq. MHD_LBscheme), a7 encode and
// store (eq. stream, AA pattern).
#include "aa.cuh"

namespace flame {
namespace {

// Step launch: 256 threads per block (a whole 256-site x row at 256^3) and
// at most 80 registers per thread (3 resident blocks per SM); the block
// shape and register budget were chosen by timing at 256^3.  Where nx is
// not a multiple of 32 a block of x rows leaves lanes idle (33 sites: 64
// threads); where that is 10 % or more of them the blocks cover consecutive
// sites instead (flat; a separate instantiation, so the row blocks keep
// their registers).  GLUPS on ~8M-site lattices, FP32 / FP16 row blocks ->
// flat: 33 12.2 -> 15.6 / 13.5 -> 22.4, 65 14.1 -> 15.4 / 16.8 -> 22.4, 100
// 14.8 -> 15.6 / 20.1 -> 22.6; flat runs at ~15.7 FP32 at any length, row
// blocks with little waste stay ahead (250: 16.3, 255: 16.4, 256: 17.3).
constexpr int kStepThreads = 256;
constexpr int kStepMinBlocks = 3;

// VAR selects the scheme: kVarFlame (the paper's), kVarBgkFluid, kVarEmhd or
// kVarFdCurrent (flame_internal.h); Bfd is the pre-collision B - B_ref field
// (storage type) written by the B pre-pass, read only by kVarFdCurrent.
template <class T, bool ODD, int VAR, bool FLAT = false>
__global__ void __launch_bounds__(kStepThreads, kStepMinBlocks)
    step_kernel(Slots<T> P, Grid g, StepConsts k, unsigned* __restrict__ flag, const T* __restrict__ Bfd) {
  int x, y, z;
  if constexpr (FLAT) {
    // consecutive sites of the updated planes (N3 < 2^31)
    const int p = blockIdx.x * kStepThreads + threadIdx.x;
    if (p >= (int)g.n3i) return;
    const int r = p / g.nx;
    x = p - r * g.nx;
    const int zz = r / g.ny;
    y = r - zz * g.ny;
    z = zz + g.z0;
  } else {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = blockIdx.z + g.z0;
    if (x >= g.nx || y >= g.ny) return;
  }
  const int site = (z * g.ny + y) * g.nx + x;
  const Nbr nb = make_nbr(x, y, z, g);

  // a1: load and decode the 48 pre-collision populations.  Fluid values are
  // kept in velocity-cube order s[px + 3 py + 9 pz], p = c + 1.
  float s[kQ];
#pragma unroll
  for (int pz = 0; pz < 3; ++pz)
#pragma unroll
    for (int py = 0; py < 3; ++py)
#pragma unroll
      for (int px = 0; px < 3; ++px) {
        const int i = idx27(px, py, pz);
        const int slot = ODD ? opp27(i) : i;
        s[px + 3 * py + 9 * pz] = Codec<T>::dec(P.p[slot][site + src_off<ODD>(nb, px - 1, py - 1, pz - 1)]);
      }
  float sg[3][kM];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int i = 0; i < kM; ++i) {
      const int slot = mslot(b, ODD ? opp7(i) : i);
      sg[b][i] = Codec<T>::dec(P.p[slot][site + src_off<ODD>(nb, mx7(i), my7(i), mz7(i))]);
    }

  // a2: rho, momentum and raw second moment (deviations from rest) by three
  // 1-D passes over the velocity cube with the 1-D weights (1, 4, 1) / 6.
  float m0[9], m1[9], m2[9];  // x pass: [py + 3 pz]
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const float sm = s[3 * q], s0 = s[3 * q + 1], sp = s[3 * q + 2];
    const float t = sp + sm;
    m0[q] = fmaf(4.f, s0, t);
    m1[q] = sp - sm;
    m2[q] = t;
  }
  float M00[3], M10[3], M20[3], M01[3], M11[3], M02[3];  // y pass: [pz]
#pragma unroll
  for (int pz = 0; pz < 3; ++pz) {
    const int q = 3 * pz;
    const float t0 = m0[q + 2] + m0[q];
    M00[pz] = fmaf(4.f, m0[q + 1], t0);
    M02[pz] = t0;
    M01[pz] = m0[q + 2] - m0[q];
    M10[pz] = fmaf(4.f, m1[q + 1], m1[q + 2] + m1[q]);
    M11[pz] = m1[q + 2] - m1[q];
    M20[pz] = fmaf(4.f, m2[q + 1], m2[q + 2] + m2[q]);
  }
  // The density deviation is divided exactly (correct rounding keeps mass
  // unbiased); momentum and stress use the reciprocal of 216 rho / of 216,
  // whose rounding is not one-signed across sites (U) or only rescales the
  // non-conserved stress by 1 + O(1e-8) (Pi).
  const float t00 = M00[2] + M00[0];
  const float drho = fmaf(4.f, M00[1], t00) / 216.f;
  const float rho = k.rho0 + drho;
  const float irho216 = 1.f / (216.f * rho);
  const float U[3] = {fmaf(4.f, M10[1], M10[2] + M10[0]) * irho216, fmaf(4.f, M01[1], M01[2] + M01[0]) * irho216,
                      (M00[2] - M00[0]) * irho216};
  constexpr float k216 = 1.f / 216.f;
  const float pxx = fmaf(4.f, M20[1], M20[2] + M20[0]) * k216;
  const float pyy = fmaf(4.f, M02[1], M02[2] + M02[0]) * k216;
  const float pzz = t00 * k216;
  const float pxy = fmaf(4.f, M11[1], M11[2] + M11[0]) * k216;
  const float pxz = (M10[2] - M10[0]) * k216;
  const float pyz = (M01[2] - M01[0]) * k216;

  // a3: B = sum_i g_i and Lambda_ab = sum_i xi_ia g_ib.
  float dB[3], lam[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    dB[b] = 0.25f * sg[b][0] + 0.125f * ((sg[b][1] + sg[b][2]) + (sg[b][3] + sg[b][4]) + (sg[b][5] + sg[b][6]));
    lam[0][b] = 0.125f * (sg[b][1] - sg[b][2]);
    lam[1][b] = 0.125f * (sg[b][3] - sg[b][4]);
    lam[2][b] = 0.125f * (sg[b][5] - sg[b][6]);
  }
  const float B[3] = {k.Bref[0] + dB[0], k.Bref[1] + dB[1], k.Bref[2] + dB[2]};

  // Non-finite guard: one relaxed flag read, and an atomic only while the
  // flag is still clear, so a blown-up field does not serialise on it.
  if (!isfinite(drho + U[0] + U[1] + U[2] + dB[0] + dB[1] + dB[2])) {
    if (*((volatile unsigned*)flag) == 0u) atomicOr(flag, 1u);
  }

  // a4: J + s J x B = y, y = -(omega_B/C^2)(A - 2 U x B), s = 2 alpha_H omega_B / C^2.
  // (Electron MHD: U is neglected against alpha_H J, here and in g^Hall(0).)
  float V[3];
  if constexpr (VAR == kVarFdCurrent) {
    // J = periodic central-difference curl of the pre-collision field
    const long long n3 = g.n3;
    auto Bn = [&](int b, int off) { return Codec<T>::dec(Bfd[b * n3 + site + off]); };
    const float J[3] = {0.5f * ((Bn(2, nb.yp) - Bn(2, nb.ym)) - (Bn(1, nb.zp) - Bn(1, nb.zm))),
                        0.5f * ((Bn(0, nb.zp) - Bn(0, nb.zm)) - (Bn(2, nb.xp) - Bn(2, nb.xm))),
                        0.5f * ((Bn(1, nb.xp) - Bn(1, nb.xm)) - (Bn(0, nb.yp) - Bn(0, nb.ym)))};
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a] = U[a] - k.alphaH * J[a];
  } else {
    const float Ue[3] = {VAR == kVarEmhd ? 0.f : U[0], VAR == kVarEmhd ? 0.f : U[1], VAR == kVarEmhd ? 0.f : U[2]};
    const float gq = 4.f * k.omegaB;
    const float A[3] = {lam[1][2] - lam[2][1], lam[2][0] - lam[0][2], lam[0][1] - lam[1][0]};
    const float uxb[3] = {Ue[1] * B[2] - Ue[2] * B[1], Ue[2] * B[0] - Ue[0] * B[2], Ue[0] * B[1] - Ue[1] * B[0]};
    const float yv[3] = {-gq * (A[0] - 2.f * uxb[0]), -gq * (A[1] - 2.f * uxb[1]), -gq * (A[2] - 2.f * uxb[2])};
    const float sH = 2.f * k.alphaH * gq;
    const float yxb[3] = {yv[1] * B[2] - yv[2] * B[1], yv[2] * B[0] - yv[0] * B[2], yv[0] * B[1] - yv[1] * B[0]};
    const float yb = yv[0] * B[0] + yv[1] * B[1] + yv[2] * B[2];
    const float b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const float iden = 1.f / (1.f + sH * sH * b2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float J = (yv[a] - sH * yxb[a] + sH * sH * yb * B[a]) * iden;
      V[a] = Ue[a] - k.alphaH * J;
    }
  }

  // a6: magnetic BGK towards g^Hall(0); deviations: rest dB_b, face
  // (axis a, sign +-) dB_b +- Lambda0_ab / C^2, Lambda0_ab = V_a B_b - B_a V_b.
  {
    const float om = k.omegaB, cm = 1.f - k.omegaB;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      P.p[mslot(b, ODD ? 0 : opp7(0))][site] = Codec<T>::enc(cm * sg[b][0] + om * dB[b]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float l0 = (a == b) ? 0.f : 4.f * (V[a] * B[b] - B[a] * V[b]);
#pragma unroll
        for (int h = 1; h <= 2; ++h) {
          const int i = 2 * a + h;
          const float v = cm * sg[b][i] + om * (h == 1 ? dB[b] + l0 : dB[b] - l0);
          P.p[mslot(b, ODD ? i : opp7(i))][site + dst_off<ODD>(nb, mx7(i), my7(i), mz7(i))] = Codec<T>::enc(v);
        }
      }
    }
  }

  // a5: fluid.  Dynamic part of the Maxwell stress M(B) - M(B_ref) =
  // miso I - N, N = Bref b + b Bref + b b, miso = Bref.b + |b|^2/2.
  const float bx = dB[0], by = dB[1], bz = dB[2];
  const float Br[3] = {k.Bref[0], k.Bref[1], k.Bref[2]};
  const float Nxx = 2.f * Br[0] * bx + bx * bx, Nyy = 2.f * Br[1] * by + by * by, Nzz = 2.f * Br[2] * bz + bz * bz;
  const float Nxy = Br[0] * by + bx * Br[1] + bx * by;
  const float Nxz = Br[0] * bz + bx * Br[2] + bx * bz;
  const float Nyz = Br[1] * bz + by * Br[2] + by * bz;
  const float miso = Br[0] * bx + Br[1] * by + Br[2] * bz + 0.5f * (bx * bx + by * by + bz * bz);
  // (1 - w) dev(Pi - rho U U - M): the non-equilibrium deviatoric stress.
  const float Sxx = pxx - rho * U[0] * U[0] + Nxx, Syy = pyy - rho * U[1] * U[1] + Nyy,
              Szz = pzz - rho * U[2] * U[2] + Nzz;
  const float r = 1.f - k.omega;
  const float tr3 = (Sxx + Syy + Szz) / 3.f;
  const float Dxx = r * (Sxx - tr3), Dyy = r * (Syy - tr3), Dzz = r * (Szz - tr3);
  const float Dxy = r * (pxy - rho * U[0] * U[1] + Nxy);
  const float Dxz = r * (pxz - rho * U[0] * U[2] + Nxz);
  const float Dyz = r * (pyz - rho * U[1] * U[2] + Nyz);

  // 1-D factors of the x and y axes, divided by the 1-D weight: e = psi/w1 - 1
  // and p0, p1 (p2 is constant), the inverse-moment maps of m0, m1, m2.
  float ex[3], ey[3], p0x[3], p0y[3], p1x[3], p1y[3];
  {
    const float u = U[0], uu = u * u;
    ex[0] = 3.f * uu - 3.f * u, ex[1] = -1.5f * uu, ex[2] = 3.f * uu + 3.f * u;
    p0x[0] = 3.f * (uu - u), p0x[1] = 1.5f * (1.f - uu), p0x[2] = 3.f * (uu + u);
    p1x[0] = 6.f * u - 3.f, p1x[1] = -3.f * u, p1x[2] = 6.f * u + 3.f;
  }
  {
    const float u = U[1], uu = u * u;
    ey[0] = 3.f * uu - 3.f * u, ey[1] = -1.5f * uu, ey[2] = 3.f * uu + 3.f * u;
    p0y[0] = 3.f * (uu - u), p0y[1] = 1.5f * (1.f - uu), p0y[2] = 3.f * (uu + u);
    p1y[0] = 6.f * u - 3.f, p1y[1] = -3.f * u, p1y[2] = 6.f * u + 3.f;
  }
  constexpr float p2[3] = {3.f, -1.5f, 3.f};
  // Along z every term is a quadratic in cz: ez(c) = e0z + e1z c + e2z c^2,
  // p0z(c) = q00 + q10 c + q20 c^2, p1z(c) = q01 + 3 c + q21 c^2,
  // p2z(c) = -1.5 + 4.5 c^2.
  const float uz = U[2], uzz = uz * uz;
  const float e0z = -1.5f * uzz, e1z = 3.f * uz, e2z = 4.5f * uzz;
  const float q00 = 1.5f * (1.f - uzz), q10 = 3.f * uz, q20 = fmaf(4.5f, uzz, -1.5f);
  const float q01 = -3.f * uz, q21 = 9.f * uz;
  // Lorentz term 4.5 (miso (|c|^2 - 1) - c.N.c) + 1.5 tr(N), split as
  // Lxy + Lz1 cz + Lz2 cz^2.
  const float Lbase = 1.5f * (Nxx + Nyy + Nzz) - 4.5f * miso;
  const float LA = 4.5f * (miso - Nxx), LB = 4.5f * (miso - Nyy), LC = 9.f * Nxy;
  const float NX = -9.f * Nxz, NY = -9.f * Nyz, LZ = 4.5f * (miso - Nzz);

  // a7: for each (cx, cy), f*/w - (rest reference) = Z0 + Z1 cz + Z2 cz^2.
#pragma unroll
  for (int py = 0; py < 3; ++py)
#pragma unroll
    for (int px = 0; px < 3; ++px) {
      const int cx = px - 1, cy = py - 1;
      const float exy = ex[px] + ey[py] + ex[px] * ey[py];
      const float g = fmaf(rho, exy, rho);
      // BGK fluid collision: no projected non-equilibrium part; the result is
      // blended with the pre-collision populations below.
      const float A0 = VAR == kVarBgkFluid ? 0.f
                                           : (Dxx * p2[px]) * p0y[py] + (Dyy * p2[py]) * p0x[px] + (Dxy * p1x[px]) * p1y[py];
      const float A1 = VAR == kVarBgkFluid ? 0.f : (Dxz * p1x[px]) * p0y[py] + (Dyz * p1y[py]) * p0x[px];
      const float A2 = VAR == kVarBgkFluid ? 0.f : (Dzz * p0x[px]) * p0y[py];
      float Lxy = Lbase;
      if (cx != 0) Lxy += LA;
      if (cy != 0) Lxy += LB;
      if (cx * cy != 0) Lxy += (cx * cy > 0) ? -LC : LC;
      float Lz1 = 0.f;
      if (cx != 0) Lz1 += (cx > 0) ? NX : -NX;
      if (cy != 0) Lz1 += (cy > 0) ? NY : -NY;
      const float Z0 = fmaf(rho, exy, drho) + g * e0z + A0 * q00 + A1 * q01 - 1.5f * A2 + Lxy;
      const float Z1 = g * e1z + A0 * q10 + 3.f * A1 + Lz1;
      const float Z2 = g * e2z + A0 * q20 + A1 * q21 + 4.5f * A2 + LZ;
      const float tz = Z0 + Z2;
      float vz[3] = {tz - Z1, Z0, tz + Z1};
      if constexpr (VAR == kVarBgkFluid) {
#pragma unroll
        for (int pz = 0; pz < 3; ++pz) vz[pz] = (1.f - k.omega) * s[px + 3 * py + 9 * pz] + k.omega * vz[pz];
      }
#pragma unroll
      for (int pz = 0; pz < 3; ++pz) {
        const int i = idx27(px, py, pz);
        const int slot = ODD ? i : opp27(i);
        P.p[slot][site + dst_off<ODD>(nb, cx, cy, pz - 1)] = Codec<T>::enc(vz[pz]);
      }
    }
}


// B - B_ref of the pre-collision populations at every site, in the storage's
// element type, for the finite-difference current variant.
template <class T, bool ODD>
__global__ void bfield_kernel(Slots<T> P, Grid g, T* __restrict__ Bfd) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  if (x >= g.nx || y >= g.ny) return;
  const int site = (z * g.ny + y) * g.nx + x;
  const Nbr nb = make_nbr(x, y, z, g);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < kM; ++i)
      v += (i == 0 ? 0.25f : 0.125f) *
           Codec<T>::dec(P.p[mslot(b, ODD ? opp7(i) : i)][site + src_off<ODD>(nb, mx7(i), my7(i), mz7(i))]);
    Bfd[(long long)b * g.n3 + site] = Codec<T>::enc(v);
  }
}

// The same for 16-bit storage and even nx, two sites (x0, x0 + 1), x0 even,
// per thread: the pair of a slot whose source is not shifted along x is one
// 32-bit load, the x-shifted sources (D3Q7 +-x on odd steps) two 16-bit
// loads, and the pair of B values one 32-bit store.  The sums run in the
// order of bfield_kernel, so both give the same B.
template <class T, bool ODD>
__global__ void bfield2_kernel(Slots<T> P, Grid g, T* __restrict__ Bfd) {
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + g.z0;
  if (x0 >= g.nx || y >= g.ny) return;
  const int s0 = (z * g.ny + y) * g.nx + x0;
  const Nbr n0 = make_nbr(x0, y, z, g), n1 = make_nbr(x0 + 1, y, z, g);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float v0 = 0.f, v1 = 0.f;
#pragma unroll
    for (int i = 0; i < kM; ++i) {
      const T* p = P.p[mslot(b, ODD ? opp7(i) : i)];
      const float w = i == 0 ? 0.25f : 0.125f;
      float a, c;
      if (!ODD || mx7(i) == 0) {
        // y and z offsets only: the same for both sites, and even
        const float2 v = dec2(p + s0 + src_off<ODD>(n0, 0, my7(i), mz7(i)));
        a = v.x;
        c = v.y;
      } else {
        a = Codec<T>::dec(p[s0 + src_off<ODD>(n0, mx7(i), 0, 0)]);
        c = Codec<T>::dec(p[s0 + 1 + src_off<ODD>(n1, mx7(i), 0, 0)]);
      }
      v0 += w * a;
      v1 += w * c;
    }
    enc2(Bfd + (long long)b * g.n3 + s0, v0, v1);
  }
}

template <class T>
cudaError_t bfield_t(int odd, const void* pop, Grid g, void* Bfd_, cudaStream_t s) {
  T* Bfd = static_cast<T*>(Bfd_);
  const Slots<T> P = make_slots<T>(pop, g);
  if constexpr (sizeof(T) == 2) {
    if (g.nx % 2 == 0) {
      const int pairs = g.nx / 2;
      const int bx = pairs >= 128 ? 128 : ((pairs + 31) / 32) * 32;
      const int by = 128 / bx < g.ny ? 128 / bx : g.ny;
      const dim3 bb(bx, by, 1), gb((pairs + bx - 1) / bx, (g.ny + by - 1) / by, g.nzi);
      if (odd)
        bfield2_kernel<T, true><<<gb, bb, 0, s>>>(P, g, Bfd);
      else
        bfield2_kernel<T, false><<<gb, bb, 0, s>>>(P, g, Bfd);
      return cudaGetLastError();
    }
  }
  const dim3 bb = site_block(g, 128), gb = site_grid(g, bb);
  if (odd)
    bfield_kernel<T, true><<<gb, bb, 0, s>>>(P, g, Bfd);
  else
    bfield_kernel<T, false><<<gb, bb, 0, s>>>(P, g, Bfd);
  return cudaGetLastError();
}

template <class T, int VAR>
void step_launch(int odd, const Slots<T>& P, Grid g, const StepConsts& k, unsigned* flag, const T* Bfd, dim3 gr,
                 dim3 b, bool flat, cudaStream_t s) {
  if (flat) {
    if (odd)
      step_kernel<T, true, VAR, true><<<gr, b, 0, s>>>(P, g, k, flag, Bfd);
    else
      step_kernel<T, false, VAR, true><<<gr, b, 0, s>>>(P, g, k, flag, Bfd);
  } else if (odd) {
    step_kernel<T, true, VAR><<<gr, b, 0, s>>>(P, g, k, flag, Bfd);
  } else {
    step_kernel<T, false, VAR><<<gr, b, 0, s>>>(P, g, k, flag, Bfd);
  }
}

template <class T>
cudaError_t step_t(int odd, void* pop, Grid g, const StepConsts& k, unsigned* flag, int variant, void* Bfd,
                   cudaStream_t s) {
  // flat blocks where blocks of x rows leave many lanes idle
  const int padded = (g.nx + 31) / 32 * 32;
  const bool flat = g.nx < padded && (double)g.nx / padded < 0.9;
  dim3 b = site_block(g, kStepThreads), gr = site_grid(g, b);
  if (flat) {
    b = dim3(kStepThreads, 1, 1);
    gr = dim3((unsigned)((g.n3i + kStepThreads - 1) / kStepThreads), 1, 1);
  }
  const Slots<T> P = make_slots<T>(pop, g);
  switch (variant) {
    case kVarFlame: step_launch<T, kVarFlame>(odd, P, g, k, flag, nullptr, gr, b, flat, s); break;
    case kVarBgkFluid: step_launch<T, kVarBgkFluid>(odd, P, g, k, flag, nullptr, gr, b, flat, s); break;
    case kVarEmhd: step_launch<T, kVarEmhd>(odd, P, g, k, flag, nullptr, gr, b, flat, s); break;
    case kVarFdCurrent: {
      if (!Bfd) return cudaErrorInvalidValue;
      const cudaError_t e = bfield_t<T>(odd, pop, g, Bfd, s);
      if (e != cudaSuccess) return e;
      step_launch<T, kVarFdCurrent>(odd, P, g, k, flag, static_cast<const T*>(Bfd), gr, b, flat, s);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}


}  // namespace

cudaError_t launch_bfield(int storage, int odd, const void* pop, Grid g, void* Bfd, cudaStream_t s) {
  if (!Bfd) return cudaErrorInvalidValue;
  switch (storage) {
    case 1: return bfield_t<float>(odd, pop, g, Bfd, s);
    case 2: return bfield_t<__half>(odd, pop, g, Bfd, s);
    case 3: return bfield_t<__nv_bfloat16>(odd, pop, g, Bfd, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step(int storage, int odd, void* pop, Grid g, const StepConsts& k, unsigned* flag,
                        cudaStream_t s, int variant, void* Bfd, int kernel) {
  if (step_row_supported(g, storage, variant, pop, kernel)) {
    if (variant == kVarFdCurrent) {
      const cudaError_t e = launch_bfield(storage, odd, pop, g, Bfd, s);
      if (e != cudaSuccess) return e;
    }
    return launch_step_row(storage, odd, pop, g, k, flag, s, variant, Bfd, 0, kernel);
  }
  switch (storage) {
    case 1: return step_t<float>(odd, pop, g, k, flag, variant, Bfd, s);
    case 2: return step_t<__half>(odd, pop, g, k, flag, variant, Bfd, s);
    case 3: return step_t<__nv_bfloat16>(odd, pop, g, k, flag, variant, Bfd, s);
  }
  return cudaErrorInvalidValue;
}


}  // namespace flame
