// step.cu -- the fused FLAME collide-and-stream step (one thread per site,
// AA in-place streaming), plus the initialisation, moments and populations
// kernels that read the same state.
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
#include "flame_internal.h"
#include "lattice.cuh"

namespace flame {
namespace {

// Step launch: 256 threads per block (a whole 256-site x row at 256^3) and
// at most 80 registers per thread (3 resident blocks per SM); the block
// shape and register budget were chosen by timing at 256^3.
constexpr int kStepThreads = 256;
constexpr int kStepMinBlocks = 3;

// Site-index offsets of the periodic neighbours.
struct Nbr {
  int xm, xp, ym, yp, zm, zp;
  __device__ __forceinline__ int operator()(int cx, int cy, int cz) const {
    return (cx < 0 ? xm : (cx > 0 ? xp : 0)) + (cy < 0 ? ym : (cy > 0 ? yp : 0)) +
           (cz < 0 ? zm : (cz > 0 ? zp : 0));
  }
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, const Grid& g) {
  Nbr n;
  const int plane = g.nx * g.ny;
  n.xm = x == 0 ? g.nx - 1 : -1;
  n.xp = x == g.nx - 1 ? -(g.nx - 1) : 1;
  n.ym = y == 0 ? (g.ny - 1) * g.nx : -g.nx;
  n.yp = y == g.ny - 1 ? -(g.ny - 1) * g.nx : g.nx;
  n.zm = z == 0 ? (g.nz - 1) * plane : -plane;
  n.zp = z == g.nz - 1 ? -(g.nz - 1) * plane : plane;
  return n;
}

// AA pattern.  Pre-collision population on velocity c of a site:
//   even parity: same site, own slot;  odd: site - c, opposite slot.
// Post-collision population on velocity c:
//   even: same site, opposite slot;    odd: site + c, own slot.
template <bool ODD>
__device__ __forceinline__ long long src27(int i, int site, const Nbr& nb, long long n3) {
  return ODD ? (long long)opp27(i) * n3 + site + nb(-cx27(i), -cy27(i), -cz27(i))
             : (long long)i * n3 + site;
}
template <bool ODD>
__device__ __forceinline__ long long dst27(int i, int site, const Nbr& nb, long long n3) {
  return ODD ? (long long)i * n3 + site + nb(cx27(i), cy27(i), cz27(i))
             : (long long)opp27(i) * n3 + site;
}
template <bool ODD>
__device__ __forceinline__ long long src7(int b, int i, int site, const Nbr& nb, long long n3) {
  return ODD ? (long long)mslot(b, opp7(i)) * n3 + site + nb(-mx7(i), -my7(i), -mz7(i))
             : (long long)mslot(b, i) * n3 + site;
}
template <bool ODD>
__device__ __forceinline__ long long dst7(int b, int i, int site, const Nbr& nb, long long n3) {
  return ODD ? (long long)mslot(b, i) * n3 + site + nb(mx7(i), my7(i), mz7(i))
             : (long long)mslot(b, opp7(i)) * n3 + site;
}

// Base pointers of the 48 slots (slot q starts at q * N3), passed as kernel
// parameters so that each access is one index computation on a parameter.
template <class T>
struct Slots {
  T* p[kPop];
};

// Site offset of the source (pre-collision) and destination
// (post-collision) of the population on velocity (cx, cy, cz), and the
// slot used there, for the two AA parities.
template <bool ODD>
__device__ __forceinline__ int src_off(const Nbr& nb, int cx, int cy, int cz) {
  return ODD ? nb(-cx, -cy, -cz) : 0;
}
template <bool ODD>
__device__ __forceinline__ int dst_off(const Nbr& nb, int cx, int cy, int cz) {
  return ODD ? nb(cx, cy, cz) : 0;
}

template <class T, bool ODD>
__global__ void __launch_bounds__(kStepThreads, kStepMinBlocks)
    step_kernel(Slots<T> P, Grid g, StepConsts k, unsigned* __restrict__ flag) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
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
  const float gq = 4.f * k.omegaB;
  const float A[3] = {lam[1][2] - lam[2][1], lam[2][0] - lam[0][2], lam[0][1] - lam[1][0]};
  const float uxb[3] = {U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2], U[0] * B[1] - U[1] * B[0]};
  const float yv[3] = {-gq * (A[0] - 2.f * uxb[0]), -gq * (A[1] - 2.f * uxb[1]), -gq * (A[2] - 2.f * uxb[2])};
  const float sH = 2.f * k.alphaH * gq;
  const float yxb[3] = {yv[1] * B[2] - yv[2] * B[1], yv[2] * B[0] - yv[0] * B[2], yv[0] * B[1] - yv[1] * B[0]};
  const float yb = yv[0] * B[0] + yv[1] * B[1] + yv[2] * B[2];
  const float b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  const float iden = 1.f / (1.f + sH * sH * b2);
  float V[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float J = (yv[a] - sH * yxb[a] + sH * sH * yb * B[a]) * iden;
    V[a] = U[a] - k.alphaH * J;
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
      const float A0 = (Dxx * p2[px]) * p0y[py] + (Dyy * p2[py]) * p0x[px] + (Dxy * p1x[px]) * p1y[py];
      const float A1 = (Dxz * p1x[px]) * p0y[py] + (Dyz * p1y[py]) * p0x[px];
      const float A2 = (Dzz * p0x[px]) * p0y[py];
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
      const float vz[3] = {tz - Z1, Z0, tz + Z1};
#pragma unroll
      for (int pz = 0; pz < 3; ++pz) {
        const int i = idx27(px, py, pz);
        const int slot = ODD ? i : opp27(i);
        P.p[slot][site + dst_off<ODD>(nb, cx, cy, pz - 1)] = Codec<T>::enc(vz[pz]);
      }
    }
}

// ---------------------------------------------------------------------------
// Initialisation (FP64 arithmetic, once per run).

__device__ __forceinline__ double cdiff(const double* F, int a, int x, int y, int z, const Grid& g) {
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
  return 0.5 * (F[((long long)zp * g.ny + yp) * g.nx + xp] - F[((long long)zm * g.ny + ym) * g.nx + xm]);
}

template <class T>
__global__ void init_kernel(T* __restrict__ pop, Grid g, StepConsts k, int noneq, const double* __restrict__ rho_f,
                            const double* __restrict__ u, const double* __restrict__ Bf,
                            const double* __restrict__ gu, const double* __restrict__ gB,
                            unsigned* __restrict__ speed_bits) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const long long n3 = g.n3;
  const long long site = ((long long)z * g.ny + y) * g.nx + x;
  const double rho = rho_f ? rho_f[site] : 1.0;
  const double U[3] = {u[site], u[n3 + site], u[2 * n3 + site]};
  const double B[3] = {Bf[site], Bf[n3 + site], Bf[2 * n3 + site]};
  double du[9], dB[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      du[3 * a + b] = gu ? gu[(3 * a + b) * n3 + site] : cdiff(u + b * n3, a, x, y, z, g);
      dB[3 * a + b] = gB ? gB[(3 * a + b) * n3 + site] : cdiff(Bf + b * n3, a, x, y, z, g);
    }
  const double J0[3] = {dB[5] - dB[7], dB[6] - dB[2], dB[1] - dB[3]};  // curl B
  const double omega = (double)k.omega, omegaB = (double)k.omegaB, aH = (double)k.alphaH;
  const double Br[3] = {(double)k.Bref[0], (double)k.Bref[1], (double)k.Bref[2]};
  const double b[3] = {B[0] - Br[0], B[1] - Br[1], B[2] - Br[2]};
  double N[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) N[a][c] = Br[a] * b[c] + b[a] * Br[c] + b[a] * b[c];
  const double miso = Br[0] * b[0] + Br[1] * b[1] + Br[2] * b[2] + 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  const double trN3 = (N[0][0] + N[1][1] + N[2][2]) / 3.0;
  double Pn[3][3];  // first-order non-equilibrium stress -(rho cs^2/omega)(du + du^T)
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) Pn[a][c] = noneq ? -(rho / (3.0 * omega)) * (du[3 * a + c] + du[3 * c + a]) : 0.0;
  const double trPn3 = (Pn[0][0] + Pn[1][1] + Pn[2][2]) / 3.0;
  const double drho = rho - (double)k.rho0;
#pragma unroll 1
  for (int i = 0; i < kQ; ++i) {
    const int c[3] = {cx27(i), cy27(i), cz27(i)};
    double E = 0.0;  // prod(psi/w1) - 1, accumulated stably
    for (int a = 0; a < 3; ++a) {
      const double uu = U[a] * U[a];
      const double ea = c[a] == 0 ? -1.5 * uu : 3.0 * uu + 3.0 * c[a] * U[a];
      E = E + ea + E * ea;
    }
    double cNc = 0.0, cPc = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) {
        cNc += c[a] * c[d] * N[a][d];
        cPc += c[a] * c[d] * Pn[a][d];
      }
    const double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    const double L = 4.5 * (miso * (c2 - 1.0) - cNc + trN3);
    const double ne = 4.5 * (cPc - trPn3);
    pop[(long long)i * n3 + site] = Codec<T>::enc((float)(drho + rho * E + L + ne));
  }
  const double V[3] = {U[0] - aH * J0[0], U[1] - aH * J0[1], U[2] - aH * J0[2]};
  for (int bb = 0; bb < 3; ++bb)
    for (int i = 0; i < kM; ++i) {
      const int xi[3] = {mx7(i), my7(i), mz7(i)};
      double l0 = 0.0, ne = 0.0;
      for (int a = 0; a < 3; ++a) {
        l0 += xi[a] * (V[a] * B[bb] - B[a] * V[bb]);
        ne += xi[a] * dB[3 * a + bb];
      }
      const double v = b[bb] + 4.0 * l0 - (noneq ? ne / omegaB : 0.0);
      pop[(long long)mslot(bb, i) * n3 + site] = Codec<T>::enc((float)v);
    }
  const double va = sqrt((B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho);
  const double um = sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
  const float sp = (float)fmax(va, um);
  if (isfinite(sp)) atomicMax(speed_bits, __float_as_uint(sp));
  else atomicMax(speed_bits, 0x7f800000u);
}

// ---------------------------------------------------------------------------
// Moments and decoded populations (FP64 arithmetic from the stored values).

template <class T, bool ODD>
__device__ __forceinline__ void load_site(const T* __restrict__ pop, int site, const Nbr& nb, long long n3,
                                          double sf[kQ], double sg[3][kM]) {
#pragma unroll
  for (int i = 0; i < kQ; ++i) sf[i] = (double)Codec<T>::dec(pop[src27<ODD>(i, site, nb, n3)]);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int i = 0; i < kM; ++i) sg[b][i] = (double)Codec<T>::dec(pop[src7<ODD>(b, i, site, nb, n3)]);
}

struct SiteMoments {
  double rho, U[3], B[3], J[3], trlam;
};

__device__ __forceinline__ SiteMoments site_moments(const double sf[kQ], const double sg[3][kM], const StepConsts& k) {
  SiteMoments m;
  double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const double t = w27d(i) * sf[i];
    drho += t;
    j[0] += cx27(i) * t;
    j[1] += cy27(i) * t;
    j[2] += cz27(i) * t;
  }
  m.rho = (double)k.rho0 + drho;
  for (int a = 0; a < 3; ++a) m.U[a] = j[a] / m.rho;
  double lam[3][3];
  for (int b = 0; b < 3; ++b) {
    m.B[b] = (double)k.Bref[b] + 0.25 * sg[b][0] + 0.125 * (sg[b][1] + sg[b][2] + sg[b][3] + sg[b][4] + sg[b][5] + sg[b][6]);
    lam[0][b] = 0.125 * (sg[b][1] - sg[b][2]);
    lam[1][b] = 0.125 * (sg[b][3] - sg[b][4]);
    lam[2][b] = 0.125 * (sg[b][5] - sg[b][6]);
  }
  m.trlam = lam[0][0] + lam[1][1] + lam[2][2];
  const double gq = 4.0 * (double)k.omegaB;
  const double* U = m.U;
  const double* B = m.B;
  const double A[3] = {lam[1][2] - lam[2][1], lam[2][0] - lam[0][2], lam[0][1] - lam[1][0]};
  const double uxb[3] = {U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2], U[0] * B[1] - U[1] * B[0]};
  const double yv[3] = {-gq * (A[0] - 2.0 * uxb[0]), -gq * (A[1] - 2.0 * uxb[1]), -gq * (A[2] - 2.0 * uxb[2])};
  const double s = 2.0 * (double)k.alphaH * gq;
  const double yxb[3] = {yv[1] * B[2] - yv[2] * B[1], yv[2] * B[0] - yv[0] * B[2], yv[0] * B[1] - yv[1] * B[0]};
  const double yb = yv[0] * B[0] + yv[1] * B[1] + yv[2] * B[2];
  const double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  for (int a = 0; a < 3; ++a) m.J[a] = (yv[a] - s * yxb[a] + s * s * yb * B[a]) / (1.0 + s * s * b2);
  return m;
}

template <class T, bool ODD>
__global__ void moments_kernel(const T* __restrict__ pop, Grid g, StepConsts k, double* __restrict__ rho,
                               double* __restrict__ u, double* __restrict__ B, double* __restrict__ J) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int site = (z * g.ny + y) * g.nx + x;
  const Nbr nb = make_nbr(x, y, z, g);
  double sf[kQ], sg[3][kM];
  load_site<T, ODD>(pop, site, nb, g.n3, sf, sg);
  const SiteMoments m = site_moments(sf, sg, k);
  if (rho) rho[site] = m.rho;
  for (int a = 0; a < 3; ++a) {
    if (u) u[a * g.n3 + site] = m.U[a];
    if (B) B[a * g.n3 + site] = m.B[a];
    if (J) J[a * g.n3 + site] = m.J[a];
  }
}

template <class T, bool ODD>
__global__ void populations_kernel(const T* __restrict__ pop, Grid g, StepConsts k, double* __restrict__ f) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int site = (z * g.ny + y) * g.nx + x;
  const Nbr nb = make_nbr(x, y, z, g);
  double sf[kQ], sg[3][kM];
  load_site<T, ODD>(pop, site, nb, g.n3, sf, sg);
  const double Br[3] = {(double)k.Bref[0], (double)k.Bref[1], (double)k.Bref[2]};
  const double br2 = Br[0] * Br[0] + Br[1] * Br[1] + Br[2] * Br[2];
#pragma unroll 1
  for (int i = 0; i < kQ; ++i) {
    const double c2 = cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i);
    const double cb = cx27(i) * Br[0] + cy27(i) * Br[1] + cz27(i) * Br[2];
    const double ell = 4.5 * (0.5 * br2 * (c2 - 1.0 / 3.0) - cb * cb);  // rest Lorentz term / w
    f[(long long)i * g.n3 + site] = w27d(i) * ((double)k.rho0 + ell + sf[i]);
  }
  for (int b = 0; b < 3; ++b)
    for (int i = 0; i < kM; ++i) f[(long long)mslot(b, i) * g.n3 + site] = w7d(i) * (Br[b] + sg[b][i]);
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
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n3; s += (long long)gridDim.x * blockDim.x) {
    const int site = (int)s;
    const int x = site % g.nx, y = (site / g.nx) % g.ny, z = site / (g.nx * g.ny);
    const Nbr nb = make_nbr(x, y, z, g);
    double sf[kQ], sg[3][kM];
    load_site<T, ODD>(pop, site, nb, n3, sf, sg);
    const SiteMoments m = site_moments(sf, sg, k);
    const double b[3] = {m.B[0] - k.Bref[0], m.B[1] - k.Bref[1], m.B[2] - k.Bref[2]};
    const double uu = m.U[0] * m.U[0] + m.U[1] * m.U[1] + m.U[2] * m.U[2];
    const double dv = 4.0 * (double)k.omegaB * m.trlam;
    const bool ok = isfinite(m.rho + uu + b[0] + b[1] + b[2] + m.J[0] + m.J[1] + m.J[2]);
    if (!ok) {
      acc[16] += 1.0;
      continue;
    }
    acc[0] += m.rho;
    for (int a = 0; a < 3; ++a) {
      acc[1 + a] += m.rho * m.U[a];
      acc[4 + a] += m.B[a];
      acc[10 + a] += m.U[a];
    }
    acc[7] += uu;
    acc[8] += b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    acc[9] += m.U[0] * b[0] + m.U[1] * b[1] + m.U[2] * b[2];
    acc[13] += m.J[0] * m.J[0] + m.J[1] * m.J[1] + m.J[2] * m.J[2];
    acc[14] = fmax(acc[14], sqrt(uu));
    acc[15] += dv * dv;
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
dim3 site_block(const Grid& g, int threads = 128) {
  int bx = g.nx >= threads ? threads : ((g.nx + 31) / 32) * 32;
  int by = threads / bx;
  if (by > g.ny) by = g.ny;
  if (by < 1) by = 1;
  return dim3(bx, by, 1);
}

dim3 site_grid(const Grid& g, dim3 b) { return dim3((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nz); }

template <class T>
cudaError_t step_t(int odd, void* pop, Grid g, const StepConsts& k, unsigned* flag, cudaStream_t s) {
  const dim3 b = site_block(g, kStepThreads), gr = site_grid(g, b);
  Slots<T> P;
  for (int q = 0; q < kPop; ++q) P.p[q] = static_cast<T*>(pop) + (size_t)q * (size_t)g.n3;
  if (odd)
    step_kernel<T, true><<<gr, b, 0, s>>>(P, g, k, flag);
  else
    step_kernel<T, false><<<gr, b, 0, s>>>(P, g, k, flag);
  return cudaGetLastError();
}

template <class T>
cudaError_t moments_t(int odd, const void* pop, Grid g, const StepConsts& k, double* rho, double* u, double* B,
                      double* J, cudaStream_t s) {
  const dim3 b = site_block(g), gr = site_grid(g, b);
  if (odd)
    moments_kernel<T, true><<<gr, b, 0, s>>>(static_cast<const T*>(pop), g, k, rho, u, B, J);
  else
    moments_kernel<T, false><<<gr, b, 0, s>>>(static_cast<const T*>(pop), g, k, rho, u, B, J);
  return cudaGetLastError();
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

cudaError_t launch_step(int storage, int odd, void* pop, Grid g, const StepConsts& k, unsigned* flag,
                        cudaStream_t s) {
  switch (storage) {
    case 1: return step_t<float>(odd, pop, g, k, flag, s);
    case 2: return step_t<__half>(odd, pop, g, k, flag, s);
    case 3: return step_t<__nv_bfloat16>(odd, pop, g, k, flag, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_init(int storage, void* pop, Grid g, const StepConsts& k, int noneq, const double* rho,
                        const double* u, const double* B, const double* gu, const double* gB,
                        unsigned* speed_bits, cudaStream_t s) {
  const dim3 b = site_block(g), gr = site_grid(g, b);
  switch (storage) {
    case 1: init_kernel<float><<<gr, b, 0, s>>>(static_cast<float*>(pop), g, k, noneq, rho, u, B, gu, gB, speed_bits); break;
    case 2: init_kernel<__half><<<gr, b, 0, s>>>(static_cast<__half*>(pop), g, k, noneq, rho, u, B, gu, gB, speed_bits); break;
    case 3: init_kernel<__nv_bfloat16><<<gr, b, 0, s>>>(static_cast<__nv_bfloat16*>(pop), g, k, noneq, rho, u, B, gu, gB, speed_bits); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_moments(int storage, int odd, const void* pop, Grid g, const StepConsts& k, double* rho,
                           double* u, double* B, double* J, cudaStream_t s) {
  switch (storage) {
    case 1: return moments_t<float>(odd, pop, g, k, rho, u, B, J, s);
    case 2: return moments_t<__half>(odd, pop, g, k, rho, u, B, J, s);
    case 3: return moments_t<__nv_bfloat16>(odd, pop, g, k, rho, u, B, J, s);
  }
  return cudaErrorInvalidValue;
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
