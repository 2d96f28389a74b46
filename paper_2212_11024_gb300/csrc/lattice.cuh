// lattice.cuh -- lattice constants and storage encodings of the GB300 FLAME
// step.  Lattice units throughout: dx = dt = 1, c_s^2 = 1/3 (Sec. 3.1.1),
// C^2 = 1/4 from 2C = sqrt(3) c_s (eq. lattice_coincidence).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace flame {

constexpr int kQ = 27;    // D3Q27 fluid velocities
constexpr int kM = 7;     // D3Q7 magnetic velocities
constexpr int kPop = 48;  // 27 + 3 * 7 populations per site

// App. A velocity set, in the paper's order (i and i+13 are opposite).
__host__ __device__ constexpr int cx27(int i) {
  constexpr int t[kQ] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, -1, -1, -1, -1, 1, 0, 0, 1, 1, 1, 1, 0, 0, 1, 1, 1, 1};
  return t[i];
}
__host__ __device__ constexpr int cy27(int i) {
  constexpr int t[kQ] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, -1, -1, 1, 1, 0, 1, 0, 1, -1, 0, 0, 1, 1, 1, 1, -1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz27(int i) {
  constexpr int t[kQ] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
  return t[i];
}

// Index of the D3Q27 velocity (px-1, py-1, pz-1), p = 0, 1, 2.
__host__ __device__ constexpr int idx27(int px, int py, int pz) {
  constexpr int t[kQ] = {10, 8, 26, 6, 3, 20, 12, 22, 24, 4, 2, 18, 1, 0, 14, 5, 15, 17, 11, 9, 25, 7, 16, 19, 13, 21, 23};
  return t[px + 3 * py + 9 * pz];
}
constexpr bool idx27_consistent() {
  for (int pz = 0; pz < 3; ++pz)
    for (int py = 0; py < 3; ++py)
      for (int px = 0; px < 3; ++px) {
        const int i = idx27(px, py, pz);
        if (cx27(i) != px - 1 || cy27(i) != py - 1 || cz27(i) != pz - 1) return false;
      }
  return true;
}
static_assert(idx27_consistent(), "idx27 must invert the App. A velocity table");

// D3Q7 (Sec. 3.2): rest, +x, -x, +y, -y, +z, -z.
__host__ __device__ constexpr int mx7(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
__host__ __device__ constexpr int my7(int i) { return i == 3 ? 1 : (i == 4 ? -1 : 0); }
__host__ __device__ constexpr int mz7(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }

__host__ __device__ constexpr int opp27(int i) { return i == 0 ? 0 : (i <= 13 ? i + 13 : i - 13); }
__host__ __device__ constexpr int opp7(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Natural slot of a population: fluid q (App. A order), magnetic 27 + 7b + i.
__host__ __device__ constexpr int mslot(int b, int i) { return kQ + kM * b + i; }

// Storage slot of natural slot q in the state: fluid populations in
// velocity-cube order (cx+1) + 3(cy+1) + 9(cz+1), magnetic ones
// velocity-major 27 + 3i + b.  Then the 48 rows an odd AA step reads for an
// x row form 16 runs of 3 consecutive storage slots, each run from a single
// (y, z) row: the fluid run of (cy, cz) and the magnetic run of velocity i.
__host__ __device__ constexpr int phys(int q) {
  return q < kQ ? (cx27(q) + 1) + 3 * (cy27(q) + 1) + 9 * (cz27(q) + 1) : kQ + 3 * ((q - kQ) % kM) + (q - kQ) / kM;
}
constexpr bool phys_is_permutation() {
  for (int a = 0; a < kPop; ++a) {
    if (phys(a) < 0 || phys(a) >= kPop) return false;
    for (int b = a + 1; b < kPop; ++b)
      if (phys(a) == phys(b)) return false;
  }
  return true;
}
static_assert(phys_is_permutation(), "storage slots must be a permutation of the natural slots");

// Sec. 3.1.1 weights by |c|^2 (8/27, 2/27, 1/54, 1/216); they factor into
// the 1-D weights 2/3 (c = 0) and 1/6 (c = +-1).
__host__ __device__ constexpr double w27d(int i) {
  return (cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i)) == 0   ? 8.0 / 27.0
         : (cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i)) == 1 ? 2.0 / 27.0
         : (cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i)) == 2 ? 1.0 / 54.0
                                                                            : 1.0 / 216.0;
}
// 216 w_i: 64, 16, 4, 1 -- exact in FP32, so moment sums in the kernel use
// the same weights the collision conserves.
__host__ __device__ constexpr int w27x216(int i) {
  return (cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i)) == 0   ? 64
         : (cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i)) == 1 ? 16
         : (cx27(i) * cx27(i) + cy27(i) * cy27(i) + cz27(i) * cz27(i)) == 2 ? 4
                                                                            : 1;
}
// Sec. 3.2 weights: 1/4 rest, 1/8 faces.
__host__ __device__ constexpr double w7d(int i) { return i == 0 ? 0.25 : 0.125; }

// ---------------------------------------------------------------------------
// Storage encodings.  A slot holds s = (population - reference) / weight in
// one of three element types; decode gives FP32, encode rounds to nearest
// even.
template <class T>
struct Codec;

template <>
struct Codec<float> {
  static __device__ __forceinline__ float load(const float* p) { return *p; }
  static __device__ __forceinline__ float dec(float v) { return v; }
  static __device__ __forceinline__ float enc(float v) { return v; }
};

template <>
struct Codec<__half> {
  static __device__ __forceinline__ __half load(const __half* p) { return *p; }
  static __device__ __forceinline__ float dec(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half enc(float v) { return __float2half_rn(v); }
};

template <>
struct Codec<__nv_bfloat16> {
  static __device__ __forceinline__ __nv_bfloat16 load(const __nv_bfloat16* p) { return *p; }
  static __device__ __forceinline__ float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 enc(float v) { return __float2bfloat16_rn(v); }
};

// Two consecutive 16-bit values as one 32-bit access (4-byte aligned).
__device__ __forceinline__ float2 dec2(const __half* p) { return __half22float2(*reinterpret_cast<const __half2*>(p)); }
__device__ __forceinline__ float2 dec2(const __nv_bfloat16* p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
__device__ __forceinline__ void enc2(__half* p, float a, float b) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void enc2(__nv_bfloat16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}

}  // namespace flame
