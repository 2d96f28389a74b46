// aa.cuh -- addressing of the in-place AA streaming pattern over the
// 48-slot structure-of-arrays population state, shared by the step, the
// diagnostics and the adjoint kernels.
#pragma once

#include "flame_internal.h"
#include "lattice.cuh"

namespace flame {

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
  return ODD ? (long long)phys(opp27(i)) * n3 + site + nb(-cx27(i), -cy27(i), -cz27(i))
             : (long long)phys(i) * n3 + site;
}
template <bool ODD>
__device__ __forceinline__ long long dst27(int i, int site, const Nbr& nb, long long n3) {
  return ODD ? (long long)phys(i) * n3 + site + nb(cx27(i), cy27(i), cz27(i))
             : (long long)phys(opp27(i)) * n3 + site;
}
template <bool ODD>
__device__ __forceinline__ long long src7(int b, int i, int site, const Nbr& nb, long long n3) {
  return ODD ? (long long)phys(mslot(b, opp7(i))) * n3 + site + nb(-mx7(i), -my7(i), -mz7(i))
             : (long long)phys(mslot(b, i)) * n3 + site;
}
template <bool ODD>
__device__ __forceinline__ long long dst7(int b, int i, int site, const Nbr& nb, long long n3) {
  return ODD ? (long long)phys(mslot(b, i)) * n3 + site + nb(mx7(i), my7(i), mz7(i))
             : (long long)phys(mslot(b, opp7(i))) * n3 + site;
}

// Base pointers of the 48 populations in natural slot order (natural slot
// q starts at phys(q) * N3), passed as kernel parameters so that each access
// is one index computation on a parameter.
template <class T>
struct Slots {
  T* p[kPop];
};
template <class T>
inline Slots<T> make_slots(const void* pop, const Grid& g) {
  Slots<T> P;
  for (int q = 0; q < kPop; ++q)
    P.p[q] = const_cast<T*>(static_cast<const T*>(pop)) + (size_t)phys(q) * (size_t)g.n3;
  return P;
}

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

// Block of `threads` threads: x-rows of up to `threads` sites, several
// rows per block when nx is small.
inline dim3 site_block(const Grid& g, int threads = 128) {
  int bx = g.nx >= threads ? threads : ((g.nx + 31) / 32) * 32;
  int by = threads / bx;
  if (by > g.ny) by = g.ny;
  if (by < 1) by = 1;
  return dim3(bx, by, 1);
}

// One grid z-layer per updated plane (z = blockIdx.z + g.z0).
inline dim3 site_grid(const Grid& g, dim3 b) { return dim3((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nzi); }

}  // namespace flame
