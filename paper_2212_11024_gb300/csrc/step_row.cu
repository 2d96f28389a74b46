// step_row.cu -- the row kernel (step_row.cuh) for the paper's scheme, and
// the host side shared by all variants: tensor maps, where the row kernel is
// used, the launch entry and the pre-capture configuration.
#include "step_row.cuh"

namespace flame {

// Tensor maps of a state (16-bit values), cached for the last state seen by
// this thread.  The encoder comes from the driver through the runtime, so the
// library links no driver library.
cudaError_t row_maps(const void* pop, const Grid& g, RowMaps* out) {
  thread_local const void* last_pop = nullptr;
  thread_local Grid last_g{};
  thread_local RowMaps last{};
  if (pop == last_pop && g.nx == last_g.nx && g.ny == last_g.ny && g.nz == last_g.nz) {
    *out = last;
    return cudaSuccess;
  }
  // looked up once (thread-safe initialisation of a function-local static)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    const cudaError_t e =
        cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    return e == cudaSuccess && q == cudaDriverEntryPointSuccess ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)
                                                                : nullptr;
  }();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)kPop};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 2, (cuuint64_t)g.nx * g.ny * 2, (cuuint64_t)g.n3 * 2};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  RowMaps m;
  for (int w = 0; w < 2; ++w) {
    const cuuint32_t box[4] = {(cuuint32_t)g.nx, 1, 1, w == 0 ? (cuuint32_t)kPop : 3u};
    CUresult r = encode(w == 0 ? &m.all : &m.run, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(pop), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  last_pop = pop;
  last_g = g;
  last = m;
  *out = m;
  return cudaSuccess;
}

cudaError_t step_row_flame(const RowCall& c) { return row_call<kVarFlame>(c); }

// Row lengths where the row kernel beats the one-site kernel, and with how
// many segments per tile.  Timed with FP16 storage on ~4M-site lattices
// (nx x m x m, GLUPS; whole rows / half rows / one-site): 72 18.6 / - /
// 18.9, 96 24.5 / - / 23.5, 120 28.2 / - / 23.2, 136 21.3 / - / 20.5, 160
// 25.2 / - / 22.6, 200 26.5 / - / 21.9, 224 28.8 / - / 23.3, 248 28.8 / - /
// 23.6, 256 31.9 / - / 24.2, 264 24.5 / - / 18.9, 320 29.2 / 20.6 / 21.2, 328 24.3 / - / 20.7,
// 384 26.6 / 22.0 / 22.5, 400 26.7 / 21.8 / 22.0, 448 27.6 / 21.9 / 22.8,
// 456 26.7 / - / 23.0, 504 28.5 / - / 24.1, 512 30.7 / 27.5 / 24.4, 520
// 19.6 / - / 20.7, 528 20.1 / 22.5 / 20.9, 544 20.8 / 23.2 / 21.3, 552 20.8
// / - / 21.3, 560 21.3 / 24.0 / 21.5, 568 21.3 / - / 21.7, 576 21.9 / 24.4
// / 21.9, 640 24.2 / 26.7 / 23.0, 704 25.0 / 20.9 / 23.2, 744 26.6 / - /
// 23.9, 768 27.8 / 24.6 / 24.3, 832 24.6 / 22.2 / 22.2, 896 26.3 / 23.7 /
// 22.9, 960 27.9 / 23.7 / 23.3, 1000 28.1 / - / 22.7, 1024 29.3 / 26.5 /
// 23.1 (384, 448 and 704-960 before the direct stores addressed their rows
// from slot bases, which gained 5-8 % at 320-1024; 64-192 as in earlier
// timings: 28.0 / 24.1, 31.8 / 24.2, 29.4 / 23.5 whole rows against
// one-site).  Whole rows win from 96 sites (and at 64) up to 512 and above
// 640; below 96 a block of under 48 threads carries a tile's copies for too
// few sites and the one-site kernel is as fast.  Between 512 and 640, a
// whole row's block of 260-320 threads (128 registers each) fits once per
// SM; there half rows per tile (three blocks per SM) are the faster tiling
// where a half row is a whole number of 16-byte units (nx a multiple of
// 16), and the one-site kernel where it is not.  Elsewhere half rows lose:
// twice the copies per site (96 per tile on odd steps, the halo across a
// row's end by a copy of its own) for the same warps per SM.
bool row_kernel_wins(int nx) {
  return !((nx > 512 && nx <= 640 && nx % 16 != 0) || (nx < 96 && nx % 64 != 0));
}

// Segments per tile of the automatic choice (kernel = 0).
int row_auto_segments(int nx) { return nx > 512 && nx <= 640 ? 2 : 1; }

// Row lengths the row kernel stages: whole 16-byte units per row (up to 256
// sites by tensor-map boxes of runs placed at 128-byte aligned offsets,
// longer rows by bulk copies).
static bool row_length_ok(int nx) { return nx % 8 == 0; }

bool step_row_supported(Grid g, int storage, int variant, const void* pop, int kernel) {
  if (kernel == 1) return false;
  const bool base = variant >= kVarFlame && variant <= kVarFdCurrent && (storage == 2 || storage == 3) &&
                    g.nx >= 64 && g.nx <= 2 * kRowMaxThreads && row_length_ok(g.nx) &&
                    (reinterpret_cast<uintptr_t>(pop) & 15u) == 0;
  if (!base) return false;
  if (kernel == 3) return g.nx > kBoxMaxX && g.nx % 16 == 0;  // half rows: whole 16-byte units per half
  if (kernel == 2) return true;
  return row_kernel_wins(g.nx);
}

int row_segments(int nx, int kernel) { return kernel == 3 ? 2 : kernel == 2 ? 1 : row_auto_segments(nx); }

namespace {
cudaError_t row_variant(int variant, const RowCall& c) {
  switch (variant) {
    case kVarFlame: return step_row_flame(c);
    case kVarBgkFluid: return step_row_bgk(c);
    case kVarEmhd: return step_row_emhd(c);
    case kVarFdCurrent: return step_row_fd(c);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_step_row(int storage, int odd, void* pop, Grid g, const StepConsts& k, unsigned* flag,
                            cudaStream_t s, int variant, const void* Bfd, unsigned stall_tries, int kernel) {
  const RowWait wt{stall_tries ? stall_tries : kWaitTries, stall_tries ? 1 : 0};
  return row_variant(variant, RowCall{storage, odd, row_segments(g.nx, kernel), pop, g, k, flag, Bfd, s, true, wt});
}

cudaError_t prepare_step(int storage, const void* pop, Grid g, int variant, int kernel) {
  if (!step_row_supported(g, storage, variant, pop, kernel)) return cudaSuccess;
  // a placeholder field: only the configuration is settled, nothing is read
  static const unsigned no_field = 0u;
  for (int odd = 0; odd < 2; ++odd) {
    const cudaError_t e = row_variant(variant, RowCall{storage, odd, row_segments(g.nx, kernel), const_cast<void*>(pop),
                                                       g, StepConsts{}, nullptr, &no_field, nullptr, false,
                                                       RowWait{kWaitTries, 0}});
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace flame
