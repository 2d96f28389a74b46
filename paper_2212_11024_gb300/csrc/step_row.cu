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

// The automatic choice among the row kernel's tilings, from a sweep of
// every multiple of 8 from 64 to 1024 with FP16 storage on ~4M-site
// lattices (nx x m x m, graph replay, GLUPS).  The unstaged pair kernel runs
// at 24.6-25.4 at every length; the staged kernel's whole rows run at 28-32
// where a row's block fits several times per SM and its stages are dense
// (64 28.1, 128 31.8, 192 29.3, 256 31.9, 320 30.0, 384 29.0, 448 30.3, 512
// 30.7, 768 28.5, 1024 31.5), and lose to the pair kernel where a block is
// under 48 threads (72-96: 18.6-24.5), where three stages of padded rows
// fit few blocks (136-152: 21.2-24.1), where a block of 260-320 threads
// fits once per SM (520-648: 20.0-24.9, half rows 22.5-26.7, ahead of the
// pair kernel from 608 where a half row is whole 16-byte units) and at
// 776-792 (24.4-25.0).  Ties (within 0.3) keep whole rows.  Odd row lengths
// take the one-site kernel.
int row_auto_segments(int nx) {
  if (nx % 8 != 0 || nx < 64 || nx > 1024) return 0;
  if ((nx > 64 && nx < 104) || (nx > 128 && nx < 160) || (nx >= 776 && nx <= 792)) return 0;
  if (nx > 512 && nx <= 648) return nx >= 608 && nx % 16 == 0 ? 2 : 0;
  return 1;
}

// Row lengths the row kernel stages: whole 16-byte units per row (up to 256
// sites by tensor-map boxes of runs placed at 128-byte aligned offsets,
// longer rows by bulk copies).
static bool row_length_ok(int nx) { return nx % 8 == 0; }

// The pair kernel: 16-bit storage, any even row length, a 4-byte aligned
// state (pairs are 32-bit accesses).
static bool pair_ok(Grid g, int storage, int variant, const void* pop) {
  return variant >= kVarFlame && variant <= kVarFdCurrent && (storage == 2 || storage == 3) && g.nx % 2 == 0 &&
         (reinterpret_cast<uintptr_t>(pop) & 3u) == 0;
}

// The staged tilings: 64 <= nx <= 1024, nx a multiple of 8, a 16-byte
// aligned state.
static bool staged_ok(Grid g, int storage, int variant, const void* pop) {
  return variant >= kVarFlame && variant <= kVarFdCurrent && (storage == 2 || storage == 3) && g.nx >= 64 &&
         g.nx <= 2 * kRowMaxThreads && row_length_ok(g.nx) && (reinterpret_cast<uintptr_t>(pop) & 15u) == 0;
}

bool step_row_supported(Grid g, int storage, int variant, const void* pop, int kernel) {
  switch (kernel) {
    case 1: return false;
    case 2: return staged_ok(g, storage, variant, pop);
    case 3: return staged_ok(g, storage, variant, pop) && g.nx > kBoxMaxX && g.nx % 16 == 0;
    case 4: return pair_ok(g, storage, variant, pop);
  }
  // automatic: the pair kernel or a staged tiling for every even row length
  return pair_ok(g, storage, variant, pop) &&
         (row_auto_segments(g.nx) == 0 || staged_ok(g, storage, variant, pop));
}

int row_segments(int nx, int kernel) {
  return kernel == 4 ? 0 : kernel == 3 ? 2 : kernel == 2 ? 1 : row_auto_segments(nx);
}

bool step_row_staged(Grid g, int storage, int variant, const void* pop, int kernel) {
  return step_row_supported(g, storage, variant, pop, kernel) && row_segments(g.nx, kernel) != 0;
}

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
