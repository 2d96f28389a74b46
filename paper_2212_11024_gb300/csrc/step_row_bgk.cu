// step_row_bgk.cu -- the row kernel (step_row.cuh) with the BGK fluid
// collision f* = f - w (f - f^mhd(0)) (Sec. 3.1.1).
#include "step_row.cuh"

namespace flame {

cudaError_t step_row_bgk(const RowCall& c) { return row_call<kVarBgkFluid>(c); }

}  // namespace flame
