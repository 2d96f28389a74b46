// step_row_emhd.cu -- the row kernel (step_row.cuh) with the electron-MHD
// magnetic equilibrium and current, U dropped (Sec. 5).
#include "step_row.cuh"

namespace flame {

cudaError_t step_row_emhd(const RowCall& c) { return row_call<kVarEmhd>(c); }

}  // namespace flame
