// step_row_fd.cu -- the row kernel (step_row.cuh) with J from the
// central-difference curl of the pre-collision B (the alternative to the
// moment current of Sec. 3.2).
#include "step_row.cuh"

namespace flame {

cudaError_t step_row_fd(const RowCall& c) { return row_call<kVarFdCurrent>(c); }

}  // namespace flame
