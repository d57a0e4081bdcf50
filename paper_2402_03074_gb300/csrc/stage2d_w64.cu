// stage2d_w64.cu -- the 64-thread instantiations of the single-solve 2D stage kernel
// (stage2d_impl.cuh), compiled apart from the other widths.
#include "stage2d_impl.cuh"

namespace hw {

HW_STAGE2D_WIDTH(64)

}  // namespace hw
