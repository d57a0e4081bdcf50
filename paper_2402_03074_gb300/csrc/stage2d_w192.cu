// stage2d_w192.cu -- the 192-thread instantiations of the single-solve 2D stage kernel
// (stage2d_impl.cuh), compiled apart from the other widths.
#include "stage2d_impl.cuh"

namespace hw {

HW_STAGE2D_WIDTH(192)

}  // namespace hw
