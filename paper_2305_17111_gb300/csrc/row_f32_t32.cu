// Row kernel, FP32 form, tiles of 32 events (VPL = 2 layout, 2 events per lane).
#define LMMEW_ROW_KERNEL_BODY
#include "row_kernel.cuh"

namespace lmmew {

RowKernel row_kernel_f32_t32(int W) {
    switch (W) {
        case 1: return rowk::k_row<1, 0, 2, 2>;
        case 2: return rowk::k_row<2, 0, 2, 2>;
        case 3: return rowk::k_row<3, 0, 2, 2>;
        case 4: return rowk::k_row<4, 0, 2, 2>;
        default: return nullptr;
    }
}

}  // namespace lmmew
