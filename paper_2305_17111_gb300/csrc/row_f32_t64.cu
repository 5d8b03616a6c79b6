// Row kernel, FP32 form, tiles of 64 events (VPL = 2 layout, 4 events per lane).
#define LMMEW_ROW_KERNEL_BODY
#include "row_kernel.cuh"

namespace lmmew {

RowKernel row_kernel_f32_t64(int W, bool streamed) {
    if (streamed) {
        switch (W) {
            case 1: return rowk::k_row<1, 0, 4, 2, true>;
            case 2: return rowk::k_row<2, 0, 4, 2, true>;
            case 3: return rowk::k_row<3, 0, 4, 2, true>;
            case 4: return rowk::k_row<4, 0, 4, 2, true>;
            default: return nullptr;
        }
    }
    switch (W) {
        case 1: return rowk::k_row<1, 0, 4, 2>;
        case 2: return rowk::k_row<2, 0, 4, 2>;
        case 3: return rowk::k_row<3, 0, 4, 2>;
        case 4: return rowk::k_row<4, 0, 4, 2>;
        default: return nullptr;
    }
}

}  // namespace lmmew
