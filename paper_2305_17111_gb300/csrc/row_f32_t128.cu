// Row kernel, FP32 form, tiles of 128 events (VPL = 4 layout, 4 events per lane), 1 to 8 lines.
#define LMMEW_ROW_KERNEL_BODY
#include "row_kernel.cuh"

namespace lmmew {

RowKernel row_kernel_f32_t128(int W, bool streamed) {
    if (streamed) {
        switch (W) {
            case 1: return rowk::k_row<1, 0, kEPL, 4, true>;
            case 2: return rowk::k_row<2, 0, kEPL, 4, true>;
            case 3: return rowk::k_row<3, 0, kEPL, 4, true>;
            case 4: return rowk::k_row<4, 0, kEPL, 4, true>;
            case 5: return rowk::k_row<5, 0, kEPL, 4, true>;
            case 6: return rowk::k_row<6, 0, kEPL, 4, true>;
            case 7: return rowk::k_row<7, 0, kEPL, 4, true>;
            default: return rowk::k_row<8, 0, kEPL, 4, true>;
        }
    }
    switch (W) {
        case 1: return rowk::k_row<1, 0, kEPL, 4>;
        case 2: return rowk::k_row<2, 0, kEPL, 4>;
        case 3: return rowk::k_row<3, 0, kEPL, 4>;
        case 4: return rowk::k_row<4, 0, kEPL, 4>;
        case 5: return rowk::k_row<5, 0, kEPL, 4>;
        case 6: return rowk::k_row<6, 0, kEPL, 4>;
        case 7: return rowk::k_row<7, 0, kEPL, 4>;
        default: return rowk::k_row<8, 0, kEPL, 4>;
    }
}

}  // namespace lmmew
