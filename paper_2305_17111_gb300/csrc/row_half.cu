// Row kernel, reduced-precision forms (FP16 / BF16 scatter sums), tiles of 128 events, up to 4 lines.
#define LMMEW_ROW_KERNEL_BODY
#include "row_kernel.cuh"

namespace lmmew {

RowKernel row_kernel_half(int W, int prec) {
    if (prec == 1) {
        switch (W) {
            case 1: return rowk::k_row<1, 1, kEPL, 4>;
            case 2: return rowk::k_row<2, 1, kEPL, 4>;
            case 3: return rowk::k_row<3, 1, kEPL, 4>;
            case 4: return rowk::k_row<4, 1, kEPL, 4>;
            default: return nullptr;
        }
    }
    if (prec == 2) {
        switch (W) {
            case 1: return rowk::k_row<1, 2, kEPL, 4>;
            case 2: return rowk::k_row<2, 2, kEPL, 4>;
            case 3: return rowk::k_row<3, 2, kEPL, 4>;
            case 4: return rowk::k_row<4, 2, kEPL, 4>;
            default: return nullptr;
        }
    }
    return nullptr;
}

}  // namespace lmmew
