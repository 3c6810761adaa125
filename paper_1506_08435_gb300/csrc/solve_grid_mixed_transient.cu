// Instantiations of the persistent solve kernel for mode MODE_MIXED_TR.
#include "grid.cuh"

namespace nnqp {

GridKernel grid_kernel_mixed_transient(int fmt, int cgv, int tpb) {
    if (fmt == FMT_SELL_SMEM) {
        if (tpb != 512) return nullptr;
        switch (cgv) {
            case 1: return k_solve_grid<2, MODE_MIXED_TR, 1, 512>;
            case 2: return k_solve_grid<2, MODE_MIXED_TR, 2, 512>;
            default: return nullptr;
        }
    }
    if (fmt == FMT_SELL_TMA) return grid_kernel_tma(MODE_MIXED_TR, cgv, tpb);
    if (fmt != NN_FMT_SELL) return nullptr;
    if (tpb == 512) {
        switch (cgv) {
            case 1: return k_solve_grid<0, MODE_MIXED_TR, 1, 512>;
            case 2: return k_solve_grid<0, MODE_MIXED_TR, 2, 512>;
            default: return nullptr;
        }
    }
    if (tpb != 256) return nullptr;
    switch (cgv) {
        case 0: return k_solve_grid<0, MODE_MIXED_TR, 0, 256>;
        case 1: return k_solve_grid<0, MODE_MIXED_TR, 1, 256>;
        case 2: return k_solve_grid<0, MODE_MIXED_TR, 2, 256>;
        default: return nullptr;
    }
}

}  // namespace nnqp
