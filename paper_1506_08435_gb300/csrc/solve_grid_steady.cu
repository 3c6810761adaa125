// Instantiations of the persistent solve kernel for mode MODE_STEADY.
#include "grid.cuh"

namespace nnqp {

GridKernel grid_kernel_steady(int fmt, int cgv, int tpb) {
    if (fmt == FMT_SELL_SMEM) {
        if (tpb != 512) return nullptr;
        switch (cgv) {
            case 1: return k_solve_grid<2, MODE_STEADY, 1, 512>;
            case 2: return k_solve_grid<2, MODE_STEADY, 2, 512>;
            default: return nullptr;
        }
    }
    if (fmt == NN_FMT_CSR) {
        if (tpb != 256) return nullptr;
        switch (cgv) {
            case 0: return k_solve_grid<1, MODE_STEADY, 0, 256>;
            case 1: return k_solve_grid<1, MODE_STEADY, 1, 256>;
            default: return nullptr;
        }
    }
    if (tpb == 768) {
        switch (cgv) {
            case 0: return k_solve_grid<0, MODE_STEADY, 0, 768>;
            case 3: return k_solve_grid<0, MODE_STEADY, 3, 768>;
            default: return nullptr;
        }
    }
    if (tpb == 512) {
        switch (cgv) {
            case 1: return k_solve_grid<0, MODE_STEADY, 1, 512>;
            case 2: return k_solve_grid<0, MODE_STEADY, 2, 512>;
            default: return nullptr;
        }
    }
    if (tpb != 256) return nullptr;
    switch (cgv) {
        case 0: return k_solve_grid<0, MODE_STEADY, 0, 256>;
        case 1: return k_solve_grid<0, MODE_STEADY, 1, 256>;
        case 2: return k_solve_grid<0, MODE_STEADY, 2, 256>;
        case 3: return k_solve_grid<0, MODE_STEADY, 3, 256>;
        default: return nullptr;
    }
}

}  // namespace nnqp
