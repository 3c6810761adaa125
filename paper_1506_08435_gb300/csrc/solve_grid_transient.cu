// Instantiations of the persistent solve kernel for mode MODE_TRANSIENT.
#include "grid.cuh"

namespace nnqp {

GridKernel grid_kernel_transient(int fmt, int cgv, int tpb) {
    if (fmt == FMT_SELL_SMEM) {
        if (tpb != 512) return nullptr;
        switch (cgv) {
            case 1: return k_solve_grid<2, MODE_TRANSIENT, 1, 512>;
            case 2: return k_solve_grid<2, MODE_TRANSIENT, 2, 512>;
            default: return nullptr;
        }
    }
    if (fmt != NN_FMT_SELL) return nullptr;
    if (tpb == 512) {
        switch (cgv) {
            case 1: return k_solve_grid<0, MODE_TRANSIENT, 1, 512>;
            case 2: return k_solve_grid<0, MODE_TRANSIENT, 2, 512>;
            default: return nullptr;
        }
    }
    if (tpb != 256) return nullptr;
    switch (cgv) {
        case 0: return k_solve_grid<0, MODE_TRANSIENT, 0, 256>;
        case 1: return k_solve_grid<0, MODE_TRANSIENT, 1, 256>;
        case 2: return k_solve_grid<0, MODE_TRANSIENT, 2, 256>;
        case 3: return k_solve_grid<0, MODE_TRANSIENT, 3, 256>;
        default: return nullptr;
    }
}

}  // namespace nnqp
