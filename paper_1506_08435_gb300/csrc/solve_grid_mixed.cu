// Instantiations of the persistent solve kernel for mode MODE_MIXED.
#include "grid.cuh"

namespace nnqp {

GridKernel grid_kernel_mixed(int fmt, int cgv) {
    if (fmt != NN_FMT_SELL) return nullptr;
    switch (cgv) {
        case 0: return k_solve_grid<0, MODE_MIXED, 0>;
        case 1: return k_solve_grid<0, MODE_MIXED, 1>;
        case 2: return k_solve_grid<0, MODE_MIXED, 2>;
        default: return nullptr;
    }
}

}  // namespace nnqp
