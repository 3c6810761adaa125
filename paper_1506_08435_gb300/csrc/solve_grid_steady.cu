// Instantiations of the persistent solve kernel for mode MODE_STEADY.
#include "grid.cuh"

namespace nnqp {

GridKernel grid_kernel_steady(int fmt, int cgv) {
    if (fmt == NN_FMT_CSR) {
        switch (cgv) {
            case 0: return k_solve_grid<1, MODE_STEADY, 0>;
            case 1: return k_solve_grid<1, MODE_STEADY, 1>;
            default: return nullptr;
        }
    }
    switch (cgv) {
        case 0: return k_solve_grid<0, MODE_STEADY, 0>;
        case 1: return k_solve_grid<0, MODE_STEADY, 1>;
        case 2: return k_solve_grid<0, MODE_STEADY, 2>;
        default: return nullptr;
    }
}

}  // namespace nnqp
