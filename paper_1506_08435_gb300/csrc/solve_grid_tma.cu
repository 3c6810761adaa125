// Instantiations of the persistent solve kernel whose FP32 inner products
// stream the operator through shared memory by bulk copies (mixed modes,
// textbook CG form; 512-thread blocks, one per SM, or 256-thread blocks).
#include "grid.cuh"

namespace nnqp {

GridKernel grid_kernel_tma(int mode, int cgv, int tpb) {
    if (cgv != 0) return nullptr;
    if (mode == MODE_MIXED) {
        if (tpb == 512) return k_solve_grid<3, MODE_MIXED, 0, 512>;
        if (tpb == 256) return k_solve_grid<3, MODE_MIXED, 0, 256>;
    }
    if (mode == MODE_MIXED_TR && tpb == 256) return k_solve_grid<3, MODE_MIXED_TR, 0, 256>;
    return nullptr;
}

}  // namespace nnqp
