// Instantiation of the persistent solve kernel whose FP32 inner products
// stream the operator through shared memory by bulk copies (steady mixed
// mode, textbook CG form, one 768-thread block per SM).
#include "grid.cuh"

namespace nnqp {

GridKernel grid_kernel_tma(int mode, int cgv, int tpb) {
    if (cgv == 0 && mode == MODE_MIXED && tpb == 768) return k_solve_grid<3, MODE_MIXED, 0, 768>;
    return nullptr;
}

}  // namespace nnqp
