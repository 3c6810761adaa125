// Instantiations of the batched-solve kernels, mixed precision.
#include "batch.cuh"

namespace nnqp {

namespace {
template <int CGV>
BatchKernel by_shape(int tpb, int cluster) {
    if (cluster > 1) return tpb == 256 ? k_batch_cluster<256, 1, CGV> : nullptr;
    switch (tpb) {
        case 128: return k_batch<128, 1, CGV>;
        case 256: return k_batch<256, 1, CGV>;
        case 512: return k_batch<512, 1, CGV>;
        default: return nullptr;
    }
}
}  // namespace

BatchKernel batch_kernel_mixed(int tpb, int cluster, int cgv) {
    switch (cgv) {
        case 0: return by_shape<0>(tpb, cluster);
        case 1: return by_shape<1>(tpb, cluster);
        case 2: return by_shape<2>(tpb, cluster);
        default: return nullptr;
    }
}

}  // namespace nnqp
