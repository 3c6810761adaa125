// Instantiations of the batched-solve kernels, FP64.
#include "batch.cuh"

namespace nnqp {

namespace {
template <int CGV>
BatchKernel by_shape(int tpb, int cluster) {
    if (cluster > 1) return tpb == 256 ? k_batch_cluster<256, 0, CGV> : nullptr;
    switch (tpb) {
        case 128: return k_batch<128, 0, CGV>;
        case 256: return k_batch<256, 0, CGV>;
        case 512: return k_batch<512, 0, CGV>;
        default: return nullptr;
    }
}
}  // namespace

BatchKernel batch_kernel_fp64(int tpb, int cluster, int cgv) {
    switch (cgv) {
        case 0: return by_shape<0>(tpb, cluster);
        case 1: return by_shape<1>(tpb, cluster);
        case 2: return by_shape<2>(tpb, cluster);
        default: return nullptr;
    }
}

}  // namespace nnqp
