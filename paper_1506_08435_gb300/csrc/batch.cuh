// Kernels of the batched solve: many independent QPs of uneven size in ONE
// persistent launch.  An instance is solved by one thread block (block
// barriers and reductions) or by one thread-block cluster (hardware cluster
// barrier, reductions through distributed shared memory); blocks / clusters
// take the next instance (largest first) from a device work counter, so no
// block ever waits on a block of another instance.  The solver is the same
// GPCG (and mixed-precision refinement) code as the single-system path.
// Instantiated per precision in batch_fp64.cu / batch_mixed.cu.
#pragma once
#include <stdint.h>
#include "internal.h"
#include "gpcg.cuh"
#include "refine.cuh"

namespace nnqp {


struct BatchInst {
    int64_t n, N, nslices;
    const int64_t *sptr;
    const int32_t *col;
    const double *val;
    const double *diag;
    const double *dinv64;
    const float *val32;
    const float *rsum32;
    const float *dinv32;
    const double *b0;
    const int32_t *free_node;
    const uint8_t *dmask;
    const double *dval;
    double lo, hi, den;
    double *c;          // full node vector: warm start in, solution out
    double *w64;        // 11 n doubles
    float *w32;         // 13 n floats (mixed)
    uint8_t *fm;        // n bytes: face mask of the CG phases
};

constexpr int kBatchCounters = 9;

// Solves instance `id` with team T; this CTA owns the rows R of it.
template <int MIXED, int CGV, class Team>
__device__ void solve_instance(Team &T, const Rows &R, const BatchInst &I, int id, unsigned rank, unsigned size,
                               const GpcgCtl &ctl, double rtol, double inner_rtol, int max_ref, int64_t *counters,
                               double *scalars) {
    const int64_t n = I.n;
    double *x = I.w64;
    R.each([&](int64_t i) { x[i] = I.c[I.free_node[i]]; });
    if (!T.sync()) return;
    const SellF64 A{n, I.nslices, I.sptr, I.col, I.val, I.diag};
    int64_t cnt[kBatchCounters] = {0};
    double gp2 = 0.0;
    int status;
    if (MIXED) {
        float *w = I.w32;
        GpcgVecs<float> v{w, w + n, w + 2 * n, w + 3 * n, w + 4 * n, w + 5 * n, w + 6 * n, w + 7 * n, w + 8 * n,
                          w + 9 * n, I.dinv32, I.fm, w + 12 * n};
        const SellF32Diff A32{n, I.nslices, I.sptr, I.col, I.val32, I.rsum32};
        double *w6 = I.w64;
        GpcgVecs<double> v64{x, w6 + n, w6 + 2 * n, w6 + 3 * n, w6 + 4 * n, w6 + 5 * n, w6 + 6 * n,
                             w6 + 7 * n, w6 + 8 * n, I.b0, I.dinv64, I.fm, w6 + 10 * n};
        MixedStats ms;
        status = mixed_solve<CGV, CGV, true>(T, R, A, A32, I.lo, I.hi, I.b0, x, v, w + 9 * n, w + 10 * n, w + 11 * n, v64,
                                rtol * I.den, inner_rtol, max_ref, ctl.max_spmv, batch_inner_product_cap(n), ctl, ctl, ms);
        cnt[1] = ms.spmv64;
        cnt[2] = ms.spmv32;
        cnt[3] = ms.cg;
        cnt[4] = ms.phases;
        cnt[5] = ms.refinements;
        cnt[6] = ms.vec64;
        cnt[7] = ms.vec32;
        cnt[8] = ms.fallback;
        gp2 = ms.gp2;
    } else {
        double *w = I.w64;
        GpcgVecs<double> v{w, w + n, w + 2 * n, w + 3 * n, w + 4 * n, w + 5 * n, w + 6 * n, w + 7 * n,
                           w + 8 * n, I.b0, I.dinv64, I.fm, w + 10 * n};
        GpcgCtl c = ctl;
        c.tol = rtol * I.den;
        c.face_tol = 0.5 * c.tol;
        GpcgStats gs;
        status = gpcg_solve<Team, SellF64, double, CGV>(T, R, A, Bounds<double>{I.lo, I.hi, nullptr, nullptr}, v, c, gs);
        x = v.x;
        cnt[1] = gs.spmv;
        cnt[3] = gs.cg;
        cnt[4] = gs.phases;
        cnt[6] = gs.vec;
        gp2 = gs.gp2;
    }
    R.each([&](int64_t i) { I.c[I.free_node[i]] = x[i]; });
    for (int64_t v = (int64_t)rank * blockDim.x + threadIdx.x; v < I.N; v += (int64_t)size * blockDim.x)
        if (I.dmask[v]) I.c[v] = I.dval[v];
    if (rank == 0 && threadIdx.x == 0) {
        cnt[0] = status;
        for (int k = 0; k < kBatchCounters; ++k) counters[(int64_t)id * kBatchCounters + k] = cnt[k];
        scalars[2 * id] = gp2;
        scalars[2 * id + 1] = I.den;
    }
}

// One thread block per instance.
template <int TPB, int MIXED, int CGV>
__global__ void __launch_bounds__(TPB) k_batch(const BatchInst *__restrict__ insts, const int *__restrict__ order,
                                               int count, unsigned *next, GpcgCtl ctl, double rtol,
                                               double inner_rtol, int max_ref, int64_t *counters, double *scalars) {
    __shared__ RedSmem sm;
    __shared__ int s_q;
    BlockTeam T{&sm};
    for (;;) {
        if (threadIdx.x == 0) s_q = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= count) return;
        const int id = order[q];
        const BatchInst I = insts[id];
        solve_instance<MIXED, CGV>(T, Rows{0, I.nslices, I.n}, I, id, 0, 1, ctl, rtol, inner_rtol, max_ref, counters,
                              scalars);
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// One thread-block cluster per instance: the instance's slices are split
// over the cluster's CTAs (one per SM), barriers are the hardware cluster
// barrier, reductions go through distributed shared memory.
template <int TPB, int MIXED, int CGV>
// CTAs per SM: 3 for FP64 (more clusters in flight hide more latency;
// measured 2.08 -> 1.94 s on the 512-instance batch), 2 for mixed precision,
// whose inner solves would spill at the 3-CTA register budget
__global__ void __launch_bounds__(TPB, MIXED ? 2 : 3) k_batch_cluster(const BatchInst *__restrict__ insts,
                                                       const int *__restrict__ order, int count, unsigned *next,
                                                       GpcgCtl ctl, double rtol, double inner_rtol, int max_ref,
                                                       int64_t *counters, double *scalars) {
    __shared__ RedSmem sm;
    __shared__ double xch[2 * kMaxCluster * kMaxRed];
    __shared__ int s_q;
    const unsigned rank = cluster_rank(), size = cluster_size();
    ClusterTeam T{&sm, xch, rank, size, 0};
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_q = (int)atomicAdd(next, 1u);
        T.sync();
        // every CTA reads the instance index taken by CTA 0
        __shared__ int s_q0;
        if (threadIdx.x == 0) {
            const uint32_t local = (uint32_t)__cvta_generic_to_shared(&s_q);
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(0u));
            int q;
            asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(q) : "r"(remote) : "memory");
            s_q0 = q;
        }
        T.sync();
        const int q = s_q0;
        if (q >= count) break;
        const int id = order[q];
        const BatchInst I = insts[id];
        solve_instance<MIXED, CGV>(T, rows_of_block(I.n, I.nslices, (int)rank, (int)size), I, id, rank, size, ctl, rtol,
                              inner_rtol, max_ref, counters, scalars);
        T.sync();
    }
    T.sync();   // no CTA leaves while another may still read its shared memory
}

using BatchKernel = void (*)(const BatchInst *, const int *, int, unsigned *, GpcgCtl, double, double, int,
                             int64_t *, double *);

// Kernel for threads per block tpb (128, 256, 512; clusters use 256), CTAs per
// instance cluster (1 = one block) and CG variant cgv (0, 1, 2); nullptr if
// that combination is not built.
BatchKernel batch_kernel_fp64(int tpb, int cluster, int cgv);
BatchKernel batch_kernel_mixed(int tpb, int cluster, int cgv);

}  // namespace nnqp
