// Device-side execution "teams" for the persistent solver kernels.
//
// A team is the set of thread blocks that cooperate on one QP:
//   GridTeam  - every block of a cooperative launch (one large problem);
//               synchronised by a grid barrier whose waits are bounded in
//               time and end with an error flag instead of hanging;
//   BlockTeam - a single thread block (one small problem of a batch);
//               synchronised by __syncthreads.
// Reductions are deterministic: warp shuffle tree -> fixed block order ->
// (grid) fixed order over per-block partials, so every block of a grid
// team obtains bit-identical scalars and takes identical branches.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nnqp {

constexpr int kMaxRed = 24;       // doubles per reduction call (at most)
constexpr int kMaxWarps = 32;

struct GridBarrier {
    unsigned long long count;     // arrivals since launch (never reset)
    int error;                    // 0 = fine, else an nn_status code
    int where;                    // diagnostic: id of the wait that gave up
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Shared scratch used by the reductions of one block.
struct RedSmem {
    double warp[kMaxWarps][kMaxRed];
    double bcast[kMaxRed];
    int flag;
};

// Sum of v over the block; the result (taken from lane 0 of warp 0, so it
// is one fixed summation order) is returned in v on every thread.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], RedSmem &sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sm.warp[warp][k] = v[k];
    __syncthreads();
    // warp w sums the entries k = w, w + nw, ... (each in one fixed order)
    for (int k = warp; k < K; k += nw) {
        double t = lane < nw ? sm.warp[lane][k] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sm.bcast[k] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = sm.bcast[k];
    __syncthreads();
}

struct BlockTeam {
    RedSmem *sm;
    __device__ __forceinline__ bool sync() {
        __syncthreads();
        return true;
    }
    template <int K>
    __device__ __forceinline__ bool reduce(double (&v)[K]) {
        block_sum<K>(v, *sm);
        return true;
    }
    __device__ __forceinline__ bool ok() const { return true; }
};

struct GridTeam {
    GridBarrier *bar;
    double *partials;             // [2][kMaxRed][nblocks]
    int nblocks;
    unsigned long long timeout_ns;
    int slot;
    int wait_id;
    RedSmem *sm;

    // Grid-wide barrier.  Every block knows how many barriers it has passed
    // (wait_id), so the k-th barrier is complete once the arrival counter
    // reaches k * nblocks.  Thread 0 of each block arrives with a release-add
    // (its block's writes become visible first) and polls the counter with
    // acquire loads, for at most timeout_ns; a wait that runs out sets the
    // error word, and a block that sees the error word set leaves as well.
    __device__ bool sync() {
        __syncthreads();
        ++wait_id;
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned long long target = (unsigned long long)wait_id * (unsigned long long)nblocks;
            red_release_add_u64(&bar->count, 1ULL);
            unsigned spins = 0;
            unsigned long long t0 = 0;
            while (ld_acquire_u64(&bar->count) < target) {
                ++spins;
                if ((spins & 63u) == 0) {
                    if (ld_relaxed_i32(&bar->error)) {
                        ok = 0;
                        break;
                    }
                    const unsigned long long now = global_ns();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > timeout_ns) {
                        if (atomicCAS(&bar->error, 0, 7 /* NN_ERR_TIMEOUT */) == 0) bar->where = wait_id;
                        ok = 0;
                        break;
                    }
                }
                if (spins > 256) __nanosleep(32);
            }
            sm->flag = ok;
        }
        __syncthreads();
        return sm->flag != 0;
    }

    template <int K>
    __device__ bool reduce(double (&v)[K]) {
        block_sum<K>(v, *sm);
        slot ^= 1;
        double *P = partials + (size_t)slot * kMaxRed * nblocks;
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < K; ++k) P[(size_t)k * nblocks + blockIdx.x] = v[k];
        if (!sync()) return false;
        // warp w sums the per-block partials of entries k = w, w + nw, ...;
        // the loads of different entries are in flight together
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int k = warp; k < K; k += nw) {
            double t = 0.0;
            for (int b = lane; b < nblocks; b += 32) t += __ldcg(P + (size_t)k * nblocks + b);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) sm->bcast[k] = t;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = sm->bcast[k];
        __syncthreads();
        return true;
    }
};

// The CTAs of one thread-block cluster (all co-scheduled by the hardware).
// Barriers are the hardware cluster barrier; a reduction writes each CTA's
// block sum to its own shared memory, and after the cluster barrier every
// CTA reads all of them through distributed shared memory in rank order, so
// all CTAs obtain the same bits.  Two exchange slots alternate: a CTA can
// only overwrite slot s after every CTA has passed the barrier that follows
// its last read of s.
struct ClusterTeam {
    RedSmem *sm;
    double *xch;                  // this CTA's [2][kMaxRed] exchange buffer (shared memory)
    unsigned rank, size;
    int slot;

    __device__ __forceinline__ static void cluster_barrier() {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                         : "memory");
    }
    __device__ __forceinline__ bool sync() {
        cluster_barrier();
        return true;
    }
    template <int K>
    __device__ bool reduce(double (&v)[K]) {
        block_sum<K>(v, *sm);
        slot ^= 1;
        double *mine = xch + slot * kMaxRed;
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < K; ++k) mine[k] = v[k];
        cluster_barrier();
        if (threadIdx.x < K) {
            const int k = threadIdx.x;
            const uint32_t local = (uint32_t)__cvta_generic_to_shared(mine + k);
            double t = 0.0;
            for (unsigned r = 0; r < size; ++r) {
                uint32_t remote;
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
                double x;
                asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(x) : "r"(remote) : "memory");
                t += x;
            }
            sm->bcast[k] = t;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = sm->bcast[k];
        __syncthreads();
        return true;
    }
};

// Rows owned by a block: the SELL slices [s0, s1); warp w of the block
// takes slices s0 + w, s0 + w + nwarps, ...; lane l takes row 32 s + l.
struct Rows {
    int64_t s0, s1, n;
    template <class F>
    __device__ __forceinline__ void each(F &&f) const {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int64_t s = s0 + (threadIdx.x >> 5); s < s1; s += nw) {
            int64_t i = s * 32 + lane;
            if (i < n) f(i);
        }
    }
};

__host__ __device__ __forceinline__ Rows rows_of_block(int64_t n, int64_t nslices, int block, int nblocks) {
    int64_t per = (nslices + nblocks - 1) / nblocks;
    int64_t s0 = per * block, s1 = s0 + per;
    if (s0 > nslices) s0 = nslices;
    if (s1 > nslices) s1 = nslices;
    return Rows{s0, s1, n};
}

}  // namespace nnqp
