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

constexpr int kMaxRed = 40;       // doubles per reduction call (at most)
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
    double sc[16];                // results of scalar steps done by warp 0
    int flag;
};

// Warp stage of a block sum: K values per lane are summed over the warp's 32
// lanes with a transposing butterfly.  While a lane holds more than one
// value, each level sends half of them to the partner lane (offset o) and
// keeps the other half, so every FP64 add is useful (K/2 + K/4 + ... adds
// instead of 5 K).  On GB300 every FP64 warp instruction occupies the SM's
// narrow FP64 pipe for many cycles whatever the active mask, so the count of
// FP64 instructions, not their latency, is what a reduction costs.  P is K
// rounded up to a power of two; on return lane l holds the warp totals of
// indices ((l >> (5 - LT)) * CF + j), j < CF, with LT the number of
// transposing levels and CF = P >> LT values left per lane.  The order of
// the additions is fixed, so every warp and block sums alike.
template <int K>
struct WarpSumShape {
    static constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : K <= 32 ? 32 : 64;
    static constexpr int LOGP = P == 1 ? 0 : P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : P == 32 ? 5 : 6;
    static constexpr int LT = LOGP < 5 ? LOGP : 5;
    static constexpr int CF = P >> LT;
};

template <int K>
__device__ __forceinline__ void warp_sum_transposed(const double (&in)[K], double (&out)[WarpSumShape<K>::CF]) {
    using S = WarpSumShape<K>;
    static_assert(K <= 64, "at most 64 values per reduction");
    double v[S::P];
#pragma unroll
    for (int k = 0; k < S::P; ++k) v[k] = k < K ? in[k] : 0.0;
    const int lane = threadIdx.x & 31;
    int cnt = S::P;
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
        const int o = 16 >> lvl;
        if (lvl < S::LT) {
            const bool up = (lane & o) != 0;
            const int h = S::P >> (lvl + 1);
#pragma unroll
            for (int j = 0; j < S::P / 2; ++j)
                if (j < h) {
                    const double keep = up ? v[j + h] : v[j];
                    const double send = up ? v[j] : v[j + h];
                    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            cnt = h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
    (void)cnt;
#pragma unroll
    for (int j = 0; j < S::CF; ++j) out[j] = v[j];
}

// Writes the warp totals of warp_sum_transposed to sm.warp[warp][OFF + k].
template <int K, int OFF = 0>
__device__ __forceinline__ void warp_totals_to_smem(const double (&t)[WarpSumShape<K>::CF], RedSmem &sm) {
    using S = WarpSumShape<K>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int sh = 5 - S::LT;
    if ((lane & ((1 << sh) - 1)) == 0) {
        const int base = (lane >> sh) * S::CF;
#pragma unroll
        for (int j = 0; j < S::CF; ++j)
            if (base + j < K) sm.warp[warp][OFF + base + j] = t[j];
    }
}

// Warp stage of a block sum: totals of v over the warp's lanes to
// sm.warp[warp][k].  More than 32 values are summed as 32 + the rest, which
// pads less than rounding K up to 64 (each padded value costs FP64 adds).
template <int K>
__device__ __forceinline__ void warp_stage(const double (&v)[K], RedSmem &sm) {
    if constexpr (K <= 32) {
        double t[WarpSumShape<K>::CF];
        warp_sum_transposed<K>(v, t);
        warp_totals_to_smem<K>(t, sm);
    } else {
        double a[32], b[K - 32];
#pragma unroll
        for (int k = 0; k < 32; ++k) a[k] = v[k];
#pragma unroll
        for (int k = 32; k < K; ++k) b[k - 32] = v[k];
        double ta[WarpSumShape<32>::CF], tb[WarpSumShape<K - 32>::CF];
        warp_sum_transposed<32>(a, ta);
        warp_sum_transposed<K - 32>(b, tb);
        warp_totals_to_smem<32, 0>(ta, sm);
        warp_totals_to_smem<K - 32, 32>(tb, sm);
    }
}

// Cross-warp stage: the per-warp totals sm.warp[w][k] (w < nw) are summed in
// a fixed butterfly order by warp 0 and stored to sm.bcast[k].  Lanes are
// packed (k, w) so that one FP64 instruction serves 32 / nw entries.
// A block whose warp count is not a power of two (24 warps of 768 threads)
// is summed as the next power of two with zero totals for the missing warps.
template <int K>
__device__ __forceinline__ void warp0_sum_warps(RedSmem &sm) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int np = 1;
    while (np < nw) np <<= 1;
    const int per = 32 / np;                  // entries per warp instruction
    const int k_in = lane / np, w = lane % np;
    for (int k0 = 0; k0 < K; k0 += per) {
        const int k = k0 + k_in;
        double t = (k < K && k_in < per && w < nw) ? sm.warp[w][k] : 0.0;
        for (int o = np >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (w == 0 && k < K && k_in < per) sm.bcast[k] = t;
    }
}

// Sum of v over the block in a fixed order; the result is returned in v on
// every thread.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], RedSmem &sm) {
    warp_stage<K>(v, sm);
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) warp0_sum_warps<K>(sm);
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
    // Arrival and bounded wait of the barrier numbered wait_id, by thread 0
    // of the block (after the block's writes it must publish); 1 = passed.
    __device__ int arrive_and_wait() {
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
        return ok;
    }

    __device__ bool sync() {
        __syncthreads();
        ++wait_id;
        if (threadIdx.x == 0) sm->flag = arrive_and_wait();
        __syncthreads();
        return sm->flag != 0;
    }

    template <int K>
    __device__ bool reduce(double (&v)[K]) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        warp_stage<K>(v, *sm);
        __syncthreads();
        slot ^= 1;
        ++wait_id;
        double *P = partials + (size_t)slot * kMaxRed * nblocks;
        // warp 0 sums the warps, publishes the block's partials and passes
        // the grid barrier; the other warps wait for it at one block barrier
        if (warp == 0) {
            warp0_sum_warps<K>(*sm);
            __syncwarp();
            for (int k = lane; k < K; k += 32) P[(size_t)k * nblocks + blockIdx.x] = sm->bcast[k];
            __syncwarp();
            if (lane == 0) sm->flag = arrive_and_wait();
        }
        __syncthreads();
        if (sm->flag == 0) return false;
        if (K <= nw) {
            // warp k sums the per-block partials of entry k; the loads of
            // different entries are in flight together
            for (int k = warp; k < K; k += nw) {
                // up to 8 partials per lane per round, all loads issued before
                // the adds (one L2 round trip per 256 blocks)
                const double *Pk = P + (size_t)k * nblocks;
                double u = 0.0;
                for (int b0 = 0; b0 < nblocks; b0 += 256) {
                    double w[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int b = b0 + lane + 32 * j;
                        w[j] = b < nblocks ? __ldcg(Pk + b) : 0.0;
                    }
                    u += ((w[0] + w[1]) + (w[2] + w[3])) + ((w[4] + w[5]) + (w[6] + w[7]));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
                if (lane == 0) sm->bcast[k] = u;
            }
        } else {
            // wide reductions: CH threads per entry, each summing every CH-th
            // partial in four independent chains (short FP64 dependency
            // chains), then one thread per entry adds the CH chunk sums in order
            const int CH = (int)blockDim.x / K < kMaxWarps ? (int)blockDim.x / K : kMaxWarps;
            const int t = threadIdx.x;
            if (t < K * CH) {
                const int k = t / CH, c = t - k * CH;
                const double *Pk = P + (size_t)k * nblocks;
                double u = 0.0;
                for (int j0 = 0; c + j0 * CH < nblocks; j0 += 16) {
                    double w[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int b = c + (j0 + j) * CH;
                        w[j] = b < nblocks ? __ldcg(Pk + b) : 0.0;
                    }
#pragma unroll
                    for (int h = 8; h > 0; h >>= 1)
#pragma unroll
                        for (int j = 0; j < h; ++j) w[j] += w[j + h];
                    u += w[0];
                }
                sm->warp[c][k] = u;
            }
            __syncthreads();
            if (t < K) {
                double u = 0.0;
                for (int c = 0; c < CH; ++c) u += sm->warp[c][t];
                sm->bcast[t] = u;
            }
        }
        __syncthreads();
        // (no barrier after the copy: the next writer of bcast or flag is
        // behind the next reduction's or barrier's first block barrier)
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = sm->bcast[k];
        return true;
    }
};

constexpr int kMaxCluster = 16;

// The CTAs of one thread-block cluster (all co-scheduled by the hardware).
// Barriers are the hardware cluster barrier.  A reduction pushes each CTA's
// block totals into every CTA's exchange buffer (remote shared-memory
// stores, no round trip), and after the cluster barrier every CTA sums the
// buffer's rows in rank order, so all CTAs obtain the same bits.  Two
// exchange slots alternate: a CTA can only overwrite slot s after every CTA
// has passed the barrier that follows its last read of s.
struct ClusterTeam {
    RedSmem *sm;
    double *xch;                  // this CTA's [2][kMaxCluster][kMaxRed] exchange buffer (shared memory)
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
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        warp_stage<K>(v, *sm);
        __syncthreads();
        slot ^= 1;
        double *buf = xch + (size_t)slot * kMaxCluster * kMaxRed;
        if (warp == 0) {
            warp0_sum_warps<K>(*sm);
            __syncwarp();
            for (int q = lane; q < (int)size * K; q += 32) {
                const unsigned r = (unsigned)(q / K);
                const int k = q - (int)r * K;
                const uint32_t local = (uint32_t)__cvta_generic_to_shared(buf + rank * kMaxRed + k);
                uint32_t remote;
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
                asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(sm->bcast[k]) : "memory");
            }
        }
        cluster_barrier();
        // rows of the exchange buffer summed in rank order (butterfly over
        // the cluster's lanes; size is a power of two)
        for (int k = warp; k < K; k += nw) {
            double u = lane < (int)size ? buf[lane * kMaxRed + k] : 0.0;
            for (int o = (int)size >> 1; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
            if (lane == 0) sm->bcast[k] = u;
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
    // Element-wise pass over the block's rows with W consecutive rows per
    // thread: f(i, cnt) handles rows i .. i + cnt - 1 (cnt = W except at the
    // end of the system), so that it can move them with one vector access
    // per array.  Each access then carries W times the bytes of a row-wise
    // pass, which keeps more of a streaming pass in flight per warp.  (Only
    // for passes with a barrier on both sides: the rows a thread touches
    // differ from the row-per-lane passes.)
    template <int W, class F>
    __device__ __forceinline__ void each_chunk(F &&f) const {
        const int64_t r0 = s0 * 32, r1 = s1 * 32 < n ? s1 * 32 : n;
        for (int64_t i = r0 + (int64_t)threadIdx.x * W; i < r1; i += (int64_t)blockDim.x * W)
            f(i, r1 - i < W ? (int)(r1 - i) : W);
    }
    // The same pass with an L2 prefetch of the warp's next slice of the NP
    // vectors it reads (esize bytes per entry), issued by one lane per
    // 128-byte line: on large systems a warp then has the next rows' loads in
    // flight while it works on these (streaming passes are bound by memory
    // parallelism).  Slices that end past row n are not prefetched.
    template <int NP, class F>
    __device__ __forceinline__ void each_pf(const void *const (&pf)[NP], int esize, bool on, F &&f) const {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const int lines = esize >> 2;   // 32 rows x esize bytes / 128-byte lines
        for (int64_t s = s0 + (threadIdx.x >> 5); s < s1; s += nw) {
            const int64_t nx = s + nw;
            if (on && nx < s1 && (nx + 1) * 32 <= n && lane < NP * lines) {
                const int j = lane / lines, l = lane - j * lines;
                const char *p = (const char *)pf[j] + nx * 32 * esize + 128 * l;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
            }
            int64_t i = s * 32 + lane;
            if (i < n) f(i);
        }
    }
};

// W consecutive entries of a vector of V moved by one vector access (16 bytes).
template <typename V>
struct Pack;
template <>
struct Pack<float> {
    static constexpr int W = 4;
    using T = float4;
};
template <>
struct Pack<double> {
    static constexpr int W = 2;
    using T = double2;
};

template <typename V>
__device__ __forceinline__ void ld_pack(const V *p, V (&o)[Pack<V>::W]) {
    const typename Pack<V>::T t = *reinterpret_cast<const typename Pack<V>::T *>(p);
    const V *e = reinterpret_cast<const V *>(&t);
#pragma unroll
    for (int k = 0; k < Pack<V>::W; ++k) o[k] = e[k];
}

template <typename V>
__device__ __forceinline__ void st_pack(V *p, const V (&o)[Pack<V>::W]) {
    typename Pack<V>::T t;
    V *e = reinterpret_cast<V *>(&t);
#pragma unroll
    for (int k = 0; k < Pack<V>::W; ++k) e[k] = o[k];
    *reinterpret_cast<typename Pack<V>::T *>(p) = t;
}

// st_pack with an L2 evict-last policy: for vectors that the next pass
// reads again (the search direction the product gathers), so that the
// operator streaming past with evict-first loads does not push them out.
__device__ __forceinline__ void st_pack_keep(float *p, const float (&o)[4], uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(o[0]), "f"(o[1]),
                 "f"(o[2]), "f"(o[3]), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_pack_keep(double *p, const double (&o)[2], uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(o[0]), "d"(o[1]), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// True if every pointer is 16-byte aligned (the packed passes need it; the
// rows of a block start at a multiple of 32).
template <int K>
__device__ __forceinline__ bool aligned16(const void *const (&p)[K]) {
    uintptr_t o = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) o |= reinterpret_cast<uintptr_t>(p[k]);
    return (o & 15) == 0;
}

__host__ __device__ __forceinline__ Rows rows_of_block(int64_t n, int64_t nslices, int block, int nblocks) {
    int64_t per = (nslices + nblocks - 1) / nblocks;
    int64_t s0 = per * block, s1 = s0 + per;
    if (s0 > nslices) s0 = nslices;
    if (s1 > nslices) s1 = nslices;
    return Rows{s0, s1, n};
}

}  // namespace nnqp
