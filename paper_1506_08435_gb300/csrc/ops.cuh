// Sparse operators y = A x on the free unknowns, each fused with a per-row
// epilogue epi(i, y_i) so that the consumer of the product (gradient,
// search direction, dot products) runs in the same pass over the rows.
//
// The product is the Hessian-vector product of the QP (the "MatMult" of the
// paper's cost model, Sec. 4, Table 2); the algorithmic traffic of one
// product is nnz*(s_val + 4) + 4(n+1) + s_x n + s_x n.
//
// SELL-32 layout with pair interleaving: in slice s (rows 32s..32s+31, width
// w_s even), entry k of row 32s+l lives at
//     sptr[s] + 64 (k/2) + 2 l + (k%2),
// so lane l reads entries (k, k+1) of its row with one vector load: 16 bytes
// for FP64 values, 8 bytes for column indices and FP32 values, and a warp
// reads 512 (256) contiguous bytes per load instruction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "team.cuh"
#include "tma.cuh"

namespace nnqp {

__host__ __device__ __forceinline__ int64_t sell_idx(int64_t base, int k, int lane) {
    return base + 64 * (int64_t)(k >> 1) + 2 * lane + (k & 1);
}

// Matrix loads.  An operator larger than about half of L2 streams through it
// once per product: its loads are marked evict-first (cache-streaming), so
// that the gathered vector stays in L2.  A smaller operator is reused from
// L2 by every product and is loaded normally.
// LOCAL operators hold a block's slices in shared memory (staged once per
// launch) and are read with ordinary loads.
template <bool LOCAL, typename T>
__device__ __forceinline__ T mat_load(const T *p, bool stream) {
    if constexpr (LOCAL)
        return *p;
    else
        return stream ? __ldcs(p) : __ldg(p);
}

// Asks L2 for the column and value bytes [b0, b1) of a slice ahead of use:
// every lane of the warp prefetches its share of the 128-byte lines, so a
// warp has the next slice's operator in flight while it works on this one.
__device__ __forceinline__ void prefetch_slice(const void *col, const void *val, int vbytes, int64_t b0, int64_t b1,
                                               int lane) {
    const char *c = (const char *)col + b0 * 4, *v = (const char *)val + b0 * vbytes;
    const int cl = (int)(((b1 - b0) * 4 + 127) >> 7), vl = (int)(((b1 - b0) * vbytes + 127) >> 7);
    for (int l = lane; l < cl; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(c + 128 * l));
    for (int l = lane; l < vl; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(v + 128 * l));
}

// SELL-32, FP64 values; off-diagonals in slices, diagonal separate:
//   y_i = d_i x_i + sum_k v_ik x_{c_ik}
// LOCAL: col/val hold only the entries [e0, ...) of the calling block's
// slices, in shared memory; entry e of the operator is col[e - e0].
template <bool LOCAL>
struct SellF64X {
    int64_t n, nslices;
    const int64_t *__restrict__ sptr;
    const int32_t *__restrict__ col;
    const double *__restrict__ val;
    const double *__restrict__ diag;
    bool stream = false;          // operator larger than L2: streaming loads + slice prefetch
    int64_t e0 = 0;               // first entry held by col/val (LOCAL)

    template <typename VX>
    __device__ __forceinline__ double row(int64_t s, int lane, int64_t base, int w, const VX *x) const {
        const int2 *c2 = reinterpret_cast<const int2 *>(col + (base - e0)) + lane;
        const double2 *v2 = reinterpret_cast<const double2 *>(val + (base - e0)) + lane;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        // 8 entries per step: every column/value load of the step is issued
        // before the gathers, and every gather before the FMAs, so a row's
        // loads are in flight together (the bound on large systems is memory
        // parallelism, not arithmetic)
        for (; k + 8 <= w; k += 8) {
            int2 c[4];
            double2 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                c[j] = mat_load<LOCAL>(c2 + 16 * (k + 2 * j), stream);
                v[j] = mat_load<LOCAL>(v2 + 16 * (k + 2 * j), stream);
            }
            double xv[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                xv[2 * j] = (double)x[c[j].x];
                xv[2 * j + 1] = (double)x[c[j].y];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                a0 = fma(v[j].x, xv[2 * j], a0);
                a1 = fma(v[j].y, xv[2 * j + 1], a1);
            }
        }
        for (; k + 4 <= w; k += 4) {
            const int2 ca = mat_load<LOCAL>(c2 + 16 * k, stream), cb = mat_load<LOCAL>(c2 + 16 * k + 32, stream);
            const double2 va = mat_load<LOCAL>(v2 + 16 * k, stream), vb = mat_load<LOCAL>(v2 + 16 * k + 32, stream);
            a0 = fma(va.x, (double)x[ca.x], a0);
            a1 = fma(va.y, (double)x[ca.y], a1);
            a0 = fma(vb.x, (double)x[cb.x], a0);
            a1 = fma(vb.y, (double)x[cb.y], a1);
        }
        if (k < w) {
            const int2 ca = mat_load<LOCAL>(c2 + 16 * k, stream);
            const double2 va = mat_load<LOCAL>(v2 + 16 * k, stream);
            a0 = fma(va.x, (double)x[ca.x], a0);
            a1 = fma(va.y, (double)x[ca.y], a1);
        }
        return a0 + a1;
    }

    template <class Epi>
    __device__ __forceinline__ void apply(const Rows &R, const double *x, Epi &&epi) const {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int64_t s = R.s0 + (threadIdx.x >> 5); s < R.s1; s += nw) {
            const int64_t base = __ldg(sptr + s);
            const int w = (int)((__ldg(sptr + s + 1) - base) >> 5);
            if (!LOCAL && stream && s + nw < R.s1) prefetch_slice(col, val, 8, __ldg(sptr + s + nw), __ldg(sptr + s + nw + 1), lane);
            const int64_t i = s * 32 + lane;
            const double acc = row(s, lane, base, w, x);
            if (i < n) epi(i, fma(__ldg(diag + i), x[i], acc));
        }
    }

    // (A x)_i for one row (used outside the fused passes).
    __device__ __forceinline__ double row_product(int64_t i, const double *x) const {
        const int64_t s = i >> 5;
        const int lane = (int)(i & 31);
        const int64_t base = sptr[s];
        const int w = (int)((sptr[s + 1] - base) >> 5);
        double acc = 0.0;
        for (int k = 0; k < w; ++k)
            acc = fma(val[sell_idx(base - e0, k, lane)], x[col[sell_idx(base - e0, k, lane)]], acc);
        return fma(diag[i], x[i], acc);
    }
};

using SellF64 = SellF64X<false>;
using SellF64Local = SellF64X<true>;

// SELL-32, FP32 values, FP32 vectors, in difference form:
//   y_i = s_i x_i + sum_k v_ik (x_{c_ik} - x_i),   s_i = sum_j A_ij (row sum)
// The implied diagonal is s_i - sum_k v_ik, so rounding the off-diagonals to
// FP32 perturbs A by a matrix with zero row sums, and rounding in the
// products scales with |x_j - x_i| instead of |x_j|.
template <bool LOCAL>
struct SellF32DiffX {
    int64_t n, nslices;
    const int64_t *__restrict__ sptr;
    const int32_t *__restrict__ col;
    const float *__restrict__ val;
    const float *__restrict__ rsum;
    bool stream = false;          // operator larger than L2: streaming loads + slice prefetch
    int64_t e0 = 0;               // first entry held by col/val (LOCAL)

    template <class Epi>
    __device__ __forceinline__ void apply(const Rows &R, const float *x, Epi &&epi) const {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int64_t s = R.s0 + (threadIdx.x >> 5); s < R.s1; s += nw) {
            const int64_t base = __ldg(sptr + s);
            const int w = (int)((__ldg(sptr + s + 1) - base) >> 5);
            if (!LOCAL && stream && s + nw < R.s1) prefetch_slice(col, val, 4, __ldg(sptr + s + nw), __ldg(sptr + s + nw + 1), lane);
            const int64_t i = s * 32 + lane;
            const float xi = i < n ? x[i] : 0.0f;
            const int2 *c2 = reinterpret_cast<const int2 *>(col + (base - e0)) + lane;
            const float2 *v2 = reinterpret_cast<const float2 *>(val + (base - e0)) + lane;
            float a0 = 0.0f, a1 = 0.0f;
            int k = 0;
            for (; k + 8 <= w; k += 8) {   // loads of 8 entries in flight together
                int2 c[4];
                float2 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    c[j] = mat_load<LOCAL>(c2 + 16 * (k + 2 * j), stream);
                    v[j] = mat_load<LOCAL>(v2 + 16 * (k + 2 * j), stream);
                }
                float xv[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    xv[2 * j] = x[c[j].x];
                    xv[2 * j + 1] = x[c[j].y];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    a0 = fmaf(v[j].x, xv[2 * j] - xi, a0);
                    a1 = fmaf(v[j].y, xv[2 * j + 1] - xi, a1);
                }
            }
            for (; k + 4 <= w; k += 4) {
                const int2 ca = mat_load<LOCAL>(c2 + 16 * k, stream), cb = mat_load<LOCAL>(c2 + 16 * k + 32, stream);
                const float2 va = mat_load<LOCAL>(v2 + 16 * k, stream), vb = mat_load<LOCAL>(v2 + 16 * k + 32, stream);
                a0 = fmaf(va.x, x[ca.x] - xi, a0);
                a1 = fmaf(va.y, x[ca.y] - xi, a1);
                a0 = fmaf(vb.x, x[cb.x] - xi, a0);
                a1 = fmaf(vb.y, x[cb.y] - xi, a1);
            }
            if (k < w) {
                const int2 ca = mat_load<LOCAL>(c2 + 16 * k, stream);
                const float2 va = mat_load<LOCAL>(v2 + 16 * k, stream);
                a0 = fmaf(va.x, x[ca.x] - xi, a0);
                a1 = fmaf(va.y, x[ca.y] - xi, a1);
            }
            if (i < n) epi(i, fmaf(__ldg(rsum + i), xi, a0 + a1));
        }
    }
};

using SellF32Diff = SellF32DiffX<false>;
using SellF32DiffLocal = SellF32DiffX<true>;

// The FP32 difference-form operator of SellF32DiffX, streamed from global
// memory through shared memory by bulk asynchronous copies (TMA) for
// operators far larger than L2.  Each warp owns a ring of D slots in the
// block's dynamic shared memory; its lane 0 copies the columns and values
// of the warp's slice s + (D-1) nw (contiguous in the SELL layout) into the
// next slot while the warp computes slice s from the current one, so every
// warp keeps D-1 slices of the operator in flight without holding them in
// registers.  The copies carry an evict-first L2 policy: the gathered vector
// stays in L2 while the operator streams past it.  Slot and mbarrier phase
// bookkeeping persists across products through a per-warp use counter in
// shared memory.  A copy that does not complete within the bounded wait sets
// the grid's error word (the host then reports NN_ERR_TIMEOUT), waits for
// the warp's other copies in flight and skips the rest of the product.
struct SellF32DiffTma {
    static constexpr int kMaxSlots = 4;   // most slots per warp
    int D;                                // slots per warp (2..kMaxSlots)
    int64_t n, nslices;
    const int64_t *__restrict__ sptr;
    const int32_t *__restrict__ col;
    const float *__restrict__ val;
    const float *__restrict__ rsum;
    int slot_entries;                     // 32 x the widest slice (even)
    uint64_t *bars;                       // [warps][D] (shared memory)
    unsigned *uses;                       // [warps] slots consumed so far (shared memory)
    unsigned char *buf;                   // [warps][D][slot_entries * 8] (shared memory)
    int *error;                           // grid error word (global memory)

    // Shared memory a block of `warps` warps with `slots` slots each needs:
    // mbarriers (at most 32 x 4 x 8 B) and use counters (128 B) in a 2 KB
    // header, then the slots.
    static constexpr int kHeader = 2048;
    __host__ __device__ static size_t smem_bytes(int warps, int slots, int slot_entries) {
        return kHeader + (size_t)warps * slots * slot_entries * 8;
    }

    // Carves the block's shared memory and initialises its mbarriers
    // (every thread calls it; ends with __syncthreads).
    __device__ void setup(unsigned char *smem) {
        const int nw = blockDim.x >> 5;
        bars = reinterpret_cast<uint64_t *>(smem);
        uses = reinterpret_cast<unsigned *>(smem + 8 * kMaxWarps * kMaxSlots);
        buf = smem + kHeader;
        if (threadIdx.x < (unsigned)(nw * D)) mbar_init(bars + threadIdx.x, 1);
        if (threadIdx.x < (unsigned)nw) uses[threadIdx.x] = 0;
        mbar_init_fence();
        __syncthreads();
    }

    template <class Epi>
    __device__ void apply(const Rows &R, const float *x, Epi &&epi) const {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const size_t slot_bytes = (size_t)slot_entries * 8;
        uint64_t *wb = bars + warp * D;
        unsigned char *wbuf = buf + (size_t)warp * D * slot_bytes;
        const uint64_t pol = l2_evict_first_policy();
        const unsigned base = uses[warp];
        const int64_t first = R.s0 + warp;
        auto issue = [&](int64_t s, unsigned u) {
            const int d = (int)(u % D);
            const int64_t e0 = __ldg(sptr + s), e1 = __ldg(sptr + s + 1);
            const unsigned ne = (unsigned)(e1 - e0);   // 32 x even width: a multiple of 64 entries
            unsigned char *dst = wbuf + (size_t)d * slot_bytes;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(wb + d, ne * 8);
            if (ne > 0) {
                bulk_copy_g2s(dst, col + e0, ne * 4, wb + d, pol);
                bulk_copy_g2s(dst + (size_t)slot_entries * 4, val + e0, ne * 4, wb + d, pol);
            }
        };
        if (lane == 0)
            for (int d = 0; d < D - 1; ++d)
                if (first + (int64_t)d * nw < R.s1) issue(first + (int64_t)d * nw, base + d);
        __syncwarp();
        unsigned k = 0;
        for (int64_t s = first; s < R.s1; s += nw, ++k) {
            const unsigned u = base + k;
            if (lane == 0 && s + (int64_t)(D - 1) * nw < R.s1) issue(s + (int64_t)(D - 1) * nw, u + D - 1);
            if (!mbar_wait_bounded(wb + (u % D), (u / D) & 1u)) {
                if (lane == 0) atomicCAS(error, 0, 7 /* NN_ERR_TIMEOUT */);
                for (unsigned j = 1; j < (unsigned)D && s + (int64_t)j * nw < R.s1; ++j)
                    mbar_wait_bounded(wb + ((u + j) % D), ((u + j) / D) & 1u);
                k += 1;
                for (int64_t t = s + nw; t < R.s1 && t <= s + (int64_t)(D - 1) * nw; t += nw) ++k;
                break;
            }
            const unsigned char *sb = wbuf + (size_t)(u % D) * slot_bytes;
            const int w = (int)((__ldg(sptr + s + 1) - __ldg(sptr + s)) >> 5);
            const int2 *c2 = reinterpret_cast<const int2 *>(sb) + lane;
            const float2 *v2 = reinterpret_cast<const float2 *>(sb + (size_t)slot_entries * 4) + lane;
            const int64_t i = s * 32 + lane;
            const float xi = i < n ? x[i] : 0.0f;
            float a0 = 0.0f, a1 = 0.0f;
            int kk = 0;
            for (; kk + 8 <= w; kk += 8) {
                int2 c[4];
                float2 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    c[j] = c2[16 * (kk + 2 * j)];
                    v[j] = v2[16 * (kk + 2 * j)];
                }
                float xv[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    xv[2 * j] = x[c[j].x];
                    xv[2 * j + 1] = x[c[j].y];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    a0 = fmaf(v[j].x, xv[2 * j] - xi, a0);
                    a1 = fmaf(v[j].y, xv[2 * j + 1] - xi, a1);
                }
            }
            for (; kk < w; kk += 2) {
                const int2 c = c2[16 * kk];
                const float2 v = v2[16 * kk];
                a0 = fmaf(v.x, x[c.x] - xi, a0);
                a1 = fmaf(v.y, x[c.y] - xi, a1);
            }
            if (i < n) epi(i, fmaf(__ldg(rsum + i), xi, a0 + a1));
            __syncwarp();
        }
        __syncwarp();
        if (lane == 0) uses[warp] = base + k;
        __syncwarp();
    }
};

// Whether an operator streams through L2 (large systems): the vector passes
// of its solves prefetch their next slices too.
template <bool L>
__device__ __forceinline__ bool op_streams(const SellF64X<L> &A) { return A.stream; }
template <bool L>
__device__ __forceinline__ bool op_streams(const SellF32DiffX<L> &A) { return A.stream; }
__device__ __forceinline__ bool op_streams(const SellF32DiffTma &) { return true; }
template <class Op>
__device__ __forceinline__ bool op_streams(const Op &) { return false; }

// CSR, FP64, one thread per row (rows taken in the same slice order as the
// SELL operators so that every pass of a solve owns the same rows).
struct CsrF64 {
    int64_t n, nslices;
    const int64_t *__restrict__ rowptr;
    const int32_t *__restrict__ col;
    const double *__restrict__ val;

    template <class Epi>
    __device__ __forceinline__ void apply(const Rows &R, const double *x, Epi &&epi) const {
        R.each([&](int64_t i) {
            double acc = 0.0;
            const int64_t e = __ldg(rowptr + i + 1);
            for (int64_t q = __ldg(rowptr + i); q < e; ++q) acc = fma(__ldg(val + q), x[__ldg(col + q)], acc);
            epi(i, acc);
        });
    }
};

}  // namespace nnqp
