// Sparse operators y = A x on the free unknowns, each fused with a per-row
// epilogue epi(i, y_i) so that the consumer of the product (gradient,
// search direction, dot products) runs in the same pass over the rows.
//
// The product is the Hessian-vector product of the QP (the "MatMult" of the
// paper's cost model, Sec. 4, Table of bytes transferred); the algorithmic
// traffic of one product is nnz*(s_val + 4) + 4(n+1) + s_x n + s_y n.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "team.cuh"

namespace nnqp {

// SELL-32, FP64 values; off-diagonals in slices, diagonal separate:
//   y_i = d_i x_i + sum_k v_ik x_{c_ik}
struct SellF64 {
    int64_t n, nslices;
    const int64_t *__restrict__ sptr;
    const int32_t *__restrict__ col;
    const double *__restrict__ val;
    const double *__restrict__ diag;

    template <class Epi>
    __device__ __forceinline__ void apply(const Rows &R, const double *x, Epi &&epi) const {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int64_t s = R.s0 + (threadIdx.x >> 5); s < R.s1; s += nw) {
            const int64_t base = __ldg(sptr + s);
            const int w = (int)((__ldg(sptr + s + 1) - base) >> 5);
            const int64_t i = s * 32 + lane;
            const int32_t *c = col + base + lane;
            const double *v = val + base + lane;
            double acc = 0.0;
#pragma unroll 4
            for (int k = 0; k < w; ++k) acc = fma(__ldg(v + 32 * k), x[__ldg(c + 32 * k)], acc);
            if (i < n) epi(i, fma(__ldg(diag + i), x[i], acc));
        }
    }
};

// SELL-32, FP32 values, FP32 vectors, in difference form:
//   y_i = s_i x_i + sum_k v_ik (x_{c_ik} - x_i),   s_i = sum_j A_ij (row sum)
// The implied diagonal is s_i - sum_k v_ik, so rounding the off-diagonals to
// FP32 perturbs A by a matrix with zero row sums, and rounding in the
// products scales with |x_j - x_i| instead of |x_j|.
struct SellF32Diff {
    int64_t n, nslices;
    const int64_t *__restrict__ sptr;
    const int32_t *__restrict__ col;
    const float *__restrict__ val;
    const float *__restrict__ rsum;

    template <class Epi>
    __device__ __forceinline__ void apply(const Rows &R, const float *x, Epi &&epi) const {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int64_t s = R.s0 + (threadIdx.x >> 5); s < R.s1; s += nw) {
            const int64_t base = __ldg(sptr + s);
            const int w = (int)((__ldg(sptr + s + 1) - base) >> 5);
            const int64_t i = s * 32 + lane;
            const int32_t *c = col + base + lane;
            const float *v = val + base + lane;
            const float xi = i < n ? x[i] : 0.0f;
            float acc = 0.0f;
#pragma unroll 4
            for (int k = 0; k < w; ++k) acc = fmaf(__ldg(v + 32 * k), x[__ldg(c + 32 * k)] - xi, acc);
            if (i < n) epi(i, fmaf(__ldg(rsum + i), xi, acc));
        }
    }
};

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
