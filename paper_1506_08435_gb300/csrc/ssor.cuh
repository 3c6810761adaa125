// Multicolour symmetric SOR as the preconditioner of the CG iterations.
//
// The paper preconditions its CG with block Jacobi/ILU(0) (Sec. 5 and 5.1,
// also inside TRON): triangular solves, sequential along the ordering of the
// unknowns.  With A_FF = D + L + U in an ordering that lists the unknowns
// colour by colour (no two coupled unknowns share a colour), a row of colour
// c couples only to rows of other colours, so each triangular solve becomes
// one parallel pass per colour.  The preconditioner is
//     M = (D + omega L) D^-1 (D + omega U) / (omega (2 - omega))
// (Saad, Iterative Methods for Sparse Linear Systems, Sec. 4.1 and 10.2),
// and z = M^-1 r is
//     forward,  colours ascending:   y_i = (r_i - omega sum_{j in L_i} a_ij y_j) / a_ii
//     backward, colours descending:  z_i = omega (2 - omega) y_i - (omega / a_ii) sum_{j in U_i} a_ij z_j
// (the backward solve of (D + omega U) z' = D y, scaled by omega (2 - omega)
// as it goes).  Restricted to the face F of a CG phase, rows outside F get
// y_i = z_i = 0, so the sums run over F only: the SSOR matrix of A_FF.
//
// One warp owns one 32-row slice of one colour at a time (lane = row; the
// slice's entries are column-major, so every load of an entry index is one
// coalesced transaction); the warps of the whole grid share a colour's
// slices, and a grid barrier separates the colours.
#pragma once
#include <stdint.h>
#include "internal.h"
#include "team.cuh"

namespace nnqp {

// Sum of a_ij v_j over the entries [e0, e0 + 32w) of lane `lane` of one
// slice part (column-major: entry k at e0 + 32k + lane), in order of k.  The
// entries are fetched 4 at a time before the gathers that need them, so a
// warp has up to 4 independent gathers in flight; operators far larger than
// L2 are read with evict-first loads (the gathered vectors stay in L2).
__device__ __forceinline__ double ssor_row_sum(const int32_t *col, const double *val, int64_t e0, int64_t w,
                                               int lane, bool stream, const double *v) {
    constexpr int U = 4;
    double t = 0.0;
    for (int64_t k0 = 0; k0 < w; k0 += U) {
        int32_t c[U];
        double a[U], x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = e0 + (k0 + u) * 32 + lane;
            const bool in = k0 + u < w;
            c[u] = in ? (stream ? __ldcs(col + e) : __ldg(col + e)) : 0;
            a[u] = in ? (stream ? __ldcs(val + e) : __ldg(val + e)) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = k0 + u < w ? v[c[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k0 + u < w) t = fma(a[u], x[u], t);
    }
    return t;
}

// z = M_F^-1 r on the rows of S (see above).  fm: face mask (1 = in F), or
// nullptr for all rows; dinv = 1 / a_ii; y: scratch of n doubles.  on_row(i,
// z_i) runs once for every row as its z_i is final (the caller's fused dot
// products).  Every pass but the last ends in a grid barrier; the caller's
// next reduction or barrier publishes the last colour's z.  false = a
// barrier gave up (timeout).
template <class Team, class F>
__device__ bool ssor_apply(Team &T, const SsorF64 &S, const uint8_t *fm, const double *dinv, const double *r,
                           double *y, double *z, F &&on_row) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const double om = S.omega;
    for (int c = 0; c < S.ncolors; ++c) {
        const int64_t s1 = S.cslice[c + 1];
        for (int64_t s = S.cslice[c] + gw; s < s1; s += nw) {
            const int32_t i = S.row[s * 32 + lane];
            const int64_t e0 = S.lptr[s];
            const double t = ssor_row_sum(S.lcol, S.lval, e0, (S.lptr[s + 1] - e0) >> 5, lane, S.stream, y);
            if (i >= 0) y[i] = (fm == nullptr || fm[i]) ? dinv[i] * fma(-om, t, r[i]) : 0.0;
        }
        if (!T.sync()) return false;
    }
    const double sc = om * (2.0 - om);
    for (int c = S.ncolors - 1; c >= 0; --c) {
        const int64_t s1 = S.cslice[c + 1];
        for (int64_t s = S.cslice[c] + gw; s < s1; s += nw) {
            const int32_t i = S.row[s * 32 + lane];
            const int64_t e0 = S.uptr[s];
            const double t = ssor_row_sum(S.ucol, S.uval, e0, (S.uptr[s + 1] - e0) >> 5, lane, S.stream, z);
            if (i >= 0) {
                const double zi = (fm == nullptr || fm[i]) ? fma(sc, y[i], -om * dinv[i] * t) : 0.0;
                z[i] = zi;
                on_row((int64_t)i, zi);
            }
        }
        if (c > 0 && !T.sync()) return false;
    }
    return true;
}

}  // namespace nnqp
