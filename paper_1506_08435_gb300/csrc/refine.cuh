// Mixed-precision iterative refinement for the box QP.
//
// Outer loop in FP64:  g = A64 x - b (FP64 product), KKT test on the
// projected gradient; the correction problem
//     minimize 1/2 d'A32 d - d'r   subject to  lo - x <= d <= hi - x
// (r = -g) is solved by GPCG with FP32 values and FP32 vectors; then
// x <- P(x + d) in FP64, so the bounds stay exact.  FP32 storage cuts the
// bytes of every inner product to 8 per stored entry (from 12) and keeps the
// work off the FP64 pipe; accuracy is recovered by the FP64 residual.
//
// Refinement contracts only while u32 * cond(A) stays well below 1.  When a
// refinement step fails to halve ||gP||, the solve continues with FP64 GPCG
// from the current iterate (same tolerance), so the result always meets the
// FP64 KKT test; MixedStats::fallback records that this happened.
#pragma once
#include "gpcg.cuh"

namespace nnqp {

// Products allowed to the first FP32 inner solve.  It starts from zero and
// has to do most of the solve's work: CG needs O(sqrt(cond)) steps and cond
// grows like n^(2/d), and GPCG adds the phases that find the active set
// (steady solves of 5e4 - 1e6 unknowns from zero take 6k - 40k products).  A
// cap only guards against an FP32 solve that cannot converge, so it is set
// well above that: 64 sqrt(n), at least 4000.  Every later inner solve (a
// correction of a residual already reduced) may take at most twice the
// products of the first, so a stagnating FP32 solve is cut off early and
// the contraction test then hands the solve to FP64.
__host__ __device__ __forceinline__ int64_t inner_product_cap(int64_t n) {
    const int64_t c = (int64_t)(64.0 * sqrt((double)n));
    return c > 4000 ? c : 4000;
}

// The same for the small instances of a batched solve (at most ~4e4
// unknowns): 8 sqrt(n), at least 4000.  A capped inner solve there still
// contracts the residual four-fold, and the refinement continues; with the
// larger cap some FP32 inner solves ran long before converging (measured on
// the 512-instance batch: 1.73M FP32 products and 275 solves/s against 1.63M
// and 310 solves/s).
__host__ __device__ __forceinline__ int64_t batch_inner_product_cap(int64_t n) {
    const int64_t c = (int64_t)(8.0 * sqrt((double)n));
    return c > 4000 ? c : 4000;
}

struct MixedStats {
    int64_t spmv64 = 0, spmv32 = 0, cg = 0, phases = 0, refinements = 0, vec64 = 0, vec32 = 0, fallback = 0;
    int64_t fl64 = 0, fl32 = 0;
    double gp2 = 0.0;
};

// With SPLIT the inner and fallback solves are separate (non-inlined) calls:
// the registers that the refinement loop keeps live across them are saved
// once per call instead of competing with the solver's inner loops for
// registers (the grid kernels, compiled for 80 or 128 registers).  Without
// SPLIT they are inlined (the batch kernels, which have 255 registers).
// The callee works on register copies of everything passed by reference:
// through the references the objects live in the caller's stack frame, and
// every global store could alias them, so each use would reload them.
template <class Team, class Op, typename V, int CGV>
__device__ __noinline__ int gpcg_call_split(Team &T, const Rows &R, const Op &A, const Bounds<V> &B,
                                            GpcgVecs<V> &v, const GpcgCtl &C, GpcgStats &st) {
    Team t = T;
    GpcgVecs<V> w = v;
    GpcgStats s = st;
    const Rows r = R;
    const Op a = A;
    const Bounds<V> b = B;
    const GpcgCtl c = C;
    const int status = gpcg_solve<Team, Op, V, CGV>(t, r, a, b, w, c, s);
    T = t;
    v = w;
    st = s;
    return status;
}

template <bool SPLIT, class Team, class Op, typename V, int CGV>
__device__ __forceinline__ int gpcg_call(Team &T, const Rows &R, const Op &A, const Bounds<V> &B, GpcgVecs<V> &v,
                                         const GpcgCtl &C, GpcgStats &st) {
    if constexpr (SPLIT)
        return gpcg_call_split<Team, Op, V, CGV>(T, R, A, B, v, C, st);
    else
        return gpcg_solve<Team, Op, V, CGV>(T, R, A, B, v, C, st);
}

// CGV: CG form of the FP64 fallback; CGV32: of the FP32 inner solves.
template <int CGV, int CGV32, bool SPLIT, class Team, class Op64, class Op32>
__device__ int mixed_solve(Team &T, const Rows &R, const Op64 &A, const Op32 &A32, double lo, double hi,
                           const double *b, double *x, GpcgVecs<float> &v, float *r32, float *l32, float *h32,
                           GpcgVecs<double> &v64, double tol, double inner_rtol, int max_ref, int64_t max_spmv,
                           int64_t inner_cap, const GpcgCtl &ctl32, const GpcgCtl &ctl64, MixedStats &st) {
    R.each([&](int64_t i) { x[i] = clampv(x[i], lo, hi); });
    st.vec64 += 2;
    if (!T.sync()) return ST_TIMEOUT;
    double prev_gp2 = -1.0;
    for (int ref = 0;; ++ref) {
        double a[1] = {0.0};
        A.apply(R, x, [&](int64_t i, double ax) {
            const double xi = x[i];
            const double gi = ax - b[i];
            const double gp = proj_grad(xi, gi, lo, hi);
            a[0] += gp * gp;
            r32[i] = (float)(-gi);
            l32[i] = (float)(lo - xi);
            h32[i] = (float)(hi - xi);
            v.x[i] = 0.0f;
        });
        if (!T.reduce(a)) return ST_TIMEOUT;
        ++st.spmv64;
        st.vec64 += 1;
        st.vec32 += 4;
        st.fl64 += 5;
        st.gp2 = a[0];
        if (!isfinite(st.gp2)) return ST_NUMERIC;
        if (st.gp2 <= tol * tol) return ST_OK;
        if (st.spmv64 + st.spmv32 >= max_spmv) return ST_NOT_CONVERGED;
        if (ref >= max_ref || (prev_gp2 > 0.0 && st.gp2 > 0.25 * prev_gp2)) {
            // refinement stopped contracting: finish in FP64 from x
            st.fallback = 1;
            GpcgCtl c = ctl64;
            c.tol = tol;
            c.face_tol = 0.5 * tol;
            c.max_spmv = max_spmv - st.spmv64 - st.spmv32;
            GpcgStats gs;
            v64.x = x;
            const int s = gpcg_call<SPLIT, Team, Op64, double, CGV>(T, R, A, Bounds<double>{lo, hi, nullptr, nullptr}, v64, c, gs);
            st.spmv64 += gs.spmv;
            st.cg += gs.cg;
            st.phases += gs.phases;
            st.vec64 += gs.vec;
            st.fl64 += gs.fl;
            st.gp2 = gs.gp2;
            if (s == ST_TIMEOUT) return s;
            if (v64.x != x) {
                R.each([&](int64_t i) { x[i] = v64.x[i]; });
                st.vec64 += 2;
                if (!T.sync()) return ST_TIMEOUT;
            }
            return s;
        }
        prev_gp2 = st.gp2;
        ++st.refinements;
        GpcgCtl c = ctl32;
        c.tol = inner_rtol * sqrt(st.gp2);
        if (c.tol < 0.25 * tol) c.tol = 0.25 * tol;
        c.face_tol = 0.5 * c.tol;
        // an inner solve that cannot reach its tolerance in FP32 (u32 * cond(A)
        // near 1) is cut off; the contraction test above then decides
        c.max_spmv = max_spmv - st.spmv64 - st.spmv32;
        if (c.max_spmv > inner_cap) c.max_spmv = inner_cap;
        GpcgStats is;
        Bounds<float> B{0.0, 0.0, l32, h32};
        int s = gpcg_call<SPLIT, Team, Op32, float, CGV32>(T, R, A32, B, v, c, is);
        if (ref == 0) {
            const int64_t later = 2 * (is.spmv > 1000 ? is.spmv : 1000);
            if (later < inner_cap) inner_cap = later;
        }
        st.spmv32 += is.spmv;
        st.cg += is.cg;
        st.phases += is.phases;
        st.vec32 += is.vec;
        st.fl32 += is.fl;
        if (s == ST_TIMEOUT || s == ST_NUMERIC) return s;
        R.each([&](int64_t i) { x[i] = clampv(x[i] + (double)v.x[i], lo, hi); });
        st.vec64 += 2;
        st.vec32 += 1;
        st.fl64 += 1;
        if (!T.sync()) return ST_TIMEOUT;
    }
}

}  // namespace nnqp
