// Gradient projection + conjugate gradient (GPCG) for the box QP
//     minimize q(x) = 1/2 x'Ax - b'x   subject to  l <= x <= h
// (the non-negative formulation, Sec. 2.1.3, and its transient form with
// c_min, c_max, Sec. 2.2.2; GPCG is the TAO method named in Sec. 3.1).
// Algorithm after More & Toraldo (SIAM J. Optim. 1, 1991):
//   * gradient-projection phase: projected steps x <- P(x - alpha gP) with
//     the Cauchy length first and Barzilai-Borwein lengths afterwards,
//     backtracking until the Armijo condition q(w) - q(x) <= mu g'(w - x)
//     holds; repeated until the active set stops changing or the decrease
//     stalls (eta1);
//   * CG phase: preconditioned CG on the face {l < x < h} (Jacobi, or the
//     multicolour SSOR of ssor.cuh with CGV = 3) with the active entries frozen, run until the face residual is small or the
//     decrease per iteration stalls (eta2); then a projected search along the
//     CG step, which clips entries that crossed a bound.  If every active
//     entry is binding (its projected gradient is zero) the next phase is CG
//     on the new face, else gradient projection.
// Objective differences use q(w) - q(x) = 1/2 (g(x) + g(w))'(w - x), exact
// for a quadratic, so no large objective values are subtracted.
//
// Every vector pass is over the rows owned by the calling thread (Rows);
// passes are separated by team barriers; every scalar comes out of a team
// reduction, so all threads take the same branches.  Per-thread partial sums
// are kept in the vector type V (FP32 in the mixed-precision inner solves,
// where FP64 arithmetic would cost 59x more per operation) and enter the
// FP64 team reduction once per pass.  The face of a CG phase is kept as a
// byte mask, so the CG iterations make no floating-point comparisons (on
// GB300 FP64 compares run on the same narrow pipe as FP64 FMAs).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "team.cuh"
#include "ops.cuh"
#include "ssor.cuh"

namespace nnqp {

enum : int {
    ST_OK = 0,
    ST_NOT_CONVERGED = 5,
    ST_NUMERIC = 6,
    ST_TIMEOUT = 7,
};

template <typename V>
struct Bounds {
    double lo, hi;
    const V *lov;                 // per-entry bounds when non-null
    const V *hiv;
    __device__ __forceinline__ V l(int64_t i) const { return lov ? lov[i] : (V)lo; }
    __device__ __forceinline__ V h(int64_t i) const { return hiv ? hiv[i] : (V)hi; }
};

template <typename V>
__device__ __forceinline__ V clampv(V x, V l, V h) {
    return x < l ? l : (x > h ? h : x);
}

// Projected gradient of the box QP at x.
template <typename V>
__device__ __forceinline__ V proj_grad(V x, V g, V l, V h) {
    if (x <= l) {
        if (x >= h) return (V)0;
        return g < (V)0 ? g : (V)0;
    }
    if (x >= h) return g > (V)0 ? g : (V)0;
    return g;
}

// Per-thread partial sum of a dot product over the thread's rows.  FP64
// terms add plainly.  FP32 terms (the mixed-precision inner solves) add with
// Kahan's compensation, so a thread's partial keeps close to FP64 accuracy
// however many rows it sums, for three more FP32 operations per term (the
// FP32 pipe is wide; GB300's FP64 pipe is not).  The partial enters the FP64
// team reduction as sum - compensation, rounded once to FP64.
template <typename V>
struct Acc {
    V s = (V)0;
    __device__ __forceinline__ void operator+=(V x) { s += x; }
    __device__ __forceinline__ double value() const { return (double)s; }
};
template <>
struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void operator+=(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Team reduction of per-thread partials kept in V.
template <class Team, typename V, int K>
__device__ __forceinline__ bool team_sum(Team &T, const V (&acc)[K], double (&out)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = (double)acc[k];
    return T.reduce(out);
}
template <class Team, typename V, int K>
__device__ __forceinline__ bool team_sum(Team &T, const Acc<V> (&acc)[K], double (&out)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = acc[k].value();
    return T.reduce(out);
}

// Team reduction followed by scalar work done once per block: f(sums, out)
// runs on warp 0 only (its lanes compute identical values) and its M results
// reach every thread through shared memory.  On GB300 every FP64 warp
// instruction occupies the SM's narrow FP64 pipe for many cycles, so a
// scalar division repeated by all warps of a block costs as much as the
// reduction itself.
template <class Team, int K, int M, class F>
__device__ __forceinline__ bool team_sum_scalar_d(Team &T, double (&d)[K], double (&out)[M], F &&f) {
    if (!T.reduce(d)) return false;
    RedSmem &sm = *T.sm;
    if ((threadIdx.x >> 5) == 0) {
        double r[M];
        f(d, r);
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int j = 0; j < M; ++j) sm.sc[j] = r[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < M; ++j) out[j] = sm.sc[j];
    // the next writer of sc is warp 0 after the next reduction, which
    // begins with a block barrier
    return true;
}
template <class Team, typename V, int K, int M, class F>
__device__ __forceinline__ bool team_sum_scalar(Team &T, const Acc<V> (&acc)[K], double (&d)[K], double (&out)[M],
                                                F &&f) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = acc[k].value();
    return team_sum_scalar_d(T, d, out, f);
}
template <class Team, typename V, int K, int M, class F>
__device__ __forceinline__ bool team_sum_scalar(Team &T, const V (&acc)[K], double (&d)[K], double (&out)[M],
                                                F &&f) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = (double)acc[k];
    return team_sum_scalar_d(T, d, out, f);
}

__device__ __forceinline__ bool flag_set(double f) { return __double_as_longlong(f) != 0; }

// State of the Chronopoulos-Gear / pipelined CG recurrences.  The
// reciprocals 1/alpha and 1/gamma are carried so that a step needs one
// dependent division (FP64 latency on GB300 is tens of cycles per
// operation, and a division is a chain of them).
struct CgScalars {
    double alpha, beta, gamma, ialpha, igamma, maxdec;
};

// From the sums d = (gamma', delta', r'r, crossings) decides whether the CG
// phase stops (returns 1.0 in r[0]) and computes the next coefficients:
//   beta' = gamma'/gamma, alpha' = gamma' / (delta' - beta' gamma'/alpha).
// r = (stop, alpha, beta, gamma, ialpha, igamma, maxdec).
__device__ __forceinline__ void cg_scalar_step(const double (&d)[4], double (&r)[7], const CgScalars &c,
                                               double eta2, double ftol2, bool count_cross) {
    const double dec = 0.5 * c.alpha * c.gamma;
    const double maxdec = dec > c.maxdec ? dec : c.maxdec;
    const double gnew = d[0];
    const double ig = 1.0 / gnew;                 // independent of the chain below
    const double bnew = gnew * c.igamma;
    const double den = fma(-bnew * gnew, c.ialpha, d[1]);
    const double anew = gnew / den;
    const bool stop = (count_cross && d[3] > 0.0) || dec <= eta2 * maxdec || d[2] <= ftol2 || !(gnew > 0.0) ||
                      !(den > 0.0);
    r[0] = stop ? 1.0 : 0.0;
    r[1] = stop ? c.alpha : anew;
    r[2] = stop ? c.beta : bnew;
    r[3] = stop ? c.gamma : gnew;
    r[4] = stop ? c.ialpha : den * ig;
    r[5] = stop ? c.igamma : ig;
    r[6] = maxdec;
}

// First coefficients of a CG phase from gamma = r'u and delta = w'u:
// r = (stop, alpha, beta = 0, gamma, ialpha, igamma, maxdec = 0).
__device__ __forceinline__ void cg_scalar_start(const double (&d)[2], double (&r)[7]) {
    const double gamma = d[0], delta = d[1];
    const bool stop = !(gamma > 0.0) || !(delta > 0.0);
    r[0] = stop ? 1.0 : 0.0;
    r[1] = gamma / delta;
    r[2] = 0.0;
    r[3] = gamma;
    r[4] = delta / gamma;
    r[5] = 1.0 / gamma;
    r[6] = 0.0;
}

__device__ __forceinline__ void cg_take(CgScalars &c, const double (&o)[7]) {
    c.alpha = o[1];
    c.beta = o[2];
    c.gamma = o[3];
    c.ialpha = o[4];
    c.igamma = o[5];
    c.maxdec = o[6];
}

template <typename V>
struct GpcgVecs {
    V *x, *g, *p, *q, *r, *z, *s, *w, *gw;
    const V *b;
    const V *dinv;
    uint8_t *fm;          // face mask of the current CG phase (1 = free)
    V *m2;                // second product input of the pipelined CG (variant 2)
    const SsorF64 *pc;    // SSOR ordering of the textbook form with CGV = 3 (else unused)
};

struct GpcgCtl {
    double tol;          // stop when ||gP||_2 <= tol
    double face_tol;     // CG stops when the face residual norm <= face_tol
    int64_t max_spmv;    // cap on products for this call
    int gp_max;          // gradient-projection steps per phase
    int cg_max;          // CG iterations per face
    double eta1, eta2;   // stall ratios of the GP and CG phases
    double mu;           // Armijo constant
    int cg_variant;      // 0: textbook PCG (3 team barriers per iteration);
                         // 1: Chronopoulos-Gear PCG (2 barriers, one fused reduction);
                         // 2: pipelined PCG (1 barrier: product, updates and
                         //    reduction in one pass; needs GpcgVecs::m2)
    int keep_p;          // 1: the packed direction pass stores p with an L2 evict-last policy
                         //    (the product gathers it next, while its operator streams past)
    int cg_bound_stop;   // 1: end the CG phase as soon as x + s leaves the box;
                         // 0: run CG to its stall test, the projected search clips
};

// vec counts vector streams (one read or write of an n-vector) and fl the
// arithmetic operations per row made by the passes beyond the products; the
// algorithmic traffic of a call is spmv * B_spmv + vec * n * sizeof(V), its
// algorithmic operations spmv * 2 nnz + fl * n.
struct GpcgStats {
    int64_t spmv = 0, cg = 0, phases = 0, vec = 0, fl = 0;
    int64_t pc = 0;   // SSOR applications (their traffic is counted apart from vec)
    double gp2 = 0.0;
};

// Runs GPCG from the iterate in v.x (projected first).  On exit v.x holds
// the final iterate, v.g its gradient (pointers may have been swapped).
// CGV >= 0 fixes the CG variant at compile time (one body per kernel);
// CGV = -1 reads it from C.cg_variant; CGV = 3 is the textbook form with the
// multicolour SSOR preconditioner of v.pc in place of Jacobi (FP64 only).
template <class Team, class Op, typename V, int CGV = -1>
__device__ int gpcg_solve(Team &T, const Rows &R, const Op &A, const Bounds<V> &B, GpcgVecs<V> &v,
                          const GpcgCtl &C, GpcgStats &st) {
    const double tol2 = C.tol * C.tol, ftol2 = C.face_tol * C.face_tol;
    const V zero = (V)0, one = (V)1;
    constexpr bool PC = CGV == 3;
    static_assert(!PC || sizeof(V) == 8, "the SSOR preconditioner runs in FP64");
    const bool pf_on = op_streams(A);   // large system: vector passes prefetch
    R.each([&](int64_t i) { v.x[i] = clampv(v.x[i], B.l(i), B.h(i)); });
    st.vec += 2;
    if (!T.sync()) return ST_TIMEOUT;
    {
        Acc<V> a[1];
        double d[1];
        A.apply(R, v.x, [&](int64_t i, V ax) {
            V gi = ax - v.b[i];
            v.g[i] = gi;
            V gp = proj_grad(v.x[i], gi, B.l(i), B.h(i));
            a[0] += gp * gp;
        });
        if (!team_sum(T, a, d)) return ST_TIMEOUT;
        ++st.spmv;
        st.vec += 1;
        st.fl += 3;
        st.gp2 = d[0];
    }
    int status = ST_NOT_CONVERGED;
    double bb = 0.0;   // step length carried between gradient-projection steps
    for (;;) {
        if (!isfinite(st.gp2)) { status = ST_NUMERIC; break; }
        if (st.gp2 <= tol2) { status = ST_OK; break; }
        if (st.spmv >= C.max_spmv) break;
        ++st.phases;
        // ------------------------------------------------ gradient projection
        double maxdec = 0.0;
        for (int it = 0; it < C.gp_max; ++it) {
            double alpha = bb;
            if (!(alpha > 0.0)) {   // Cauchy length along -gP
                R.each([&](int64_t i) { v.p[i] = -proj_grad(v.x[i], v.g[i], B.l(i), B.h(i)); });
                st.vec += 3;
                if (!T.sync()) return ST_TIMEOUT;
                Acc<V> a1[1];
                double d1[1], oc[2];
                A.apply(R, v.p, [&](int64_t i, V ap) { a1[0] += v.p[i] * ap; });
                const double gp2 = st.gp2;
                if (!team_sum_scalar(T, a1, d1, oc, [&](const double (&d)[1], double (&r)[2]) {
                        r[0] = d[0] > 0.0 ? 1.0 : 0.0;
                        r[1] = gp2 / d[0];
                    }))
                    return ST_TIMEOUT;
                ++st.spmv;
                st.fl += 2;
                if (!flag_set(oc[0])) break;
                alpha = oc[1];
            }
            bool accepted = false;
            double d2[6], o2[5];
            for (int ls = 0; ls < 48 && st.spmv < C.max_spmv; ++ls) {
                Acc<V> a2[6];
                const V va = (V)alpha;
                R.each([&](int64_t i) {
                    V l = B.l(i), h = B.h(i), xi = v.x[i];
                    V wi = clampv(xi - va * proj_grad(xi, v.g[i], l, h), l, h);
                    v.w[i] = wi;
                    a2[0] += v.g[i] * (wi - xi);
                    a2[1] += ((xi <= l || xi >= h) != (wi <= l || wi >= h)) ? one : zero;
                });
                if (!T.sync()) return ST_TIMEOUT;
                A.apply(R, v.w, [&](int64_t i, V aw) {
                    V gwi = aw - v.b[i];
                    v.gw[i] = gwi;
                    V wi = v.w[i];
                    V si = wi - v.x[i], yi = gwi - v.g[i];
                    a2[2] += (v.g[i] + gwi) * si;
                    V gp = proj_grad(wi, gwi, B.l(i), B.h(i));
                    a2[3] += gp * gp;
                    a2[4] += si * si;
                    a2[5] += si * yi;
                });
                // Armijo test; on acceptance the Barzilai-Borwein length s's/s'y
                // for the next step and the phase's stall test (no change of the
                // active set, or a decrease below eta1 times the best)
                const double al = alpha, md = maxdec;
                if (!team_sum_scalar(T, a2, d2, o2, [&](const double (&d)[6], double (&r)[5]) {
                        const bool acc = 0.5 * d[2] <= C.mu * d[0];
                        const double dec = -0.5 * d[2];
                        const double mdn = dec > md ? dec : md;
                        r[0] = acc ? 1.0 : 0.0;
                        r[1] = 0.5 * al;
                        r[2] = d[5] > 0.0 ? d[4] / d[5] : 0.0;
                        r[3] = mdn;
                        r[4] = (d[3] <= tol2 || d[1] == 0.0 || dec <= C.eta1 * mdn) ? 1.0 : 0.0;
                    }))
                    return ST_TIMEOUT;
                ++st.spmv;
                st.vec += 7;
                st.fl += 17;
                if (flag_set(o2[0])) {
                    accepted = true;
                    break;
                }
                alpha = o2[1];
            }
            if (!accepted) {
                bb = 0.0;
                break;
            }
            V *t = v.x; v.x = v.w; v.w = t;
            t = v.g; v.g = v.gw; v.gw = t;
            st.gp2 = d2[3];
            bb = o2[2];
            maxdec = o2[3];
            if (flag_set(o2[4]) || st.spmv >= C.max_spmv) break;
        }
        if (st.gp2 <= tol2 || st.spmv >= C.max_spmv || !isfinite(st.gp2)) continue;
        // ------------------------------------------------ CG on faces
        const bool count_cross = C.cg_bound_stop != 0;
        for (;;) {
            if ((CGV >= 0 ? CGV : C.cg_variant) == 1) {
                // Chronopoulos-Gear form: one fused reduction per iteration
                // (gamma = r'u and delta = w'u with u = D^-1 r, w = A_F u), the
                // product A p carried by the recurrence q = w + beta q.
                R.each([&](int64_t i) {
                    V xi = v.x[i];
                    const bool fr = xi > B.l(i) && xi < B.h(i);
                    v.fm[i] = fr ? 1 : 0;
                    V ri = fr ? -v.g[i] : zero;
                    v.r[i] = ri;
                    v.z[i] = v.dinv[i] * ri;
                    v.s[i] = zero;
                    v.p[i] = zero;
                    v.q[i] = zero;
                });
                st.vec += 8;
                st.fl += 1;
                if (!T.sync()) return ST_TIMEOUT;
                Acc<V> a3[2];
                double d3[2];
                A.apply(R, v.z, [&](int64_t i, V au) {
                    V wi = v.fm[i] ? au : zero;
                    v.w[i] = wi;
                    V ui = v.z[i];
                    a3[0] += v.r[i] * ui;
                    a3[1] += wi * ui;
                });
                double o3[7];
                if (!team_sum_scalar(T, a3, d3, o3, [&](const double (&d)[2], double (&r)[7]) { cg_scalar_start(d, r); }))
                    return ST_TIMEOUT;
                ++st.spmv;
                st.vec += 3;
                st.fl += 4;
                if (flag_set(o3[0])) break;
                CgScalars cs;
                cg_take(cs, o3);
                for (int k = 0; k < C.cg_max; ++k) {
                    const V va = (V)cs.alpha, vb = (V)cs.beta;
                    Acc<V> a4[4];   // gamma, delta, r'r, bound crossings
                    const void *pf6[6] = {v.z, v.p, v.w, v.q, v.s, v.r};
                    R.each_pf(pf6, (int)sizeof(V), pf_on, [&](int64_t i) {
                        V pi = v.z[i] + vb * v.p[i];
                        V qi = v.w[i] + vb * v.q[i];
                        V si = v.s[i] + va * pi;
                        V ri = v.r[i] - va * qi;
                        v.p[i] = pi;
                        v.q[i] = qi;
                        v.s[i] = si;
                        v.r[i] = ri;
                        v.z[i] = v.dinv[i] * ri;
                        if (count_cross) {
                            V xs = v.x[i] + si;
                            a4[3] += (xs < B.l(i) || xs > B.h(i)) ? one : zero;
                        }
                    });
                    st.vec += count_cross ? 13 : 12;
                    st.fl += 9;
                    if (!T.sync()) return ST_TIMEOUT;
                    A.apply(R, v.z, [&](int64_t i, V au) {
                        V wi = v.fm[i] ? au : zero;
                        v.w[i] = wi;
                        V ri = v.r[i], ui = v.z[i];
                        a4[0] += ri * ui;
                        a4[1] += wi * ui;
                        a4[2] += ri * ri;
                    });
                    double d4[4], o[7];
                    if (!team_sum_scalar(T, a4, d4, o, [&](const double (&d)[4], double (&r)[7]) {
                            cg_scalar_step(d, r, cs, C.eta2, ftol2, count_cross);
                        }))
                        return ST_TIMEOUT;
                    ++st.spmv;
                    ++st.cg;
                    st.vec += 3;
                    st.fl += 6;
                    if (flag_set(o[0]) || st.spmv >= C.max_spmv) break;
                    cg_take(cs, o);
                }
            } else if ((CGV >= 0 ? CGV : C.cg_variant) == 2) {
                // Pipelined form (Ghysels & Vanroose, Parallel Comput. 40, 2014)
                // with the Jacobi preconditioner applied explicitly: u = D^-1 r,
                // m = D^-1 w, w = A_F u.  The product n = A_F m of iteration i
                // only needs vectors of iteration i, so it is fused with every
                // update of the iteration and with the partial dot products of
                // the next one; the reduction's barrier also publishes m.  m is
                // double-buffered (gw, m2): a pass reads m_i of other rows while
                // writing m_(i+1) of its own.  Recurrences (q = A_F p via v.q,
                // z = A_F D^-1 A_F p via v.z):
                //   z = n + beta z, q = w + beta q, p = u + beta p,
                //   s += alpha p, r -= alpha q, w -= alpha z.
                V *mc = v.gw, *mn = v.m2;
                R.each([&](int64_t i) {
                    V xi = v.x[i];
                    const bool fr = xi > B.l(i) && xi < B.h(i);
                    v.fm[i] = fr ? 1 : 0;
                    V ri = fr ? -v.g[i] : zero;
                    v.r[i] = ri;
                    mn[i] = v.dinv[i] * ri;    // u_0, input of the first product
                    v.s[i] = zero;
                    v.p[i] = zero;
                    v.q[i] = zero;
                    v.z[i] = zero;
                });
                st.vec += 10;
                st.fl += 1;
                if (!T.sync()) return ST_TIMEOUT;
                Acc<V> a3[2];
                double d3[2];
                A.apply(R, mn, [&](int64_t i, V au) {
                    V wi = v.fm[i] ? au : zero;
                    V di = v.dinv[i];
                    v.w[i] = wi;
                    mc[i] = di * wi;
                    V ri = v.r[i], ui = di * ri;
                    a3[0] += ri * ui;
                    a3[1] += wi * ui;
                });
                double o3[7];
                if (!team_sum_scalar(T, a3, d3, o3, [&](const double (&d)[2], double (&r)[7]) { cg_scalar_start(d, r); }))
                    return ST_TIMEOUT;
                ++st.spmv;
                st.vec += 5;
                st.fl += 6;
                if (flag_set(o3[0])) break;
                CgScalars cs;
                cg_take(cs, o3);
                for (int k = 0; k < C.cg_max; ++k) {
                    const V va = (V)cs.alpha, vb = (V)cs.beta;
                    Acc<V> a4[4];   // gamma, delta, r'r, bound crossings
                    A.apply(R, mc, [&](int64_t i, V an) {
                        V ni = v.fm[i] ? an : zero;
                        V di = v.dinv[i];
                        V ri = v.r[i], wi = v.w[i];
                        V zi = ni + vb * v.z[i];
                        V qi = wi + vb * v.q[i];
                        V pi = di * ri + vb * v.p[i];
                        V si = v.s[i] + va * pi;
                        ri = ri - va * qi;
                        wi = wi - va * zi;
                        v.z[i] = zi;
                        v.q[i] = qi;
                        v.p[i] = pi;
                        v.s[i] = si;
                        v.r[i] = ri;
                        v.w[i] = wi;
                        mn[i] = di * wi;
                        V ui = di * ri;
                        a4[0] += ri * ui;
                        a4[1] += wi * ui;
                        a4[2] += ri * ri;
                        if (count_cross) {
                            V xs = v.x[i] + si;
                            a4[3] += (xs < B.l(i) || xs > B.h(i)) ? one : zero;
                        }
                    });
                    double d4[4], o[7];
                    if (!team_sum_scalar(T, a4, d4, o, [&](const double (&d)[4], double (&r)[7]) {
                            cg_scalar_step(d, r, cs, C.eta2, ftol2, count_cross);
                        }))
                        return ST_TIMEOUT;
                    ++st.spmv;
                    ++st.cg;
                    st.vec += count_cross ? 15 : 14;
                    st.fl += 21;
                    if (flag_set(o[0]) || st.spmv >= C.max_spmv) break;
                    cg_take(cs, o);
                    V *t = mc;
                    mc = mn;
                    mn = t;
                }
            } else {
                // textbook preconditioned CG (z = D^-1 r, or z = M_F^-1 r by
                // the SSOR sweeps when PC)
                Acc<V> a3[1];
                double d3[1];
                if constexpr (PC) {
                    R.each([&](int64_t i) {
                        V xi = v.x[i];
                        const bool fr = xi > B.l(i) && xi < B.h(i);
                        v.fm[i] = fr ? 1 : 0;
                        v.r[i] = fr ? -v.g[i] : zero;
                        v.s[i] = zero;
                    });
                    st.vec += 5;
                    if (!T.sync()) return ST_TIMEOUT;
                    if (!ssor_apply(T, *v.pc, v.fm, v.dinv, v.r, v.w, v.z, [&](int64_t i, double zi) {
                            v.p[i] = zi;
                            a3[0] += v.r[i] * zi;
                        }))
                        return ST_TIMEOUT;
                    ++st.pc;
                    st.vec += 2;
                    st.fl += 2;
                } else {
                    R.each([&](int64_t i) {
                        V xi = v.x[i];
                        const bool fr = xi > B.l(i) && xi < B.h(i);
                        v.fm[i] = fr ? 1 : 0;
                        V ri = fr ? -v.g[i] : zero;
                        V zi = v.dinv[i] * ri;
                        v.r[i] = ri;
                        v.z[i] = zi;
                        v.p[i] = zi;
                        v.s[i] = zero;
                        a3[0] += ri * zi;
                    });
                    st.vec += 8;
                    st.fl += 3;
                }
                if (!team_sum(T, a3, d3)) return ST_TIMEOUT;
                double rho = d3[0];
                if (!(rho > 0.0)) break;
                double maxdec = 0.0;
                for (int k = 0; k < C.cg_max; ++k) {
                    Acc<V> a4[1];
                    double d4[1];
                    A.apply(R, v.p, [&](int64_t i, V ap) {
                        V qi = v.fm[i] ? ap : zero;
                        v.q[i] = qi;
                        a4[0] += v.p[i] * qi;
                    });
                    // alpha = rho / p'q, computed once per block by warp 0
                    double o4[2];
                    if (!team_sum_scalar(T, a4, d4, o4, [&](const double (&d)[1], double (&r)[2]) {
                            r[0] = d[0] > 0.0 ? 1.0 : 0.0;
                            r[1] = rho / d[0];
                        }))
                        return ST_TIMEOUT;
                    ++st.spmv;
                    st.vec += 2;
                    st.fl += 2;
                    if (!flag_set(o4[0])) break;
                    const double alpha = o4[1];
                    const V va = (V)alpha;
                    Acc<V> a5[3];
                    double d5[3];
                    const void *pf5[5] = {v.s, v.p, v.r, v.q, v.dinv};
                    auto upd = [&](int64_t i) {
                        V si = v.s[i] + va * v.p[i];
                        V ri = v.r[i] - va * v.q[i];
                        V zi = v.dinv[i] * ri;
                        v.s[i] = si;
                        v.r[i] = ri;
                        v.z[i] = zi;
                        a5[0] += ri * zi;
                        a5[1] += ri * ri;
                        if (count_cross) {
                            V xs = v.x[i] + si;
                            a5[2] += (xs < B.l(i) || xs > B.h(i)) ? one : zero;
                        }
                    };
                    const void *al6[6] = {v.s, v.p, v.r, v.q, v.dinv, v.z};
                    if constexpr (PC) {
                        // s and r only: z comes from the sweeps below
                        const void *pf4[4] = {v.s, v.p, v.r, v.q};
                        R.each_pf(pf4, (int)sizeof(V), pf_on, [&](int64_t i) {
                            V si = v.s[i] + va * v.p[i];
                            V ri = v.r[i] - va * v.q[i];
                            v.s[i] = si;
                            v.r[i] = ri;
                            a5[1] += ri * ri;
                            if (count_cross) {
                                V xs = v.x[i] + si;
                                a5[2] += (xs < B.l(i) || xs > B.h(i)) ? one : zero;
                            }
                        });
                        if (!T.sync()) return ST_TIMEOUT;
                        if (!ssor_apply(T, *v.pc, v.fm, v.dinv, v.r, v.w, v.z,
                                        [&](int64_t i, double zi) { a5[0] += v.r[i] * zi; }))
                            return ST_TIMEOUT;
                        ++st.pc;
                        st.vec -= 2;   // no D^-1 read, no z write in the update pass
                        st.vec += 1;   // r read again by the dot product of the sweep
                        st.fl -= 1;
                    } else if (!count_cross && aligned16(al6)) {
                        constexpr int W = Pack<V>::W;
                        R.each_chunk<W>([&](int64_t i, int cnt) {
                            if (cnt < W) {
                                for (int j = 0; j < cnt; ++j) upd(i + j);
                                return;
                            }
                            V sv[W], pv[W], rv[W], qv[W], dv[W];
                            ld_pack(v.s + i, sv);
                            ld_pack(v.p + i, pv);
                            ld_pack(v.r + i, rv);
                            ld_pack(v.q + i, qv);
                            ld_pack(v.dinv + i, dv);
#pragma unroll
                            for (int j = 0; j < W; ++j) {
                                sv[j] = sv[j] + va * pv[j];
                                rv[j] = rv[j] - va * qv[j];
                                dv[j] = dv[j] * rv[j];
                                a5[0] += rv[j] * dv[j];
                                a5[1] += rv[j] * rv[j];
                            }
                            st_pack(v.s + i, sv);
                            st_pack(v.r + i, rv);
                            st_pack(v.z + i, dv);
                        });
                    } else {
                        R.each_pf(pf5, (int)sizeof(V), pf_on, upd);
                    }
                    // stop test and beta = rho' / rho, once per block by warp 0
                    double o5[3];
                    const double md = maxdec;
                    if (!team_sum_scalar(T, a5, d5, o5, [&](const double (&d)[3], double (&r)[3]) {
                            const double dec = 0.5 * alpha * rho;
                            const double mdn = dec > md ? dec : md;
                            r[0] = ((count_cross && d[2] > 0.0) || dec <= C.eta2 * mdn || d[1] <= ftol2 || !(d[0] > 0.0))
                                       ? 1.0
                                       : 0.0;
                            r[1] = d[0] / rho;
                            r[2] = mdn;
                        }))
                        return ST_TIMEOUT;
                    ++st.cg;
                    st.vec += count_cross ? 9 : 8;
                    st.fl += 9;
                    maxdec = o5[2];
                    if (flag_set(o5[0]) || st.spmv >= C.max_spmv) break;
                    const V vb = (V)o5[1];
                    rho = d5[0];
                    const void *pf2[2] = {v.z, v.p};
                    if (aligned16(pf2)) {
                        constexpr int W = Pack<V>::W;
                        const uint64_t keep = l2_evict_last_policy();
                        R.each_chunk<W>([&](int64_t i, int cnt) {
                            if (cnt < W) {
                                for (int j = 0; j < cnt; ++j) v.p[i + j] = v.z[i + j] + vb * v.p[i + j];
                                return;
                            }
                            V zv[W], pv[W];
                            ld_pack(v.z + i, zv);
                            ld_pack(v.p + i, pv);
#pragma unroll
                            for (int j = 0; j < W; ++j) pv[j] = zv[j] + vb * pv[j];
                            if (C.keep_p)
                                st_pack_keep(v.p + i, pv, keep);
                            else
                                st_pack(v.p + i, pv);
                        });
                    } else {
                        R.each_pf(pf2, (int)sizeof(V), pf_on, [&](int64_t i) { v.p[i] = v.z[i] + vb * v.p[i]; });
                    }
                    st.vec += 3;
                    st.fl += 2;
                    if (!T.sync()) return ST_TIMEOUT;
                }
            }
            // projected search along the CG step s
            double alpha = 1.0;
            bool accepted = false;
            double d6[5], o6[3];
            for (int ls = 0; ls < 48; ++ls) {
                Acc<V> a6[5];
                const V va = (V)alpha;
                R.each([&](int64_t i) {
                    V xi = v.x[i];
                    V wi = clampv(xi + va * v.s[i], B.l(i), B.h(i));
                    v.w[i] = wi;
                    a6[0] += v.g[i] * (wi - xi);
                });
                if (!T.sync()) return ST_TIMEOUT;
                A.apply(R, v.w, [&](int64_t i, V aw) {
                    V gwi = aw - v.b[i];
                    v.gw[i] = gwi;
                    V wi = v.w[i], l = B.l(i), h = B.h(i);
                    a6[2] += (v.g[i] + gwi) * (wi - v.x[i]);
                    V gp = proj_grad(wi, gwi, l, h);
                    a6[3] += gp * gp;
                    a6[4] += ((wi <= l || wi >= h) && gp != zero) ? one : zero;
                });
                // Armijo test; after acceptance the face loop ends on convergence
                // or on a non-binding active entry (back to gradient projection)
                const double al = alpha;
                if (!team_sum_scalar(T, a6, d6, o6, [&](const double (&d)[5], double (&r)[3]) {
                        r[0] = 0.5 * d[2] <= C.mu * d[0] ? 1.0 : 0.0;
                        r[1] = (d[3] <= tol2 || !isfinite(d[3]) || d[4] > 0.0) ? 1.0 : 0.0;
                        r[2] = 0.5 * al;
                    }))
                    return ST_TIMEOUT;
                ++st.spmv;
                st.vec += 7;
                st.fl += 11;
                if (flag_set(o6[0])) {
                    accepted = true;
                    break;
                }
                alpha = o6[2];
            }
            if (!accepted) break;
            V *t = v.x; v.x = v.w; v.w = t;
            t = v.g; v.g = v.gw; v.gw = t;
            st.gp2 = d6[3];
            if (flag_set(o6[1]) || st.spmv >= C.max_spmv) break;
        }
    }
    return status;
}

}  // namespace nnqp
