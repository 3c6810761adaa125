// Trust-region Newton method for bound constraints (TRON: Lin & More,
// SIAM J. Optim. 9, 1999), the active-set Newton trust-region solver the
// paper runs through TAO (Sec. 3.1; Sec. 5.1 compares KSP tolerances 1e-1,
// 1e-2 and 1e-3 as TRON1/2/3), for the box QP
//     minimize q(x) = 1/2 x'Ax - b'x   subject to  l <= x <= h.
// The Hessian is A itself, so the quadratic model of every iteration is the
// objective and the ratio of actual to predicted reduction is 1: each step
// is accepted and the radius only grows.  One outer iteration:
//   * Cauchy step: s(alpha) = P(x - alpha g) - x along the projected
//     gradient path, alpha carried from the previous iteration, extrapolated
//     (x10) while s(alpha) satisfies both the sufficient decrease
//     q(x+s) - q(x) <= mu0 g's and ||s|| <= mu1 Delta and still changes,
//     else backtracked (x0.1) until it does;
//   * subspace steps: preconditioned CG (Jacobi, or the multicolour SSOR of
//     ssor.cuh when v.pc is set) on the face {l < x < h} for
//     A_FF w = -g_F, truncated where it leaves the trust region ||w|| <=
//     Delta (Steihaug) and stopped once the face residual is at most
//     ksp_rtol times the face gradient at the Cauchy point, then a projected
//     search x <- P(x + beta w) (beta = 1, 1/2, ...) with the sufficient
//     decrease test; repeated on the new face while the search adds active
//     bounds, the CG step stayed inside the region and the face gradient is
//     still above that tolerance;
//   * radius update: Delta <- max(Delta, sigma3 ||x_(k+1) - x_k||).
// Objective differences use q(w) - q(x) = 1/2 (g(x) + g(w))'(w - x), exact
// for a quadratic.  Passes, barriers and reductions follow the conventions
// of gpcg.cuh (every scalar comes out of a team reduction, so all threads
// take the same branches).
#pragma once
#include "gpcg.cuh"

namespace nnqp {

struct TronCtl {
    double tol;        // stop when ||gP||_2 <= tol
    double face_tol;   // absolute floor of the CG residual test
    double ksp_rtol;   // subspace steps stop at ||g_F|| <= ksp_rtol ||g_F(Cauchy point)||
    int64_t max_spmv;  // cap on products for this call
    int max_minor;     // subspace steps per outer iteration
};

struct TronStats {
    int64_t spmv = 0, cg = 0, iters = 0, minor = 0, vec = 0, fl = 0;
    int64_t pc = 0;   // SSOR applications (their traffic is counted apart from vec)
    double gp2 = 0.0;
};

struct TronVecs {
    double *x, *g;            // iterate and its gradient
    double *w, *gw;           // trial point and its gradient
    double *p, *q, *r, *z, *s; // CG vectors; p, q also keep the last accepted Cauchy trial
    double *xo;               // iterate at the start of the outer iteration
    const double *b, *dinv;
    uint8_t *fm;              // face mask of the subspace step (1 = free)
    const SsorF64 *pc;        // SSOR ordering, or nullptr for Jacobi
};

constexpr double kTronMu0 = 1e-2;     // sufficient decrease
constexpr double kTronMu1 = 1.0;      // Cauchy step length bound, in units of Delta
constexpr double kTronSigma3 = 4.0;   // radius expansion
constexpr int kTronCauchyTrials = 60;
constexpr int kTronExtrapolations = 20;

template <class Team, class Op>
__device__ int tron_solve(Team &T, const Rows &R, const Op &A, const Bounds<double> &B, TronVecs &v,
                          const TronCtl &C, TronStats &st) {
    const double tol2 = C.tol * C.tol;
    R.each([&](int64_t i) { v.x[i] = clampv(v.x[i], B.l(i), B.h(i)); });
    st.vec += 2;
    if (!T.sync()) return ST_TIMEOUT;
    {
        double a[1] = {0.0}, d[1];
        A.apply(R, v.x, [&](int64_t i, double ax) {
            const double xi = v.x[i], gi = ax - v.b[i];
            v.g[i] = gi;
            v.xo[i] = xi;
            const double gp = proj_grad(xi, gi, B.l(i), B.h(i));
            a[0] += gp * gp;
        });
        if (!team_sum(T, a, d)) return ST_TIMEOUT;
        ++st.spmv;
        st.vec += 4;
        st.fl += 3;
        st.gp2 = d[0];
    }
    double delta = sqrt(st.gp2);   // initial radius ||gP(x_0)|| (Lin & More)
    double alpha_c = 1.0;          // Cauchy step length carried between iterations
    int status = ST_NOT_CONVERGED;
    for (;;) {
        if (!isfinite(st.gp2)) { status = ST_NUMERIC; break; }
        if (st.gp2 <= tol2) { status = ST_OK; break; }
        if (st.spmv >= C.max_spmv) break;
        ++st.iters;
        // ------------------------------------------------ Cauchy step
        // dir: +1 extrapolating from an acceptable first trial, -1 backtracking
        int dir = 0;
        bool have = false;             // an accepted trial is kept in (p, q)
        double acc_gp2 = 0.0, acc_alpha = 0.0, ss_prev = -1.0;
        double alpha = alpha_c;
        bool done = false;
        for (int t = 0; t < kTronCauchyTrials && st.spmv < C.max_spmv; ++t) {
            double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            const bool first = t == 0;
            R.each([&](int64_t i) {
                const double xi = v.x[i];
                v.w[i] = clampv(xi - alpha * v.g[i], B.l(i), B.h(i));
                if (first) {                       // ||x_k - x_(k-1)||^2 for the radius
                    const double dx = xi - v.xo[i];
                    a[4] += dx * dx;
                    v.xo[i] = xi;
                }
            });
            st.vec += first ? 5 : 3;
            st.fl += first ? 6 : 3;
            if (!T.sync()) return ST_TIMEOUT;
            A.apply(R, v.w, [&](int64_t i, double aw) {
                const double gwi = aw - v.b[i], wi = v.w[i], gi = v.g[i];
                v.gw[i] = gwi;
                const double si = wi - v.x[i];
                a[0] += gi * si;
                a[1] += (gi + gwi) * si;
                a[2] += si * si;
                const double gp = proj_grad(wi, gwi, B.l(i), B.h(i));
                a[3] += gp * gp;
            });
            double d[5], o[2];
            const double dl = delta;
            if (!team_sum_scalar(T, a, d, o, [&](const double (&s)[5], double (&r)[2]) {
                    // radius after the previous iteration (ratio 1: the model is exact)
                    const double dn = first ? fmax(dl, kTronSigma3 * sqrt(s[4])) : dl;
                    const double mr = kTronMu1 * dn;
                    r[0] = (0.5 * s[1] <= kTronMu0 * s[0] && s[2] <= mr * mr) ? 1.0 : 0.0;
                    r[1] = dn;
                }))
                return ST_TIMEOUT;
            ++st.spmv;
            st.vec += 4;
            st.fl += 14;
            delta = o[1];
            const bool ok = flag_set(o[0]);
            if (first) dir = ok ? 1 : -1;
            if (dir < 0) {
                if (ok) {                          // accept the current trial
                    double *t1 = v.x; v.x = v.w; v.w = t1;
                    t1 = v.g; v.g = v.gw; v.gw = t1;
                    st.gp2 = d[3];
                    alpha_c = alpha;
                    done = true;
                    break;
                }
                alpha *= 0.1;
            } else {
                if (ok && (first || d[2] > ss_prev * (1.0 + 1e-12))) {
                    double *t1 = v.p; v.p = v.w; v.w = t1;     // keep it, try a longer step
                    t1 = v.q; v.q = v.gw; v.gw = t1;
                    have = true;
                    acc_gp2 = d[3];
                    acc_alpha = alpha;
                    ss_prev = d[2];
                    if (t >= kTronExtrapolations) break;
                    alpha *= 10.0;
                } else {
                    break;
                }
            }
        }
        if (!done) {
            if (!have) break;                      // no acceptable step within the trials
            double *t1 = v.x; v.x = v.p; v.p = t1;
            t1 = v.g; v.g = v.q; v.q = t1;
            st.gp2 = acc_gp2;
            alpha_c = acc_alpha;
        }
        // ------------------------------------------------ subspace steps
        double ktol2 = 0.0;   // fixed at the Cauchy point for the whole phase
        for (int mi = 0; mi < C.max_minor; ++mi) {
            if (!(st.gp2 > tol2) || st.spmv >= C.max_spmv) break;
            ++st.minor;
            double a0[2] = {0.0, 0.0}, d0[2];
            if (v.pc) {
                R.each([&](int64_t i) {
                    const double xi = v.x[i];
                    const bool fr = xi > B.l(i) && xi < B.h(i);
                    v.fm[i] = fr ? 1 : 0;
                    const double ri = fr ? -v.g[i] : 0.0;
                    v.r[i] = ri;
                    v.s[i] = 0.0;
                    a0[1] += ri * ri;
                });
                if (!T.sync()) return ST_TIMEOUT;
                if (!ssor_apply(T, *v.pc, v.fm, v.dinv, v.r, v.w, v.z, [&](int64_t i, double zi) {
                        v.p[i] = zi;
                        a0[0] += v.r[i] * zi;
                    }))
                    return ST_TIMEOUT;
                ++st.pc;
                st.vec += 7;
                st.fl += 4;
            } else {
                R.each([&](int64_t i) {
                    const double xi = v.x[i];
                    const bool fr = xi > B.l(i) && xi < B.h(i);
                    v.fm[i] = fr ? 1 : 0;
                    const double ri = fr ? -v.g[i] : 0.0;
                    const double zi = v.dinv[i] * ri;
                    v.r[i] = ri;
                    v.z[i] = zi;
                    v.p[i] = zi;
                    v.s[i] = 0.0;
                    a0[0] += ri * zi;
                    a0[1] += ri * ri;
                });
                st.vec += 8;
                st.fl += 5;
            }
            if (!team_sum(T, a0, d0)) return ST_TIMEOUT;
            double rz = d0[0];
            if (!(rz > 0.0)) break;                // nothing to do on this face
            if (mi == 0) ktol2 = fmax(C.ksp_rtol * C.ksp_rtol * d0[1], C.face_tol * C.face_tol);
            else if (d0[1] <= ktol2) break;        // the face gradient is small enough
            const double dd = delta * delta;
            double ss = 0.0;
            bool hit = false;
            for (;;) {
                double a1[3] = {0.0, 0.0, 0.0}, d1[3], o1[4];
                A.apply(R, v.p, [&](int64_t i, double ap) {
                    const double qi = v.fm[i] ? ap : 0.0, pi = v.p[i];
                    v.q[i] = qi;
                    a1[0] += pi * qi;
                    a1[1] += pi * pi;
                    a1[2] += v.s[i] * pi;
                });
                const double rzc = rz, ssc = ss;
                if (!team_sum_scalar(T, a1, d1, o1, [&](const double (&s)[3], double (&r)[4]) {
                        const double pq = s[0], pp = s[1], sp = s[2];
                        const double al = rzc / pq;
                        const bool curv = pq > 0.0;
                        const bool out = curv && ssc + al * (2.0 * sp + al * pp) >= dd;
                        // step to the boundary: the root tau >= 0 of |s + tau p|^2 = Delta^2
                        const double tau = (-sp + sqrt(fmax(sp * sp + pp * (dd - ssc), 0.0))) / pp;
                        r[0] = curv ? 1.0 : 0.0;
                        r[1] = out ? 1.0 : 0.0;
                        r[2] = al;
                        r[3] = tau;
                    }))
                    return ST_TIMEOUT;
                ++st.spmv;
                st.vec += 4;
                st.fl += 6;
                if (!flag_set(o1[0])) break;
                if (flag_set(o1[1])) {             // truncate on the trust-region boundary
                    const double tau = o1[3];
                    R.each([&](int64_t i) { v.s[i] += tau * v.p[i]; });
                    st.vec += 3;
                    st.fl += 2;
                    if (!T.sync()) return ST_TIMEOUT;
                    hit = true;
                    break;
                }
                const double al = o1[2];
                double a2[3] = {0.0, 0.0, 0.0}, d2[3];
                if (v.pc) {
                    R.each([&](int64_t i) {
                        const double si = v.s[i] + al * v.p[i];
                        const double ri = v.r[i] - al * v.q[i];
                        v.s[i] = si;
                        v.r[i] = ri;
                        a2[1] += ri * ri;
                        a2[2] += si * si;
                    });
                    if (!T.sync()) return ST_TIMEOUT;
                    if (!ssor_apply(T, *v.pc, v.fm, v.dinv, v.r, v.w, v.z,
                                    [&](int64_t i, double zi) { a2[0] += v.r[i] * zi; }))
                        return ST_TIMEOUT;
                    ++st.pc;
                    st.vec += 7;
                    st.fl += 10;
                } else {
                    R.each([&](int64_t i) {
                        const double si = v.s[i] + al * v.p[i];
                        const double ri = v.r[i] - al * v.q[i];
                        const double zi = v.dinv[i] * ri;
                        v.s[i] = si;
                        v.r[i] = ri;
                        v.z[i] = zi;
                        a2[0] += ri * zi;
                        a2[1] += ri * ri;
                        a2[2] += si * si;
                    });
                    st.vec += 8;
                    st.fl += 11;
                }
                if (!team_sum(T, a2, d2)) return ST_TIMEOUT;
                ++st.cg;
                ss = d2[2];
                if (d2[1] <= ktol2 || !(d2[0] > 0.0) || st.spmv >= C.max_spmv) break;
                const double beta = d2[0] / rz;
                rz = d2[0];
                R.each([&](int64_t i) { v.p[i] = v.z[i] + beta * v.p[i]; });
                st.vec += 3;
                st.fl += 2;
                if (!T.sync()) return ST_TIMEOUT;
            }
            // projected search along s
            double beta = 1.0;
            bool accepted = false;
            double d3[4];
            for (int ls = 0; ls < 48 && st.spmv < C.max_spmv; ++ls) {
                double a3[4] = {0.0, 0.0, 0.0, 0.0};
                R.each([&](int64_t i) {
                    const double xi = v.x[i];
                    const double wi = clampv(xi + beta * v.s[i], B.l(i), B.h(i));
                    v.w[i] = wi;
                    a3[0] += v.g[i] * (wi - xi);
                });
                if (!T.sync()) return ST_TIMEOUT;
                A.apply(R, v.w, [&](int64_t i, double aw) {
                    const double gwi = aw - v.b[i];
                    v.gw[i] = gwi;
                    const double wi = v.w[i], xi = v.x[i], l = B.l(i), h = B.h(i);
                    a3[1] += (v.g[i] + gwi) * (wi - xi);
                    const double gp = proj_grad(wi, gwi, l, h);
                    a3[2] += gp * gp;
                    a3[3] += ((wi <= l || wi >= h) && xi > l && xi < h) ? 1.0 : 0.0;   // newly active
                });
                double o3[1];
                if (!team_sum_scalar(T, a3, d3, o3, [&](const double (&s)[4], double (&r)[1]) {
                        r[0] = 0.5 * s[1] <= kTronMu0 * s[0] ? 1.0 : 0.0;
                    }))
                    return ST_TIMEOUT;
                ++st.spmv;
                st.vec += 7;
                st.fl += 12;
                if (flag_set(o3[0])) {
                    accepted = true;
                    break;
                }
                beta *= 0.5;
            }
            if (!accepted) break;
            double *t1 = v.x; v.x = v.w; v.w = t1;
            t1 = v.g; v.g = v.gw; v.gw = t1;
            st.gp2 = d3[2];
            if (d3[3] == 0.0 || hit) break;        // no new bound: back to a Cauchy step
        }
    }
    return status;
}

}  // namespace nnqp
