// Projected limited-memory quasi-Newton method for the box QP
//     minimize 1/2 x'Ax - b'x  subject to  lo <= x <= hi
// in the manner of TAO's BLMVM (bounded limited-memory variable metric,
// Benson & More 2001; the solver the paper runs in Sec. 3.1 / Sec. 5):
// the step direction is d = -H gP with H the L-BFGS inverse-Hessian model
// built from the last m pairs (s, y) = (x+ - x, g+ - g), d is zeroed on the
// binding set, and x+ = P(x + alpha d) with alpha halved until the Armijo
// condition holds.  Pairs with s'y <= 1e-12 |s||y| are skipped.  H is
// applied in the compact form (lbfgs_small.h), so one iteration is a fixed
// number of fused passes: dots S'gP, Y'gP -> direction -> trial point ->
// product A w fused with the new pair and all dots the model update needs.
#pragma once
#include "gpcg.cuh"
#include "lbfgs_small.h"

namespace nnqp {

constexpr int kLbMaxM = 6;   // pairs kept on the device (reductions are 3m+6 wide)

struct LbSmem {
    double SY[kLbfgsMax * kLbfgsMax];
    double YY[kLbfgsMax * kLbfgsMax];
    double cs[kLbfgsMax], cy[kLbfgsMax];
    int ok;
};

struct LbCtl {
    double tol;
    int64_t max_spmv;
    int m;
    double mu;
    double h0;            // initial model scale (1 / ||A||_inf)
};

struct LbStats {
    int64_t spmv = 0, iters = 0, vec = 0, resets = 0;
    double gp2 = 0.0;
};

// S, Y: (m+1) slots of n doubles each (one spare slot receives the trial pair).
template <class Team, class Op>
__device__ int lbfgs_solve(Team &T, const Rows &R, const Op &A, double lo, double hi, const double *b, double *&x,
                           double *&g, double *d, double *&w, double *&gw, double *S, double *Y, int64_t n,
                           const LbCtl &C, LbStats &st, LbSmem &sm) {
    const int m = C.m;
    int ord[kLbMaxM];
    int k = 0, spare = 0;
    R.each([&](int64_t i) { x[i] = clampv(x[i], lo, hi); });
    st.vec += 2;
    if (!T.sync()) return ST_TIMEOUT;
    {
        double a[1] = {0.0};
        A.apply(R, x, [&](int64_t i, double ax) {
            const double gi = ax - b[i];
            g[i] = gi;
            const double gp = proj_grad(x[i], gi, lo, hi);
            a[0] += gp * gp;
        });
        if (!T.reduce(a)) return ST_TIMEOUT;
        ++st.spmv;
        st.vec += 1;
        st.gp2 = a[0];
    }
    const double tol2 = C.tol * C.tol;
    for (;;) {
        if (!isfinite(st.gp2)) return ST_NUMERIC;
        if (st.gp2 <= tol2) return ST_OK;
        if (st.spmv >= C.max_spmv) return ST_NOT_CONVERGED;
        ++st.iters;
        // ---- model coefficients from u = S'gP, v = Y'gP
        bool use_model = k > 0;
        if (use_model) {
            double a[2 * kLbMaxM] = {0.0};
            R.each([&](int64_t i) {
                const double gp = proj_grad(x[i], g[i], lo, hi);
#pragma unroll
                for (int j = 0; j < kLbMaxM; ++j)
                    if (j < k) {
                        a[j] += S[(int64_t)ord[j] * n + i] * gp;
                        a[kLbMaxM + j] += Y[(int64_t)ord[j] * n + i] * gp;
                    }
            });
            if (!T.reduce(a)) return ST_TIMEOUT;
            st.vec += 2 + 2 * k;
            if (threadIdx.x == 0) {
                const double gamma = sm.SY[(k - 1) * kLbfgsMax + (k - 1)] / sm.YY[(k - 1) * kLbfgsMax + (k - 1)];
                sm.ok = lbfgs_coefficients(k, sm.SY, sm.YY, a, a + kLbMaxM, gamma, sm.cs, sm.cy) ? 1 : 0;
                sm.cs[kLbfgsMax - 1] = gamma;
            }
            __syncthreads();
            use_model = sm.ok != 0;
        }
        // ---- direction d = -H gP, zero on the binding set; descent test
        double gd;
        for (int attempt = 0; attempt < 2; ++attempt) {
            const double gamma = use_model ? sm.cs[kLbfgsMax - 1] : C.h0;
            double a[1] = {0.0};
            R.each([&](int64_t i) {
                const double xi = x[i], gp = proj_grad(xi, g[i], lo, hi);
                double hg = gamma * gp;
                if (use_model) {
#pragma unroll
                    for (int j = 0; j < kLbMaxM; ++j)
                        if (j < k) hg += sm.cs[j] * S[(int64_t)ord[j] * n + i] + sm.cy[j] * Y[(int64_t)ord[j] * n + i];
                }
                const bool binding = (xi <= lo || xi >= hi) && gp == 0.0;
                const double di = binding ? 0.0 : -hg;
                d[i] = di;
                a[0] += gp * di;
            });
            if (!T.reduce(a)) return ST_TIMEOUT;
            st.vec += use_model ? 3 + 2 * k : 3;
            gd = a[0];
            if (gd < 0.0 || !use_model) break;
            use_model = false;   // not a descent direction: drop the memory
            k = 0;
            ++st.resets;
        }
        if (!(gd < 0.0)) return ST_NUMERIC;
        // ---- projected backtracking search
        double alpha = 1.0;
        bool accepted = false;
        double a[3 * kLbMaxM + 6];
        for (int ls = 0; ls < 60; ++ls) {
            for (int q = 0; q < 3 * kLbMaxM + 6; ++q) a[q] = 0.0;
            R.each([&](int64_t i) {
                const double xi = x[i];
                const double wi = clampv(xi + alpha * d[i], lo, hi);
                w[i] = wi;
                a[0] += g[i] * (wi - xi);
            });
            if (!T.sync()) return ST_TIMEOUT;
            double *Sn = S + (int64_t)spare * n, *Yn = Y + (int64_t)spare * n;
            A.apply(R, w, [&](int64_t i, double aw) {
                const double gwi = aw - b[i];
                gw[i] = gwi;
                const double wi = w[i];
                const double si = wi - x[i], yi = gwi - g[i];
                Sn[i] = si;
                Yn[i] = yi;
                a[1] += (g[i] + gwi) * si;
                const double gp = proj_grad(wi, gwi, lo, hi);
                a[2] += gp * gp;
                a[3] += si * yi;
                a[4] += si * si;
                a[5] += yi * yi;
#pragma unroll
                for (int j = 0; j < kLbMaxM; ++j)
                    if (j < k) {
                        const double sj = S[(int64_t)ord[j] * n + i], yj = Y[(int64_t)ord[j] * n + i];
                        a[6 + j] += si * yj;
                        a[6 + kLbMaxM + j] += sj * yi;
                        a[6 + 2 * kLbMaxM + j] += yi * yj;
                    }
            });
            if (!T.reduce(a)) return ST_TIMEOUT;
            ++st.spmv;
            st.vec += 6 + 2 * k + 3;
            if (0.5 * a[1] <= C.mu * a[0]) {
                accepted = true;
                break;
            }
            alpha *= 0.5;
            if (st.spmv >= C.max_spmv) break;
        }
        if (!accepted) return ST_NOT_CONVERGED;
        double *t = x; x = w; w = t;
        t = g; g = gw; gw = t;
        st.gp2 = a[2];
        // ---- memory update
        if (a[3] > 1e-12 * sqrt(a[4] * a[5])) {
            if (threadIdx.x == 0) {
                int drop = k == m ? 1 : 0;
                // new dots indexed by the old positions j; after a drop old j maps to j - 1
                if (drop)
                    for (int i = 0; i + 1 < k; ++i)
                        for (int j = 0; j + 1 < k; ++j) {
                            sm.SY[i * kLbfgsMax + j] = sm.SY[(i + 1) * kLbfgsMax + j + 1];
                            sm.YY[i * kLbfgsMax + j] = sm.YY[(i + 1) * kLbfgsMax + j + 1];
                        }
                const int kn = k - drop;   // old pairs kept
                for (int j = 0; j < kn; ++j) {
                    const int oj = j + drop;
                    sm.SY[kn * kLbfgsMax + j] = a[6 + oj];
                    sm.SY[j * kLbfgsMax + kn] = a[6 + kLbMaxM + oj];
                    sm.YY[kn * kLbfgsMax + j] = sm.YY[j * kLbfgsMax + kn] = a[6 + 2 * kLbMaxM + oj];
                }
                sm.SY[kn * kLbfgsMax + kn] = a[3];
                sm.YY[kn * kLbfgsMax + kn] = a[5];
            }
            __syncthreads();
            if (k == m) {
                const int old = ord[0];
                for (int j = 0; j + 1 < k; ++j) ord[j] = ord[j + 1];
                ord[k - 1] = spare;
                spare = old;
            } else {
                ord[k] = spare;
                ++k;
                // the spare slot is the lowest slot not in use
                for (int cand = 0; cand <= m; ++cand) {
                    bool used = false;
                    for (int j = 0; j < k; ++j) used |= ord[j] == cand;
                    if (!used) {
                        spare = cand;
                        break;
                    }
                }
            }
        }
    }
}

}  // namespace nnqp
