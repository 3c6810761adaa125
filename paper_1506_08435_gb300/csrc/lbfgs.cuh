// Projected limited-memory quasi-Newton method for the box QP
//     minimize 1/2 x'Ax - b'x  subject to  lo <= x <= hi
// in the manner of TAO's BLMVM (bounded limited-memory variable metric,
// Benson & More 2001; the solver the paper runs in Sec. 3.1 / Sec. 5):
// the step direction is d = -H gP with H the L-BFGS inverse-Hessian model
// built from the last m pairs (s, y) = (x+ - x, g+ - g), d is zeroed on the
// binding set, and x+ = P(x + alpha d) with alpha halved until the Armijo
// condition holds.  Pairs with s'y <= 1e-12 |s||y| are skipped.  H is
// applied in the compact form (lbfgs_small.h), so one iteration is two fused
// passes: direction + trial point -> product A w fused with the new pair and
// all dots that the model update and the next direction need.
#pragma once
#include "gpcg.cuh"
#include "lbfgs_small.h"

namespace nnqp {

constexpr int kLbMaxM = 6;   // pairs kept on the device (reductions are 5m+9 wide)

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

// Layout of the per-trial reduction (one per product).
constexpr int kLbW = 9 + 5 * kLbMaxM;
static_assert(kLbW <= kMaxRed, "L-BFGS reduction wider than the team reduction buffers");
enum : int {
    LB_GDX = 0,   // g'(w - x)                   (trial pass)
    LB_QD = 1,    // (g + gw)'s = 2 (q(w) - q(x))
    LB_GP2 = 2,   // ||gP(w)||^2
    LB_SY = 3,    // s'y
    LB_SS = 4,    // s's
    LB_YY = 5,    // y'y
    LB_GD = 6,    // gP(x)'d                     (trial pass, first trial)
    LB_SNG = 7,   // s'gP(w)
    LB_YNG = 8,   // y'gP(w)
    LB_X = 9,     // [j]: s'y_j, y_j's... : s y_j | s_j y | y y_j | s_j gP(w) | y_j gP(w)
};

// S, Y: (m+1) slots of n doubles each (one spare slot receives the trial pair).
// One iteration = (trial pass: direction on the first trial, trial point)
// -> barrier -> (product A w fused with the trial pair and every dot that the
// Armijo test, the pair update and the NEXT iteration's model need) ->
// reduction.  The model coefficients of the next iteration therefore come
// from the accepted trial's reduction, so an accepted first trial costs one
// barrier and one reduction per product.
template <class Team, class Op>
__device__ int lbfgs_solve(Team &T, const Rows &R, const Op &A, double lo, double hi, const double *b, double *&x,
                           double *&g, double *d, double *&w, double *&gw, double *S, double *Y, int64_t n,
                           const LbCtl &C, LbStats &st, LbSmem &sm) {
    const int m = C.m;
    int ord[kLbMaxM];
    int k = 0, spare = 0;
    double uv[2 * kLbMaxM];   // S_j'gP(x), Y_j'gP(x) for the pairs in ord
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
        // ---- model coefficients from u = S'gP, v = Y'gP (carried over)
        bool use_model = k > 0;
        if (use_model) {
            if (threadIdx.x == 0) {
                const double gamma = sm.SY[(k - 1) * kLbfgsMax + (k - 1)] / sm.YY[(k - 1) * kLbfgsMax + (k - 1)];
                sm.ok = lbfgs_coefficients(k, sm.SY, sm.YY, uv, uv + kLbMaxM, gamma, sm.cs, sm.cy) ? 1 : 0;
                sm.cs[kLbfgsMax - 1] = gamma;
            }
            __syncthreads();
            use_model = sm.ok != 0;
        }
        // ---- projected backtracking search along d = -H gP (zero on the binding set)
        double alpha = 1.0;
        bool accepted = false, have_d = false;
        double a[kLbW];
        for (int ls = 0; ls < 60; ++ls) {
#pragma unroll
            for (int q = 0; q < kLbW; ++q) a[q] = 0.0;
            const double gamma = use_model ? sm.cs[kLbfgsMax - 1] : C.h0;
            const int kk = use_model ? k : 0;
            const bool first = !have_d;
            R.each([&](int64_t i) {
                const double xi = x[i];
                double di;
                if (first) {
                    const double gp = proj_grad(xi, g[i], lo, hi);
                    double hg = gamma * gp;
#pragma unroll
                    for (int j = 0; j < kLbMaxM; ++j)
                        if (j < kk) hg += sm.cs[j] * S[(int64_t)ord[j] * n + i] + sm.cy[j] * Y[(int64_t)ord[j] * n + i];
                    const bool binding = (xi <= lo || xi >= hi) && gp == 0.0;
                    di = binding ? 0.0 : -hg;
                    d[i] = di;
                    a[LB_GD] += gp * di;
                } else {
                    di = d[i];
                }
                const double wi = clampv(xi + alpha * di, lo, hi);
                w[i] = wi;
                a[LB_GDX] += g[i] * (wi - xi);
            });
            st.vec += first ? 4 + 2 * kk : 4;
            if (!T.sync()) return ST_TIMEOUT;
            double *Sn = S + (int64_t)spare * n, *Yn = Y + (int64_t)spare * n;
            A.apply(R, w, [&](int64_t i, double aw) {
                const double gwi = aw - b[i];
                gw[i] = gwi;
                const double wi = w[i];
                const double si = wi - x[i], yi = gwi - g[i];
                Sn[i] = si;
                Yn[i] = yi;
                a[LB_QD] += (g[i] + gwi) * si;
                const double gp = proj_grad(wi, gwi, lo, hi);
                a[LB_GP2] += gp * gp;
                a[LB_SY] += si * yi;
                a[LB_SS] += si * si;
                a[LB_YY] += yi * yi;
                a[LB_SNG] += si * gp;
                a[LB_YNG] += yi * gp;
#pragma unroll
                for (int j = 0; j < kLbMaxM; ++j)
                    if (j < k) {
                        const double sj = S[(int64_t)ord[j] * n + i], yj = Y[(int64_t)ord[j] * n + i];
                        a[LB_X + j] += si * yj;
                        a[LB_X + kLbMaxM + j] += sj * yi;
                        a[LB_X + 2 * kLbMaxM + j] += yi * yj;
                        a[LB_X + 3 * kLbMaxM + j] += sj * gp;
                        a[LB_X + 4 * kLbMaxM + j] += yj * gp;
                    }
            });
            if (!T.reduce(a)) return ST_TIMEOUT;
            ++st.spmv;
            st.vec += 6 + 2 * k + 3;
            if (first) {
                have_d = true;
                if (!(a[LB_GD] < 0.0)) {
                    if (!use_model) return ST_NUMERIC;
                    use_model = false;   // not a descent direction: drop the memory
                    k = 0;
                    have_d = false;
                    ++st.resets;
                    continue;
                }
            }
            if (0.5 * a[LB_QD] <= C.mu * a[LB_GDX]) {
                accepted = true;
                break;
            }
            alpha *= 0.5;
            if (st.spmv >= C.max_spmv) break;
        }
        if (!accepted) return ST_NOT_CONVERGED;
        double *t = x; x = w; w = t;
        t = g; g = gw; gw = t;
        st.gp2 = a[LB_GP2];
        // ---- memory update; uv follows the pairs to their new positions
        if (a[LB_SY] > 1e-12 * sqrt(a[LB_SS] * a[LB_YY])) {
            const int drop = k == m ? 1 : 0;
            if (threadIdx.x == 0) {
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
                    sm.SY[kn * kLbfgsMax + j] = a[LB_X + oj];
                    sm.SY[j * kLbfgsMax + kn] = a[LB_X + kLbMaxM + oj];
                    sm.YY[kn * kLbfgsMax + j] = sm.YY[j * kLbfgsMax + kn] = a[LB_X + 2 * kLbMaxM + oj];
                }
                sm.SY[kn * kLbfgsMax + kn] = a[LB_SY];
                sm.YY[kn * kLbfgsMax + kn] = a[LB_YY];
            }
            __syncthreads();
            const int kn = k - drop;
#pragma unroll
            for (int j = 0; j < kLbMaxM; ++j)
                if (j < kn) {
                    uv[j] = a[LB_X + 3 * kLbMaxM + j + drop];
                    uv[kLbMaxM + j] = a[LB_X + 4 * kLbMaxM + j + drop];
                }
            uv[kn] = a[LB_SNG];
            uv[kLbMaxM + kn] = a[LB_YNG];
            if (drop) {
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
        } else {
#pragma unroll
            for (int j = 0; j < kLbMaxM; ++j)
                if (j < k) {
                    uv[j] = a[LB_X + 3 * kLbMaxM + j];
                    uv[kLbMaxM + j] = a[LB_X + 4 * kLbMaxM + j];
                }
        }
    }
}

}  // namespace nnqp
