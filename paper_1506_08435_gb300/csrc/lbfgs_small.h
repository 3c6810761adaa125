// Small dense algebra of the compact limited-memory BFGS representation
// (Byrd, Nocedal & Schnabel, Math. Prog. 63, 1994):
//     H = gamma I + [S  gamma Y] M [S^T; gamma Y^T],
//     M = [[R^-T (D + gamma Y^T Y) R^-1, -R^-T], [-R^-1, 0]],
// with S, Y the n x k matrices of the stored pairs (oldest first),
// R_ij = s_i^T y_j (i <= j, upper triangle of S^T Y), D = diag(s_i^T y_i).
// Given u = S^T g and v = Y^T g, H g = gamma g + S p - gamma Y t with
//     t = R^-1 u,   p = R^-T ((D + gamma Y^T Y) t - gamma v).
// Plain C++ usable from host and device code (k <= kLbfgsMax).
#pragma once

#if defined(__CUDACC__)
#define NN_HD __host__ __device__
#else
#define NN_HD
#endif

namespace nnqp {

constexpr int kLbfgsMax = 16;

// SY[i][j] = s_i^T y_j, YY[i][j] = y_i^T y_j (k x k, row stride kLbfgsMax).
// Outputs coefficients cs[k] (of S) and cy[k] (of Y) such that
// H g = gamma g + sum_j cs[j] s_j + sum_j cy[j] y_j.  Returns false if R is
// singular (then the caller falls back to a gradient step).
NN_HD inline bool lbfgs_coefficients(int k, const double *SY, const double *YY, const double *u,
                                     const double *v, double gamma, double *cs, double *cy) {
    double t[kLbfgsMax], w[kLbfgsMax], rinv[kLbfgsMax];
    // reciprocals of R's diagonal first: k independent divisions instead of
    // one division on every step of both substitution chains
    for (int i = 0; i < k; ++i) {
        const double rii = SY[i * kLbfgsMax + i];
        if (!(rii > 0.0)) return false;
        rinv[i] = 1.0 / rii;
    }
    // back substitution R t = u, R upper triangular with R_ij = SY[i][j]
    for (int i = k - 1; i >= 0; --i) {
        double s = u[i];
        for (int j = i + 1; j < k; ++j) s -= SY[i * kLbfgsMax + j] * t[j];
        t[i] = s * rinv[i];
    }
    // w = (D + gamma Y^T Y) t - gamma v
    for (int i = 0; i < k; ++i) {
        double s = SY[i * kLbfgsMax + i] * t[i] - gamma * v[i];
        for (int j = 0; j < k; ++j) s += gamma * YY[i * kLbfgsMax + j] * t[j];
        w[i] = s;
    }
    // forward substitution R^T p = w
    for (int i = 0; i < k; ++i) {
        double s = w[i];
        for (int j = 0; j < i; ++j) s -= SY[j * kLbfgsMax + i] * cs[j];
        cs[i] = s * rinv[i];
    }
    for (int i = 0; i < k; ++i) cy[i] = -gamma * t[i];
    return true;
}

}  // namespace nnqp
