// Device assembly of the Galerkin system and the reduced QP.
//
//   mesh (structured generator or caller arrays)
//   -> node/element incidence (sorted by element id)
//   -> CSR pattern of the node graph (sorted unique columns per row)
//   -> element kernel: K_e = |e| G^T D_e G (upper triangle), |e|
//      (bilinear form B(w;c), Sec. 2.1.2; Jacobian F_{1,1} = D, Sec. 3.2;
//       D_e from the dispersion law, Sec. 5, when a cell velocity is given)
//   -> node-centric gather: every row sums its elements' contributions in
//      ascending element order (deterministic, no floating-point atomics);
//      M_e = |e|(1 + delta_ab)/((d+1)(d+2)) (capacity matrix, F_{0,0} = 1/dt,
//      Sec. 3.2) and F_e = f_e |e|/(d+1) in the same pass
//   -> Dirichlet elimination (Sec. 2.1, c = c^p on Gamma^D): free unknowns
//      in ascending node order, A = K_FF + M_FF/dt, b0 = F_F - K_FD c_D
//   -> SELL-32 copies (FP64 off-diagonals + diagonal, FP32 off-diagonals +
//      row sums for the mixed path, M_FF off-diagonals for transients).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include "internal.h"
#include "scan.cuh"
#include "ops.cuh"

namespace nnqp {

constexpr int kMaxCand = 256;   // element-vertex incidences gathered per row
constexpr int kMaxRow = 64;     // nonzeros per row of the node graph
constexpr int TPB = 256;

__device__ __forceinline__ void set_status(int *st, int code) { atomicCAS(st, 0, code); }

static inline unsigned nblk(int64_t n, int t = TPB) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ mesh

__global__ void k_coords(int dim, int nx, int ny, int nz, int64_t N, double *coords) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int64_t sx = nx + 1, sy = ny + 1;
    const int64_t i = v % sx, j = (v / sx) % sy, k = v / (sx * sy);
    coords[v * dim + 0] = (double)i / (double)nx;
    coords[v * dim + 1] = (double)j / (double)ny;
    if (dim == 3) coords[v * 3 + 2] = (double)k / (double)nz;
}

__global__ void k_conn2d(int nx, int ny, int32_t *conn) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)nx * ny) return;
    const int i = (int)(q % nx), j = (int)(q / nx);
    const int32_t v00 = i + (nx + 1) * j, v10 = v00 + 1, v01 = v00 + nx + 1, v11 = v01 + 1;
    int32_t *t = conn + 6 * q;
    t[0] = v00; t[1] = v10; t[2] = v11;
    t[3] = v00; t[4] = v11; t[5] = v01;
}

__global__ void k_conn3d(int nx, int ny, int nz, int32_t *conn) {
    int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= (int64_t)nx * ny * nz) return;
    const int64_t i = h % nx, j = (h / nx) % ny, k = h / ((int64_t)nx * ny);
    const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
    const int64_t step[3] = {1, sy, sz};
    // axis permutations in lexicographic order
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int64_t v0 = i + sy * j + sz * k;
    int32_t *t = conn + 24 * h;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        int64_t v = v0;
        t[4 * p] = (int32_t)v;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            v += step[perm[p][s]];
            t[4 * p + 1 + s] = (int32_t)v;
        }
    }
}

// ------------------------------------------------------------------ validation

__global__ void k_check_nodes(int64_t N, const uint8_t *dmask, const double *dval, double lo, double hi, int *st) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= N || !dmask[v]) return;
    double c = dval[v];
    if (!(c == c)) set_status(st, NN_ERR_NUMERIC);
    else if (c < lo || c > hi) set_status(st, NN_ERR_INFEASIBLE);
}

__global__ void k_check_conn(int64_t E, int nv, const int32_t *conn, int64_t N, int *st) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= E * nv) return;
    int32_t v = conn[q];
    if (v < 0 || v >= N) set_status(st, NN_ERR_INVALID_ARG);
}

// ------------------------------------------------------------------ incidence

__global__ void k_inc_count(int64_t E, int nv, const int32_t *conn, int64_t N, unsigned long long *cnt) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= E * nv) return;
    int32_t v = conn[q];
    if (v >= 0 && v < N) atomicAdd(cnt + v, 1ULL);
}

__global__ void k_inc_fill(int64_t E, int nv, const int32_t *conn, int64_t N, const int64_t *ptr,
                           unsigned long long *fill, int32_t *inc) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= E * nv) return;
    int32_t v = conn[q];
    if (v < 0 || v >= N) return;
    unsigned long long k = atomicAdd(fill + v, 1ULL);
    inc[ptr[v] + (int64_t)k] = (int32_t)q;   // q = e*nv + a
}

// Sort each node's incidence list by (element, local vertex).
__global__ void k_inc_sort(int64_t N, const int64_t *ptr, int32_t *inc) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= N) return;
    int32_t *a = inc + ptr[v];
    const int64_t m = ptr[v + 1] - ptr[v];
    for (int64_t i = 1; i < m; ++i) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = x;
    }
}

// ------------------------------------------------------------------ pattern

// Pass 0 writes the unique column count of every row; pass 1 writes the
// sorted columns at rowptr.
__global__ void k_pattern(int64_t N, int nv, const int32_t *conn, const int64_t *iptr, const int32_t *inc,
                          int pass, const int64_t *rowptr, int64_t *rowcnt, int32_t *col, int *st) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= N) return;
    int32_t cand[kMaxCand];
    int m = 0;
    for (int64_t q = iptr[v]; q < iptr[v + 1]; ++q) {
        const int64_t e = inc[q] / nv;
        for (int b = 0; b < nv; ++b) {
            if (m == kMaxCand) {
                set_status(st, NN_ERR_INVALID_ARG);
                return;
            }
            cand[m++] = conn[e * nv + b];
        }
    }
    if (m == 0) cand[m++] = (int32_t)v;   // isolated node keeps its diagonal
    for (int i = 1; i < m; ++i) {
        int32_t x = cand[i];
        int j = i - 1;
        while (j >= 0 && cand[j] > x) {
            cand[j + 1] = cand[j];
            --j;
        }
        cand[j + 1] = x;
    }
    int u = 0;
    for (int i = 0; i < m; ++i)
        if (i == 0 || cand[i] != cand[i - 1]) cand[u++] = cand[i];
    if (u > kMaxRow) {
        set_status(st, NN_ERR_INVALID_ARG);
        return;
    }
    if (pass == 0) {
        rowcnt[v] = u;
    } else {
        int32_t *c = col + rowptr[v];
        for (int i = 0; i < u; ++i) c[i] = cand[i];
    }
}

// ------------------------------------------------------------------ element kernel

__device__ __forceinline__ int tri_index(int a, int b, int nv) {  // a <= b, packed upper triangle
    return a * nv - (a * (a - 1)) / 2 + (b - a);
}

// K_e (packed upper triangle, nv(nv+1)/2 values) and |e| of every element.
__global__ void __launch_bounds__(TPB) k_element(int64_t E, int dim, const double *__restrict__ coords,
                                                 const int32_t *__restrict__ conn, int kind,
                                                 const double *__restrict__ coef, double aL, double aT, double DM,
                                                 double *__restrict__ Ke, double *__restrict__ vol, int *st) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int nv = dim + 1, nk = nv * (nv + 1) / 2;
    double X[4][3];
    for (int a = 0; a < nv; ++a)
        for (int p = 0; p < dim; ++p) X[a][p] = coords[(int64_t)conn[e * nv + a] * dim + p];
    // Jacobian J[p][k] = (x_{k+1} - x_0)_p; the gradient of the barycentric
    // coordinate k+1 is row k of J^{-1}; that of vertex 0 is minus their sum.
    double G[4][3], det, J[3][3], Ji[3][3];
    for (int p = 0; p < dim; ++p)
        for (int k = 0; k < dim; ++k) J[p][k] = X[k + 1][p] - X[0][p];
    double fact;
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det;
        Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det;
        Ji[1][1] = J[0][0] / det;
        fact = 2.0;
    } else {
        const double m00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double m01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double m02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * m00 + J[0][1] * m01 + J[0][2] * m02;
        // inverse = transpose of the cofactor matrix / det
        Ji[0][0] = m00 / det;
        Ji[1][0] = m01 / det;
        Ji[2][0] = m02 / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        fact = 6.0;
    }
    if (det == 0.0 || !isfinite(det)) {
        set_status(st, NN_ERR_DEGENERATE);
        return;
    }
    for (int p = 0; p < dim; ++p) {
        double s = 0.0;
        for (int k = 0; k < dim; ++k) {
            G[k + 1][p] = Ji[k][p];
            s += Ji[k][p];
        }
        G[0][p] = -s;
    }
    // element diffusivity
    double D[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (kind == NN_COEF_TENSOR) {
        const double *c = coef + e * (dim == 2 ? 3 : 6);
        for (int q = 0; q < (dim == 2 ? 3 : 6); ++q)
            if (!isfinite(c[q])) {
                set_status(st, NN_ERR_NUMERIC);
                return;
            }
        if (dim == 2) {
            D[0][0] = c[0]; D[0][1] = D[1][0] = c[1]; D[1][1] = c[2];
        } else {
            D[0][0] = c[0]; D[0][1] = D[1][0] = c[1]; D[0][2] = D[2][0] = c[2];
            D[1][1] = c[3]; D[1][2] = D[2][1] = c[4]; D[2][2] = c[5];
        }
    } else {
        const double *vv = coef + e * dim;
        double n2 = 0.0;
        for (int p = 0; p < dim; ++p) {
            if (!isfinite(vv[p])) {
                set_status(st, NN_ERR_NUMERIC);
                return;
            }
            n2 += vv[p] * vv[p];
        }
        const double vn = sqrt(n2);
        const double iso = aT * vn + DM;
        const double lon = vn > 0.0 ? (aL - aT) / vn : 0.0;
        for (int p = 0; p < dim; ++p)
            for (int q = 0; q < dim; ++q) D[p][q] = lon * vv[p] * vv[q] + (p == q ? iso : 0.0);
    }
    // symmetric positive definite: leading principal minors > 0
    const double d1 = D[0][0], d2 = D[0][0] * D[1][1] - D[0][1] * D[1][0];
    bool spd = d1 > 0.0 && d2 > 0.0;
    if (dim == 3 && spd) {
        const double d3 = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                          D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                          D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
        spd = d3 > 0.0;
    }
    if (!spd) {
        set_status(st, NN_ERR_NOT_SPD);
        return;
    }
    const double v = fabs(det) / fact;
    // DG[b][p] = sum_q D[p][q] G[b][q]
    double DG[4][3];
    for (int b = 0; b < nv; ++b)
        for (int p = 0; p < dim; ++p) {
            double s = 0.0;
            for (int q = 0; q < dim; ++q) s += D[p][q] * G[b][q];
            DG[b][p] = s;
        }
    double *out = Ke + e * nk;
    for (int a = 0; a < nv; ++a)
        for (int b = a; b < nv; ++b) {
            double s = 0.0;
            for (int p = 0; p < dim; ++p) s += G[a][p] * DG[b][p];
            out[tri_index(a, b, nv)] = v * s;
        }
    vol[e] = v;
}

// Row r of K, M and F: contributions of the elements around node r, summed
// in ascending element order.  M is the consistent P1 capacity matrix
// |e|(1 + delta_ab)/((d+1)(d+2)), or with lumped != 0 its row-sum lumping
// |e| delta_ab/(d+1).
__global__ void __launch_bounds__(TPB) k_gather(int64_t N, int nv, const int32_t *__restrict__ conn,
                                                const int64_t *__restrict__ iptr, const int32_t *__restrict__ inc,
                                                const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                const double *__restrict__ Ke, const double *__restrict__ vol,
                                                const double *__restrict__ f_elem, double *__restrict__ Kval,
                                                double *__restrict__ Mval, double *__restrict__ F, int lumped) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int nk = nv * (nv + 1) / 2;
    const double md = lumped ? 1.0 / nv : 2.0 / (nv * (nv + 1)), mo = lumped ? 0.0 : 1.0 / (nv * (nv + 1));
    const int64_t r0 = rowptr[r];
    const int len = (int)(rowptr[r + 1] - r0);
    int32_t cols[kMaxRow];
    double ak[kMaxRow], am[kMaxRow];
    for (int k = 0; k < len; ++k) {
        cols[k] = col[r0 + k];
        ak[k] = 0.0;
        am[k] = 0.0;
    }
    double fr = 0.0;
    for (int64_t q = iptr[r]; q < iptr[r + 1]; ++q) {
        const int32_t code = inc[q];
        const int64_t e = code / nv;
        const int a = code - (int)(e * nv);
        const double ve = vol[e];
        for (int b = 0; b < nv; ++b) {
            const int32_t c = conn[e * nv + b];
            int pos = 0;
            while (pos < len && cols[pos] != c) ++pos;
            if (pos == len) continue;  // cannot happen for a pattern built from conn
            const int lo = a < b ? a : b, hi = a < b ? b : a;
            ak[pos] += Ke[e * nk + tri_index(lo, hi, nv)];
            am[pos] += ve * (a == b ? md : mo);
        }
        if (f_elem) fr += f_elem[e] * ve / nv;
    }
    for (int k = 0; k < len; ++k) {
        Kval[r0 + k] = ak[k];
        if (Mval) Mval[r0 + k] = am[k];
    }
    F[r] = fr;
}

// ------------------------------------------------------------------ elimination

__global__ void k_free_flags(int64_t N, const uint8_t *dmask, int64_t *flag) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < N) flag[v] = dmask[v] ? 0 : 1;
}

__global__ void k_free_map(int64_t N, const uint8_t *dmask, const int64_t *fscan, int32_t *free_node,
                           int32_t *free_id) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= N) return;
    if (dmask[v]) {
        free_id[v] = -1;
    } else {
        free_id[v] = (int32_t)fscan[v];
        free_node[fscan[v]] = (int32_t)v;
    }
}

__global__ void k_red_count(int64_t NF, const int32_t *free_node, const int64_t *rowptr, const int32_t *col,
                            const uint8_t *dmask, int64_t *cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= NF) return;
    const int32_t v = free_node[i];
    int64_t c = 0;
    for (int64_t q = rowptr[v]; q < rowptr[v + 1]; ++q) c += dmask[col[q]] ? 0 : 1;
    cnt[i] = c;
}

// Reduced CSR row, lifting, diagonal, row sums, |row| sums, off-diagonal count.
__global__ void k_red_fill(int64_t NF, const int32_t *free_node, const int32_t *free_id, const int64_t *rowptr,
                           const int32_t *col, const double *Kval, const double *Mval, double inv_dt,
                           const double *F, const double *dval, const uint8_t *dmask, const int64_t *arow,
                           int32_t *acol, double *aval, double *amval, double *b0, double *diag, double *mdiag,
                           double *rsum, double *rabs, int64_t *offcnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= NF) return;
    const int32_t v = free_node[i];
    int64_t o = arow[i];
    double lift = 0.0, rs = 0.0, ra = 0.0, dg = 0.0, mdg = 0.0;
    for (int64_t q = rowptr[v]; q < rowptr[v + 1]; ++q) {
        const int32_t c = col[q];
        const double k = Kval[q];
        if (dmask[c]) {
            lift += k * dval[c];
            continue;
        }
        const double m = Mval ? Mval[q] : 0.0;
        const double a = Mval ? k + m * inv_dt : k;
        acol[o] = free_id[c];
        aval[o] = a;
        if (amval) amval[o] = m;
        if (c == v) {
            dg = a;
            mdg = m;
        }
        rs += a;
        ra += fabs(a);
        ++o;
    }
    b0[i] = F[v] - lift;
    diag[i] = dg;
    if (mdiag) mdiag[i] = mdg;
    rsum[i] = rs;
    rabs[i] = ra;
    offcnt[i] = (o - arow[i]) - 1;
}

__global__ void k_slice_width(int64_t NF, int64_t nslices, const int64_t *offcnt, int64_t *wslots) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int64_t w = 0;
    for (int l = 0; l < 32; ++l) {
        int64_t i = s * 32 + l;
        if (i < NF && offcnt[i] > w) w = offcnt[i];
    }
    wslots[s] = 32 * (w + (w & 1));   // even width: entries are stored in pairs
}

// One thread per slot row: writes the row's off-diagonals into its SELL
// column (and pads with the row's own index and 0).
__global__ void k_sell_fill(int64_t NF, int64_t nslices, const int64_t *arow, const int32_t *acol,
                            const double *aval, const double *amval, const double *rsum, const int64_t *sptr,
                            int32_t *scol, double *sval, float *sval32, double *smval, float *rsum32,
                            float *dinv32, double *dinv64, const double *diag) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nslices * 32) return;
    const int64_t s = t >> 5;
    const int lane = (int)(t & 31);
    const int64_t base = sptr[s];
    const int w = (int)((sptr[s + 1] - base) >> 5);
    if (t >= NF) {
        for (int k = 0; k < w; ++k) {
            const int64_t idx = sell_idx(base, k, lane);
            scol[idx] = 0;
            sval[idx] = 0.0;
            if (sval32) sval32[idx] = 0.0f;
            if (smval) smval[idx] = 0.0;
        }
        return;
    }
    int k = 0;
    double off32sum = 0.0;
    for (int64_t q = arow[t]; q < arow[t + 1]; ++q) {
        if (acol[q] == t) continue;
        const int64_t idx = sell_idx(base, k, lane);
        scol[idx] = acol[q];
        sval[idx] = aval[q];
        if (sval32) {
            const float f = (float)aval[q];
            sval32[idx] = f;
            off32sum += (double)f;
        }
        if (smval) smval[idx] = amval[q];
        ++k;
    }
    for (; k < w; ++k) {
        const int64_t idx = sell_idx(base, k, lane);
        scol[idx] = (int32_t)t;
        sval[idx] = 0.0;
        if (sval32) sval32[idx] = 0.0f;
        if (smval) smval[idx] = 0.0;
    }
    dinv64[t] = 1.0 / diag[t];
    if (sval32) {
        rsum32[t] = (float)rsum[t];
        dinv32[t] = (float)(1.0 / (rsum[t] - off32sum));
    }
}

__global__ void k_fill_dval(int64_t N, const uint8_t *dmask, const double *dv, double *out) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < N) out[v] = dmask[v] ? dv[v] : 0.0;
}

// ------------------------------------------------------------------ host orchestration

namespace {

struct Temp {
    DevArena a;
    cudaStream_t st;
    ~Temp() { a.release(st); }
};

template <typename T>
nn_status to_device(const T *src, size_t count, int memory, T **dst, DevArena &arena, cudaStream_t st) {
    NN_TRY(arena.alloc(dst, count, st));
    cudaMemcpyKind kind = memory == NN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    NN_CUDA_TRY(cudaMemcpyAsync(*dst, src, count * sizeof(T), kind, st));
    return NN_OK;
}

template <typename T>
nn_status read_scalar(const T *dptr, T *h, cudaStream_t st) {
    NN_CUDA_TRY(cudaMemcpyAsync(h, dptr, sizeof(T), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    return NN_OK;
}

nn_status check_status(int *d_status, cudaStream_t st, const char *stage) {
    int h = 0;
    NN_TRY(read_scalar(d_status, &h, st));
    if (h != 0) {
        const char *what = h == NN_ERR_INVALID_ARG    ? "invalid connectivity or node degree above the limit"
                           : h == NN_ERR_INFEASIBLE   ? "a Dirichlet value lies outside [lo, hi]"
                           : h == NN_ERR_NOT_SPD      ? "an element diffusivity is not symmetric positive definite"
                           : h == NN_ERR_DEGENERATE   ? "an element has zero measure"
                           : h == NN_ERR_NUMERIC      ? "NaN or Inf in the input"
                                                      : "device check failed";
        set_error("nn_assemble (%s): %s", stage, what);
        return (nn_status)h;
    }
    return NN_OK;
}

}  // namespace

nn_status assemble_impl(const nn_problem *p, const nn_assemble_opts *o, cudaStream_t st, nn_system **out) {
    *out = nullptr;
    if (!p) {
        set_error("nn_assemble: problem is NULL");
        return NN_ERR_INVALID_ARG;
    }
    const int dim = p->dim;
    if (dim != 2 && dim != 3) {
        set_error("nn_assemble: dim must be 2 or 3 (got %d)", dim);
        return NN_ERR_INVALID_ARG;
    }
    if (p->memory != NN_MEM_HOST && p->memory != NN_MEM_DEVICE) {
        set_error("nn_assemble: memory flag must be NN_MEM_HOST or NN_MEM_DEVICE");
        return NN_ERR_INVALID_ARG;
    }
    if (std::isnan(p->lo) || std::isnan(p->hi) || p->lo > p->hi || p->lo == INFINITY || p->hi == -INFINITY) {
        set_error("nn_assemble: bounds must satisfy lo <= hi (lo=%g, hi=%g)", p->lo, p->hi);
        return NN_ERR_INFEASIBLE;
    }
    if (!(p->dt >= 0.0) || std::isinf(p->dt)) {
        set_error("nn_assemble: dt must be finite and >= 0");
        return NN_ERR_INVALID_ARG;
    }
    if (o->lumped_mass != 0 && o->lumped_mass != 1) {
        set_error("nn_assemble: lumped_mass must be 0 or 1 (got %d)", o->lumped_mass);
        return NN_ERR_INVALID_ARG;
    }
    if (p->coef_kind != NN_COEF_TENSOR && p->coef_kind != NN_COEF_VELOCITY) {
        set_error("nn_assemble: unknown coef_kind %d", p->coef_kind);
        return NN_ERR_INVALID_ARG;
    }
    if (!p->coef || !p->dirichlet_mask || !p->dirichlet_value) {
        set_error("nn_assemble: coef, dirichlet_mask and dirichlet_value are required");
        return NN_ERR_INVALID_ARG;
    }
    const bool structured = p->coords == nullptr;
    int64_t N, E;
    if (structured) {
        if (p->nx < 1 || p->ny < 1 || (dim == 3 && p->nz < 1) || p->nx > 100000 || p->ny > 100000 ||
            p->nz > 100000) {
            set_error("nn_assemble: structured sizes must be >= 1");
            return NN_ERR_INVALID_ARG;
        }
        NN_TRY(nn_mesh_counts(dim, p->nx, p->ny, p->nz, &N, &E));
    } else {
        N = p->n_nodes;
        E = p->n_elems;
        if (N < 1 || E < 1 || !p->conn) {
            set_error("nn_assemble: explicit mesh needs n_nodes, n_elems >= 1 and conn");
            return NN_ERR_INVALID_ARG;
        }
    }
    const int nv = dim + 1;
    if (N >= (1LL << 31) || E * nv >= (1LL << 31)) {
        set_error("nn_assemble: mesh too large for 32-bit node/incidence ids");
        return NN_ERR_INVALID_ARG;
    }
    nn_system *s = new nn_system();
    s->dim = dim;
    s->N = N;
    s->E = E;
    s->lo = p->lo;
    s->hi = p->hi;
    s->dt = p->dt;
    Temp T;
    T.st = st;
    auto fail = [&](nn_status code) {
        s->arena.release(st);
        delete s;
        return code;
    };
#define TRYF(expr)                         \
    do {                                   \
        nn_status _q = (expr);             \
        if (_q != NN_OK) return fail(_q);  \
    } while (0)
#define CUF(expr)                                                                                   \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) {                                                                    \
            set_error("%s: %s", #expr, cudaGetErrorString(_e));                                     \
            return fail(_e == cudaErrorMemoryAllocation ? NN_ERR_OOM : NN_ERR_CUDA);                \
        }                                                                                           \
    } while (0)

    int *d_status;
    TRYF(T.a.alloc(&d_status, 1, st));
    CUF(cudaMemsetAsync(d_status, 0, sizeof(int), st));

    // ---- mesh
    TRYF(s->arena.alloc(&s->coords, (size_t)N * dim, st));
    TRYF(s->arena.alloc(&s->conn, (size_t)E * nv, st));
    if (structured) {
        (k_coords<<<nblk(N), TPB, 0, st>>>(dim, p->nx, p->ny, dim == 3 ? p->nz : 1, N, s->coords), ::nnqp::count_launch());
        if (dim == 2) (k_conn2d<<<nblk((int64_t)p->nx * p->ny), TPB, 0, st>>>(p->nx, p->ny, s->conn), ::nnqp::count_launch());
        else (k_conn3d<<<nblk((int64_t)p->nx * p->ny * p->nz), TPB, 0, st>>>(p->nx, p->ny, p->nz, s->conn), ::nnqp::count_launch());
    } else {
        cudaMemcpyKind kind = p->memory == NN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CUF(cudaMemcpyAsync(s->coords, p->coords, sizeof(double) * N * dim, kind, st));
        CUF(cudaMemcpyAsync(s->conn, p->conn, sizeof(int32_t) * E * nv, kind, st));
        (k_check_conn<<<nblk(E * nv), TPB, 0, st>>>(E, nv, s->conn, N, d_status), ::nnqp::count_launch());
    }
    // ---- inputs
    const int ncoef = p->coef_kind == NN_COEF_TENSOR ? (dim == 2 ? 3 : 6) : dim;
    double *coef, *fel = nullptr;
    TRYF(to_device(p->coef, (size_t)E * ncoef, p->memory, &coef, T.a, st));
    if (p->f_elem) TRYF(to_device(p->f_elem, (size_t)E, p->memory, &fel, T.a, st));
    uint8_t *dmask_in;
    double *dval_in;
    TRYF(to_device(p->dirichlet_mask, (size_t)N, p->memory, &dmask_in, T.a, st));
    TRYF(to_device(p->dirichlet_value, (size_t)N, p->memory, &dval_in, T.a, st));
    TRYF(s->arena.alloc(&s->dmask, N, st));
    TRYF(s->arena.alloc(&s->dval, N, st));
    // normalise the mask to 0/1
    CUF(cudaMemcpyAsync(s->dmask, dmask_in, N, cudaMemcpyDeviceToDevice, st));
    (k_fill_dval<<<nblk(N), TPB, 0, st>>>(N, s->dmask, dval_in, s->dval), ::nnqp::count_launch());
    (k_check_nodes<<<nblk(N), TPB, 0, st>>>(N, s->dmask, s->dval, p->lo, p->hi, d_status), ::nnqp::count_launch());

    // ---- incidence
    int64_t *iptr, *scratch;
    unsigned long long *cnt;
    int32_t *inc;
    const size_t stmp = scan_tmp_elems(std::max<int64_t>(N, 1) + 1) + 64;
    TRYF(T.a.alloc(&scratch, stmp, st));
    TRYF(T.a.alloc(&cnt, N, st));
    TRYF(T.a.alloc(&iptr, N + 1, st));
    TRYF(T.a.alloc(&inc, (size_t)E * nv, st));
    CUF(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * N, st));
    (k_inc_count<<<nblk(E * nv), TPB, 0, st>>>(E, nv, s->conn, N, cnt), ::nnqp::count_launch());
    CUF(exclusive_scan((const int64_t *)cnt, iptr, N, scratch, st));
    CUF(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * N, st));
    (k_inc_fill<<<nblk(E * nv), TPB, 0, st>>>(E, nv, s->conn, N, iptr, cnt, inc), ::nnqp::count_launch());
    (k_inc_sort<<<nblk(N), TPB, 0, st>>>(N, iptr, inc), ::nnqp::count_launch());
    TRYF(check_status(d_status, st, "mesh"));

    // ---- pattern
    int64_t *rowcnt;
    TRYF(T.a.alloc(&rowcnt, N, st));
    TRYF(s->arena.alloc(&s->rowptr, N + 1, st));
    (k_pattern<<<nblk(N), TPB, 0, st>>>(N, nv, s->conn, iptr, inc, 0, nullptr, rowcnt, nullptr, d_status), ::nnqp::count_launch());
    CUF(exclusive_scan(rowcnt, s->rowptr, N, scratch, st));
    int64_t nnz = 0;
    TRYF(read_scalar(s->rowptr + N, &nnz, st));
    TRYF(check_status(d_status, st, "pattern"));
    s->nnz = nnz;
    TRYF(s->arena.alloc(&s->col, nnz, st));
    (k_pattern<<<nblk(N), TPB, 0, st>>>(N, nv, s->conn, iptr, inc, 1, s->rowptr, nullptr, s->col, d_status), ::nnqp::count_launch());

    // ---- element matrices and gather
    const int nk = nv * (nv + 1) / 2;
    double *Ke, *vol;
    TRYF(T.a.alloc(&Ke, (size_t)E * nk, st));
    TRYF(T.a.alloc(&vol, E, st));
    (k_element<<<nblk(E), TPB, 0, st>>>(E, dim, s->coords, s->conn, p->coef_kind, coef, p->alpha_L, p->alpha_T,
                                         p->D_M, Ke, vol, d_status), ::nnqp::count_launch());
    const bool transient = p->dt > 0.0;
    TRYF(s->arena.alloc(&s->Kval, nnz, st));
    if (transient || o->keep_full) TRYF(s->arena.alloc(&s->Mval, nnz, st));
    TRYF(s->arena.alloc(&s->F, N, st));
    (k_gather<<<nblk(N), TPB, 0, st>>>(N, nv, s->conn, iptr, inc, s->rowptr, s->col, Ke, vol, fel, s->Kval,
                                        s->Mval, s->F, o->lumped_mass), ::nnqp::count_launch());
    TRYF(check_status(d_status, st, "elements"));

    // ---- elimination
    int64_t *flag, *fscan;
    int32_t *free_id;
    TRYF(T.a.alloc(&flag, N, st));
    TRYF(T.a.alloc(&fscan, N + 1, st));
    TRYF(T.a.alloc(&free_id, N, st));
    (k_free_flags<<<nblk(N), TPB, 0, st>>>(N, s->dmask, flag), ::nnqp::count_launch());
    CUF(exclusive_scan(flag, fscan, N, scratch, st));
    int64_t NF = 0;
    TRYF(read_scalar(fscan + N, &NF, st));
    s->NF = NF;
    if (NF == 0) {
        set_error("nn_assemble: every node is a Dirichlet node (no unknowns)");
        return fail(NN_ERR_INVALID_ARG);
    }
    TRYF(s->arena.alloc(&s->free_node, NF, st));
    (k_free_map<<<nblk(N), TPB, 0, st>>>(N, s->dmask, fscan, s->free_node, free_id), ::nnqp::count_launch());
    int64_t *rcnt;
    TRYF(T.a.alloc(&rcnt, NF, st));
    TRYF(s->arena.alloc(&s->arow, NF + 1, st));
    (k_red_count<<<nblk(NF), TPB, 0, st>>>(NF, s->free_node, s->rowptr, s->col, s->dmask, rcnt), ::nnqp::count_launch());
    int64_t *scratch2;
    TRYF(T.a.alloc(&scratch2, scan_tmp_elems(NF + 1) + 64, st));
    CUF(exclusive_scan(rcnt, s->arow, NF, scratch2, st));
    int64_t nnzF = 0;
    TRYF(read_scalar(s->arow + NF, &nnzF, st));
    s->nnzF = nnzF;
    TRYF(s->arena.alloc(&s->acol, nnzF, st));
    TRYF(s->arena.alloc(&s->aval, nnzF, st));
    double *amval = nullptr, *rsum, *rabs;
    int64_t *offcnt;
    if (transient) TRYF(T.a.alloc(&amval, nnzF, st));
    TRYF(s->arena.alloc(&s->b0, NF, st));
    TRYF(s->arena.alloc(&s->diag64, NF, st));
    TRYF(s->arena.alloc(&s->dinv64, NF, st));
    if (transient) TRYF(s->arena.alloc(&s->mdiag64, NF, st));
    TRYF(T.a.alloc(&rsum, NF, st));
    TRYF(T.a.alloc(&rabs, NF, st));
    TRYF(T.a.alloc(&offcnt, NF, st));
    (k_red_fill<<<nblk(NF), TPB, 0, st>>>(NF, s->free_node, free_id, s->rowptr, s->col, s->Kval,
                                          transient ? s->Mval : nullptr, transient ? 1.0 / p->dt : 0.0, s->F,
                                          s->dval, s->dmask, s->arow, s->acol, s->aval, amval, s->b0, s->diag64,
                                          s->mdiag64, rsum, rabs, offcnt), ::nnqp::count_launch());

    // ---- SELL-32
    const int64_t nslices = (NF + 31) / 32;
    int64_t *wslots;
    TRYF(T.a.alloc(&wslots, nslices, st));
    int64_t *sptr;
    TRYF(s->arena.alloc(&sptr, nslices + 1, st));
    (k_slice_width<<<nblk(nslices), TPB, 0, st>>>(NF, nslices, offcnt, wslots), ::nnqp::count_launch());
    int64_t *scratch3;
    TRYF(T.a.alloc(&scratch3, scan_tmp_elems(nslices + 1) + 64, st));
    CUF(exclusive_scan(wslots, sptr, nslices, scratch3, st));
    int64_t stored = 0;
    TRYF(read_scalar(sptr + nslices, &stored, st));
    s->A64.n = NF;
    s->A64.nslices = nslices;
    s->A64.stored = stored;
    s->A64.sptr = sptr;
    TRYF(s->arena.alloc(&s->A64.col, stored, st));
    TRYF(s->arena.alloc(&s->A64.val, stored, st));
    const bool mixed = o->build_mixed != 0;
    if (mixed) {
        s->A32.n = NF;
        s->A32.nslices = nslices;
        s->A32.stored = stored;
        s->A32.sptr = sptr;
        s->A32.col = s->A64.col;
        TRYF(s->arena.alloc(&s->A32.val, stored, st));
        TRYF(s->arena.alloc(&s->rsum32, NF, st));
        TRYF(s->arena.alloc(&s->dinv32, NF, st));
        s->has_mixed = true;
    }
    if (transient) {
        s->M64.n = NF;
        s->M64.nslices = nslices;
        s->M64.stored = stored;
        s->M64.sptr = sptr;
        s->M64.col = s->A64.col;
        TRYF(s->arena.alloc(&s->M64.val, stored, st));
    }
    (k_sell_fill<<<nblk(nslices * 32), TPB, 0, st>>>(NF, nslices, s->arow, s->acol, s->aval, amval, rsum, sptr,
                                                     s->A64.col, s->A64.val, mixed ? s->A32.val : nullptr,
                                                     transient ? s->M64.val : nullptr, s->rsum32, s->dinv32,
                                                     s->dinv64, s->diag64), ::nnqp::count_launch());
    // ---- norms
    double *dn;
    TRYF(T.a.alloc(&dn, 2 + 1024, st));
    CUF(det_max(rabs, NF, dn, dn + 2, st));
    CUF(det_sumsq(s->b0, NF, dn + 1, dn + 2, st));
    double hn[2];
    CUF(cudaMemcpyAsync(hn, dn, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUF(cudaStreamSynchronize(st));
    s->anorm_inf = hn[0];
    s->b0norm = std::sqrt(hn[1]);
    s->has_csr = true;  // the reduced CSR is always kept (small next to SELL; used by nn_spmv)
    s->has_full = true;
    // nothing is freed before this point: the most device memory the
    // assembly held at once is the system plus every temporary
    s->assembly_peak_bytes = s->arena.bytes + T.a.bytes;
    CUF(cudaGetLastError());
    *out = s;
    return NN_OK;
#undef TRYF
#undef CUF
}

}  // namespace nnqp

namespace nnqp {

nn_status mesh_structured_impl(int dim, int nx, int ny, int nz, double *coords, int32_t *conn, cudaStream_t st) {
    int64_t N, E;
    NN_TRY(nn_mesh_counts(dim, nx, ny, nz, &N, &E));
    if (!coords || !conn) {
        set_error("nn_mesh_structured: coords and conn are required");
        return NN_ERR_INVALID_ARG;
    }
    (k_coords<<<nblk(N), TPB, 0, st>>>(dim, nx, ny, dim == 3 ? nz : 1, N, coords), ::nnqp::count_launch());
    if (dim == 2) (k_conn2d<<<nblk((int64_t)nx * ny), TPB, 0, st>>>(nx, ny, conn), ::nnqp::count_launch());
    else (k_conn3d<<<nblk((int64_t)nx * ny * nz), TPB, 0, st>>>(nx, ny, nz, conn), ::nnqp::count_launch());
    NN_CUDA_TRY(cudaGetLastError());
    return NN_OK;
}

}  // namespace nnqp
