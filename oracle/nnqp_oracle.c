/*
 * nnqp_oracle.c -- plain FP64 CPU oracle for the non-negative diffusion QP.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py use it.  It shares no code with
 * the CUDA path.
 *
 * What it computes (Chang, Karra & Nakshatrala, arXiv 1506.08435):
 *   - P1 simplicial meshes of the unit square / cube (Sec. 2.1.3, the
 *     finite element spaces U^h, W^h with k = 1).  The paper's meshes are
 *     unstructured; this oracle uses a structured "/"-diagonal triangle split
 *     and a 6-tetrahedron Kuhn split of each hexahedron (reading, see header
 *     of oracle.py).
 *   - Element stiffness  K_e = |e| G^T D G  (the bilinear form B(w;c), Eq.
 *     for B and L in Sec. 2.1.2; Jacobian with F_{1,1} = D, Sec. 3.2),
 *     consistent mass M_e (F_{0,0} = 1/dt in the transient pointwise
 *     functions, Sec. 3.2), one-point load F_e = f(x_c)|e|/(d+1).
 *   - Dispersion tensor D = (a_T|v| + D_M) I + (a_L - a_T) v v^T/|v|
 *     (Sec. 5, dispersion tensor equation).
 *   - Box-constrained QP  min 1/2 x^T A x - b^T x,  lo <= x <= hi
 *     (Sec. 2.1.3 non-negative formulation; Sec. 2.2.2 transient QP with
 *     c_min <= c <= c_max).  Solved by projected Gauss-Seidel (Cryer's
 *     projected SOR with omega = 1) and by MPRGP (Dostal & Schoeberl 2005),
 *     both published methods, written here from their definitions.
 *   - KKT residual of the QP (first-order optimality of the convex QP).
 *
 * All arithmetic is IEEE double.  Loops are plain and unblocked.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_DEGENERATE 2
#define ORC_ERR_NOT_SPD 3
#define ORC_ERR_NAN 4
#define ORC_ERR_OOM 5

/* ------------------------------------------------------------------ */
/* Mesh: structured P1 simplices of [0,1]^d                            */
/* ------------------------------------------------------------------ */

void orc_mesh_counts(int dim, int nx, int ny, int nz, int64_t *n_nodes, int64_t *n_elems)
{
    if (dim == 2) {
        *n_nodes = (int64_t)(nx + 1) * (ny + 1);
        *n_elems = 2LL * nx * ny;
    } else {
        *n_nodes = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
        *n_elems = 6LL * nx * ny * nz;
    }
}

/* Node (i,j[,k]) has id i + (nx+1)(j + (ny+1)k) and coordinates (i/nx, j/ny, k/nz).
 * 2D: square (i,j) gives T0 = (v00,v10,v11), T1 = (v00,v11,v01), ids 2(i+nx j)+t.
 * 3D: hexahedron (i,j,k) (id i + nx(j + ny k)) gives 6 tetrahedra, one per
 * permutation p of the axes in lexicographic order; tet p is the monotone
 * lattice path v0 -> v0+e_p0 -> +e_p1 -> +e_p2, id 6*hex + p. */
void orc_mesh_structured(int dim, int nx, int ny, int nz, double *coords, int32_t *conn)
{
    if (dim == 2) {
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i <= nx; i++) {
                int64_t v = i + (int64_t)(nx + 1) * j;
                coords[2 * v + 0] = (double)i / (double)nx;
                coords[2 * v + 1] = (double)j / (double)ny;
            }
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int32_t v00 = i + (nx + 1) * j, v10 = v00 + 1;
                int32_t v01 = v00 + (nx + 1), v11 = v01 + 1;
                int64_t e = 2 * (i + (int64_t)nx * j);
                int32_t *t0 = conn + 3 * e, *t1 = conn + 3 * (e + 1);
                t0[0] = v00; t0[1] = v10; t0[2] = v11;
                t1[0] = v00; t1[1] = v11; t1[2] = v01;
            }
        return;
    }
    static const int perms[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
    int64_t sx = 1, sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
    int64_t step[3] = {sx, sy, sz};
    for (int k = 0; k <= nz; k++)
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i <= nx; i++) {
                int64_t v = i + sy * j + sz * k;
                coords[3 * v + 0] = (double)i / (double)nx;
                coords[3 * v + 1] = (double)j / (double)ny;
                coords[3 * v + 2] = (double)k / (double)nz;
            }
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int64_t hex = i + (int64_t)nx * (j + (int64_t)ny * k);
                int64_t v0 = i + sy * j + sz * k;
                for (int p = 0; p < 6; p++) {
                    int32_t *t = conn + 4 * (6 * hex + p);
                    int64_t v = v0;
                    t[0] = (int32_t)v;
                    for (int s = 0; s < 3; s++) {
                        v += step[perms[p][s]];
                        t[1 + s] = (int32_t)v;
                    }
                }
            }
}

/* ------------------------------------------------------------------ */
/* CSR pattern of the node graph: column j is in row i iff nodes i and */
/* j share an element (i == j included).  Columns ascending.           */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* mode 0: fill rowptr (N+1) and return nnz; mode 1: fill col using rowptr. */
static int64_t pattern_pass(int64_t N, int64_t E, int nv, const int32_t *conn,
                            int64_t *rowptr, int32_t *col, int mode)
{
    /* node -> element incidence, by counting */
    int64_t *inc_ptr = calloc((size_t)N + 1, sizeof(int64_t));
    int64_t *inc = malloc(sizeof(int64_t) * (size_t)(E * nv + 1));
    int64_t *fill = calloc((size_t)N, sizeof(int64_t));
    if (!inc_ptr || !inc || !fill) { free(inc_ptr); free(inc); free(fill); return -1; }
    for (int64_t e = 0; e < E; e++)
        for (int a = 0; a < nv; a++) inc_ptr[conn[e * nv + a] + 1]++;
    for (int64_t v = 0; v < N; v++) inc_ptr[v + 1] += inc_ptr[v];
    for (int64_t e = 0; e < E; e++)
        for (int a = 0; a < nv; a++) {
            int64_t v = conn[e * nv + a];
            inc[inc_ptr[v] + fill[v]++] = e;
        }
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < N; v++) {
        int64_t d = inc_ptr[v + 1] - inc_ptr[v];
        if (d > maxdeg) maxdeg = d;
    }
    int32_t *buf = malloc(sizeof(int32_t) * (size_t)(maxdeg * nv + 1));
    int64_t nnz = 0;
    if (mode == 0) rowptr[0] = 0;
    for (int64_t v = 0; v < N; v++) {
        int64_t m = 0;
        for (int64_t q = inc_ptr[v]; q < inc_ptr[v + 1]; q++) {
            int64_t e = inc[q];
            for (int a = 0; a < nv; a++) buf[m++] = conn[e * nv + a];
        }
        if (m == 0) buf[m++] = (int32_t)v; /* isolated node keeps its diagonal */
        qsort(buf, (size_t)m, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t q = 0; q < m; q++)
            if (q == 0 || buf[q] != buf[q - 1]) buf[u++] = buf[q];
        if (mode == 0) {
            nnz += u;
            rowptr[v + 1] = nnz;
        } else {
            memcpy(col + rowptr[v], buf, sizeof(int32_t) * (size_t)u);
        }
    }
    free(buf); free(inc_ptr); free(inc); free(fill);
    return mode == 0 ? nnz : rowptr[N];
}

int64_t orc_pattern_rowptr(int64_t N, int64_t E, int nv, const int32_t *conn, int64_t *rowptr)
{
    return pattern_pass(N, E, nv, conn, rowptr, NULL, 0);
}

int64_t orc_pattern_cols(int64_t N, int64_t E, int nv, const int32_t *conn,
                         const int64_t *rowptr, int32_t *col)
{
    return pattern_pass(N, E, nv, conn, (int64_t *)rowptr, col, 1);
}

/* ------------------------------------------------------------------ */
/* Element matrices and assembly                                       */
/* ------------------------------------------------------------------ */

/* Diffusivity of one element as a full d x d matrix.
 * kind 0: coef holds the upper triangle (2D: xx,xy,yy; 3D: xx,xy,xz,yy,yz,zz).
 * kind 1: coef holds the cell velocity v; D follows the dispersion law. */
static void element_D(int dim, int kind, const double *coef, double aL, double aT,
                      double DM, double D[3][3])
{
    memset(D, 0, sizeof(double) * 9);
    if (kind == 0) {
        if (dim == 2) {
            D[0][0] = coef[0]; D[0][1] = D[1][0] = coef[1]; D[1][1] = coef[2];
        } else {
            D[0][0] = coef[0]; D[0][1] = D[1][0] = coef[1]; D[0][2] = D[2][0] = coef[2];
            D[1][1] = coef[3]; D[1][2] = D[2][1] = coef[4]; D[2][2] = coef[5];
        }
        return;
    }
    double vv = 0.0;
    for (int p = 0; p < dim; p++) vv += coef[p] * coef[p];
    double vn = sqrt(vv);
    for (int p = 0; p < dim; p++) D[p][p] = aT * vn + DM;
    if (vn > 0.0)
        for (int p = 0; p < dim; p++)
            for (int q = 0; q < dim; q++) D[p][q] += (aL - aT) * coef[p] * coef[q] / vn;
}

/* Sylvester's criterion on the leading principal minors. */
static int is_spd(int dim, double D[3][3])
{
    double m1 = D[0][0];
    double m2 = D[0][0] * D[1][1] - D[0][1] * D[1][0];
    if (!(m1 > 0.0) || !(m2 > 0.0)) return 0;
    if (dim == 2) return 1;
    double m3 = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1])
              - D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0])
              + D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
    return m3 > 0.0;
}

/* Barycentric gradients G[a][p] = d lambda_a / d x_p and the measure |e|.
 * With J = [x1-x0, ..., xd-x0], lambda_{1..d}(x) = J^{-1}(x - x0), so the
 * gradient of lambda_k is row k of J^{-1}; lambda_0 = 1 - sum of the others. */
static int element_geometry(int dim, const double *X /* (dim+1) x dim */,
                            double G[4][3], double *vol)
{
    double J[3][3], Ji[3][3], det;
    for (int p = 0; p < dim; p++)
        for (int k = 0; k < dim; k++) J[p][k] = X[(k + 1) * dim + p] - X[p];
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (det == 0.0 || isnan(det)) return ORC_ERR_DEGENERATE;
        Ji[0][0] = J[1][1] / det;  Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
        *vol = fabs(det) / 2.0;
    } else {
        double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        if (det == 0.0 || isnan(det)) return ORC_ERR_DEGENERATE;
        /* inverse = adjugate / det; adj[k][p] = cofactor[p][k] */
        double cof[3][3];
        cof[0][0] = c00; cof[0][1] = c01; cof[0][2] = c02;
        cof[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        cof[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        cof[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        cof[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        cof[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        cof[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        for (int k = 0; k < 3; k++)
            for (int p = 0; p < 3; p++) Ji[k][p] = cof[p][k] / det;
        *vol = fabs(det) / 6.0;
    }
    for (int p = 0; p < dim; p++) {
        double s = 0.0;
        for (int k = 0; k < dim; k++) {
            G[k + 1][p] = Ji[k][p];
            s += Ji[k][p];
        }
        G[0][p] = -s;
    }
    return ORC_OK;
}

static int64_t find_col(const int64_t *rowptr, const int32_t *col, int64_t row, int32_t c)
{
    int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (col[mid] == c) return mid;
        if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Assemble the full stiffness K, optionally the consistent mass M, and the
 * load F over all N nodes, summing element contributions in element order.
 * f_elem may be NULL (f = 0).  Kval/Mval/F are overwritten. */
int orc_assemble(int dim, int64_t N, int64_t E, const double *coords, const int32_t *conn,
                 int coef_kind, const double *coef, double aL, double aT, double DM,
                 const double *f_elem, const int64_t *rowptr, const int32_t *col,
                 double *Kval, double *Mval, double *F)
{
    int nv = dim + 1;
    int ncoef = coef_kind == 0 ? (dim == 2 ? 3 : 6) : dim;
    memset(Kval, 0, sizeof(double) * (size_t)rowptr[N]);
    if (Mval) memset(Mval, 0, sizeof(double) * (size_t)rowptr[N]);
    memset(F, 0, sizeof(double) * (size_t)N);
    double mdiag = 2.0 / ((nv) * (nv + 1)), moff = 1.0 / ((nv) * (nv + 1));
    for (int64_t e = 0; e < E; e++) {
        double X[12], G[4][3], vol, D[3][3];
        const int32_t *t = conn + e * nv;
        for (int a = 0; a < nv; a++) {
            if (t[a] < 0 || t[a] >= N) return ORC_ERR_ARG;
            for (int p = 0; p < dim; p++) X[a * dim + p] = coords[(int64_t)t[a] * dim + p];
        }
        const double *ce = coef + e * ncoef;
        for (int q = 0; q < ncoef; q++)
            if (isnan(ce[q]) || isinf(ce[q])) return ORC_ERR_NAN;
        int st = element_geometry(dim, X, G, &vol);
        if (st) return st;
        element_D(dim, coef_kind, ce, aL, aT, DM, D);
        if (!is_spd(dim, D)) return ORC_ERR_NOT_SPD;
        for (int a = 0; a < nv; a++) {
            for (int b = 0; b < nv; b++) {
                double kab = 0.0;
                for (int p = 0; p < dim; p++)
                    for (int q = 0; q < dim; q++) kab += G[a][p] * D[p][q] * G[b][q];
                int64_t pos = find_col(rowptr, col, t[a], t[b]);
                if (pos < 0) return ORC_ERR_ARG;
                Kval[pos] += vol * kab;
                if (Mval) Mval[pos] += vol * (a == b ? mdiag : moff);
            }
            if (f_elem) F[t[a]] += f_elem[e] * vol / nv;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sparse kernels on a CSR matrix (rowptr int64, col int32)            */
/* ------------------------------------------------------------------ */

void orc_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
              const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) s += v[q] * x[ci[q]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static double clampd(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

/* Projected gradient of the box QP: free entries keep g, entries at the
 * lower bound keep min(g,0), entries at the upper bound keep max(g,0). */
static double proj_grad(double x, double g, double lo, double hi)
{
    if (x <= lo && x >= hi) return 0.0;
    if (x <= lo) return g < 0.0 ? g : 0.0;
    if (x >= hi) return g > 0.0 ? g : 0.0;
    return g;
}

/* KKT measures of x for min 1/2 x'Ax - b'x on [lo,hi]^n.
 * out[0] = ||gP||_2 / den2, out[1] = ||gP||_inf / deninf,
 * out[2] = 1 if lo <= x_i <= hi for all i (exact), else 0,
 * out[3] = objective 1/2 x'Ax - b'x,
 * out[4] = ||gP||_2 (absolute).
 * den2 = ||b||_2 (deninf = ||b||_inf); when b = 0 both become
 * ||A||_inf * max(|lo| if finite, |hi| if finite, 1). */
void orc_kkt(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
             const double *b, double lo, double hi, const double *x, double *out)
{
    double *Ax = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_spmv(n, rp, ci, v, x, Ax);
    double gp2 = 0.0, gpi = 0.0, b2 = 0.0, bi = 0.0, xAx = 0.0, bx = 0.0, anorm = 0.0;
    int ok = 1;
    for (int64_t i = 0; i < n; i++) {
        double g = Ax[i] - b[i];
        double gp = proj_grad(x[i], g, lo, hi);
        gp2 += gp * gp;
        if (fabs(gp) > gpi) gpi = fabs(gp);
        b2 += b[i] * b[i];
        if (fabs(b[i]) > bi) bi = fabs(b[i]);
        xAx += x[i] * Ax[i];
        bx += b[i] * x[i];
        if (!(x[i] >= lo && x[i] <= hi)) ok = 0;
        double rs = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) rs += fabs(v[q]);
        if (rs > anorm) anorm = rs;
    }
    double den2 = sqrt(b2), deninf = bi;
    if (b2 == 0.0) {
        double s = 1.0;
        if (isfinite(lo) && fabs(lo) > s) s = fabs(lo);
        if (isfinite(hi) && fabs(hi) > s) s = fabs(hi);
        den2 = deninf = anorm * s;
        if (den2 == 0.0) den2 = deninf = 1.0;
    }
    out[0] = sqrt(gp2) / den2;
    out[1] = gpi / deninf;
    out[2] = ok ? 1.0 : 0.0;
    out[3] = 0.5 * xAx - bx;
    out[4] = sqrt(gp2);
    free(Ax);
}

/* ------------------------------------------------------------------ */
/* Projected Gauss-Seidel (Cryer's projected SOR, omega = 1)            */
/* ------------------------------------------------------------------ */

/* Sweeps i = 0..n-1 in natural order:
 *   x_i <- clamp((b_i - sum_{j != i} A_ij x_j) / A_ii, lo, hi)
 * until the largest change in a sweep is <= tol * max(1, ||x||_inf) or
 * maxsweep sweeps are done.  Returns the number of sweeps (negative if the
 * limit was reached). */
int64_t orc_pgs(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                const double *b, double lo, double hi, double *x, double tol, int64_t maxsweep)
{
    for (int64_t i = 0; i < n; i++) x[i] = clampd(x[i], lo, hi);
    for (int64_t s = 1; s <= maxsweep; s++) {
        double dmax = 0.0, xmax = 1.0;
        for (int64_t i = 0; i < n; i++) {
            double diag = 0.0, r = b[i];
            for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
                if (ci[q] == i) diag = v[q];
                else r -= v[q] * x[ci[q]];
            }
            double xn = clampd(r / diag, lo, hi);
            double d = fabs(xn - x[i]);
            if (d > dmax) dmax = d;
            x[i] = xn;
            if (fabs(xn) > xmax) xmax = fabs(xn);
        }
        if (dmax <= tol * xmax) return s;
    }
    return -maxsweep;
}

/* ------------------------------------------------------------------ */
/* MPRGP: modified proportioning with reduced gradient projections      */
/* (Dostal & Schoeberl, Comput. Optim. Appl. 30 (2005)), two-sided box.  */
/* ------------------------------------------------------------------ */

/* Stops when ||gP||_2 <= rtol * den (den as in orc_kkt).  Gamma = 1 and
 * the expansion step length abar = 1.9 / ||A||_inf (||A||_inf >= lambda_max,
 * so abar < 2/||A||).  Returns iterations (negative if maxit reached). */
int64_t orc_mprgp(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                  const double *b, double lo, double hi, double *x, double rtol,
                  int64_t maxit, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    if (n == 0) return 0;
    size_t sz = sizeof(double) * (size_t)n;
    double *g = malloc(sz), *p = malloc(sz), *Ap = malloc(sz), *phi = malloc(sz), *w = malloc(sz);
    double anorm = 0.0, b2 = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double rs = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) rs += fabs(v[q]);
        if (rs > anorm) anorm = rs;
        b2 += b[i] * b[i];
    }
    double den = sqrt(b2);
    if (b2 == 0.0) {
        double s = 1.0;
        if (isfinite(lo) && fabs(lo) > s) s = fabs(lo);
        if (isfinite(hi) && fabs(hi) > s) s = fabs(hi);
        den = anorm * s;
    }
    double abar = 1.9 / anorm, Gamma = 1.0;
    for (int64_t i = 0; i < n; i++) x[i] = clampd(x[i], lo, hi);
    orc_spmv(n, rp, ci, v, x, g);
    for (int64_t i = 0; i < n; i++) g[i] -= b[i];
#define FREE(i) (x[i] > lo && x[i] < hi)
    for (int64_t i = 0; i < n; i++) p[i] = FREE(i) ? g[i] : 0.0;
    int64_t it;
    for (it = 0; it < maxit; it++) {
        /* norms of the chopped gradient beta, the free gradient phi and the
         * reduced free gradient phit (phit'phi in the proportioning test) */
        double gp2 = 0.0, beta2 = 0.0, phitphi = 0.0;
        for (int64_t i = 0; i < n; i++) {
            double gi = g[i];
            if (FREE(i)) {
                phi[i] = gi;
                double t;
                if (gi > 0.0) t = fmin((x[i] - lo) / abar, gi);
                else t = fmax((x[i] - hi) / abar, gi);
                phitphi += t * gi;
                gp2 += gi * gi;
            } else {
                phi[i] = 0.0;
                double bt = proj_grad(x[i], gi, lo, hi);
                beta2 += bt * bt;
                gp2 += bt * bt;
            }
        }
        if (sqrt(gp2) <= rtol * den) break;
        if (beta2 <= Gamma * Gamma * phitphi) {
            /* conjugate gradient direction p on the free set */
            orc_spmv(n, rp, ci, v, p, Ap);
            double pAp = dot(n, p, Ap);
            double acg = dot(n, g, p) / pAp;
            double af = INFINITY;
            for (int64_t i = 0; i < n; i++) {
                if (p[i] > 0.0) af = fmin(af, (x[i] - lo) / p[i]);
                else if (p[i] < 0.0) af = fmin(af, (x[i] - hi) / p[i]);
            }
            if (acg <= af) {
                for (int64_t i = 0; i < n; i++) {
                    x[i] = clampd(x[i] - acg * p[i], lo, hi);
                    g[i] -= acg * Ap[i];
                }
                double num = 0.0;
                for (int64_t i = 0; i < n; i++) num += (FREE(i) ? g[i] : 0.0) * Ap[i];
                double gam = num / pAp;
                for (int64_t i = 0; i < n; i++) p[i] = (FREE(i) ? g[i] : 0.0) - gam * p[i];
            } else {
                /* expansion: feasible half step, then a projected step of
                 * length abar along the free gradient */
                for (int64_t i = 0; i < n; i++) {
                    x[i] = clampd(x[i] - af * p[i], lo, hi);
                    g[i] -= af * Ap[i];
                }
                for (int64_t i = 0; i < n; i++) {
                    double ph = FREE(i) ? g[i] : 0.0;
                    w[i] = clampd(x[i] - abar * ph, lo, hi);
                }
                memcpy(x, w, sz);
                orc_spmv(n, rp, ci, v, x, g);
                for (int64_t i = 0; i < n; i++) g[i] -= b[i];
                for (int64_t i = 0; i < n; i++) p[i] = FREE(i) ? g[i] : 0.0;
            }
        } else {
            /* proportioning: step along the chopped gradient */
            for (int64_t i = 0; i < n; i++) w[i] = FREE(i) ? 0.0 : proj_grad(x[i], g[i], lo, hi);
            orc_spmv(n, rp, ci, v, w, Ap);
            double a = dot(n, g, w) / dot(n, w, Ap);
            for (int64_t i = 0; i < n; i++) x[i] = clampd(x[i] - a * w[i], lo, hi);
            orc_spmv(n, rp, ci, v, x, g);
            for (int64_t i = 0; i < n; i++) g[i] -= b[i];
            for (int64_t i = 0; i < n; i++) p[i] = FREE(i) ? g[i] : 0.0;
        }
        if ((it + 1) % 64 == 0) { /* refresh g against drift */
            orc_spmv(n, rp, ci, v, x, g);
            for (int64_t i = 0; i < n; i++) g[i] -= b[i];
        }
    }
#undef FREE
    free(g); free(p); free(Ap); free(phi); free(w);
    return it < maxit ? it : -maxit;
}

/* ------------------------------------------------------------------ */
/* CG on a face: solve A_FF x_F = b_F - A_FA x_A for the entries with   */
/* fixed[i] == 0, holding the others at their current values.  Jacobi   */
/* preconditioned; stops at ||r|| <= tol * ||b_F - A_FA x_A||.          */
/* ------------------------------------------------------------------ */

int64_t orc_cg_face(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                    const double *b, const uint8_t *fixed, double *x, double tol, int64_t maxit)
{
    if (n == 0) return 0;
    size_t sz = sizeof(double) * (size_t)n;
    double *r = malloc(sz), *z = malloc(sz), *p = malloc(sz), *q = malloc(sz), *dinv = malloc(sz);
    double *xf = malloc(sz);
    for (int64_t i = 0; i < n; i++) {
        double d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) if (ci[k] == i) d = v[k];
        dinv[i] = d != 0.0 ? 1.0 / d : 1.0;
        xf[i] = fixed[i] ? x[i] : 0.0;
    }
    /* right-hand side of the face system: b - A x_fixed, restricted */
    orc_spmv(n, rp, ci, v, xf, q);
    double rhs2 = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double rhs = fixed[i] ? 0.0 : b[i] - q[i];
        rhs2 += rhs * rhs;
        xf[i] = fixed[i] ? 0.0 : x[i];
    }
    /* residual r = rhs - A_FF x_F */
    orc_spmv(n, rp, ci, v, xf, q);
    for (int64_t i = 0; i < n; i++) {
        r[i] = 0.0;
        if (!fixed[i]) {
            double rr = b[i] - q[i];
            for (int64_t k = rp[i]; k < rp[i + 1]; k++)
                if (fixed[ci[k]]) rr -= v[k] * x[ci[k]];
            r[i] = rr;
        }
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    double rz = dot(n, r, z);
    double stop = tol * sqrt(rhs2);
    int64_t it;
    for (it = 0; it < maxit; it++) {
        if (sqrt(dot(n, r, r)) <= stop) break;
        orc_spmv(n, rp, ci, v, p, q);
        for (int64_t i = 0; i < n; i++) if (fixed[i]) q[i] = 0.0;
        double a = rz / dot(n, p, q);
        for (int64_t i = 0; i < n; i++) {
            if (fixed[i]) continue;
            x[i] += a * p[i];
            r[i] -= a * q[i];
            z[i] = dinv[i] * r[i];
        }
        double rz2 = dot(n, r, z);
        double beta = rz2 / rz;
        rz = rz2;
        for (int64_t i = 0; i < n; i++) p[i] = fixed[i] ? 0.0 : z[i] + beta * p[i];
    }
    free(r); free(z); free(p); free(q); free(dinv); free(xf);
    return it < maxit ? it : -maxit;
}
