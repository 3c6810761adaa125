// Host check of the SSOR ordering the library builds (nnqp::ssor_layout,
// the host half of nn_precond_setup) and of the sweep index arithmetic of
// ssor.cuh, without a GPU: reads an n x n CSR matrix, a vector r, a face
// mask and omega from argv[1]; stores A's off-diagonals in pair-interleaved
// SELL-32 as the assembly does; calls the library's layout; runs the two
// sweeps slice by slice with the kernels' indexing (rows of one colour are
// independent, so a sequential pass computes what the parallel one does);
// writes z and the colours to argv[2].  Test infrastructure only.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <vector>
#include "internal.h"

using namespace nnqp;

static int64_t sell_pos(int64_t base, int k, int lane) { return base + 64 * (int64_t)(k >> 1) + 2 * lane + (k & 1); }

template <typename T>
static bool get(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t n = 0, nnz = 0;
    if (!get(f, &n, 1) || !get(f, &nnz, 1)) return 2;
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> ci(nnz);
    std::vector<double> v(nnz), r(n), dinv(n, 0.0);
    std::vector<uint8_t> fm(n);
    double om = 1.0;
    if (!get(f, rp.data(), n + 1) || !get(f, ci.data(), nnz) || !get(f, v.data(), nnz) || !get(f, r.data(), n) ||
        !get(f, fm.data(), n) || !get(f, &om, 1))
        return 2;
    fclose(f);
    const int64_t ns = (n + 31) / 32;
    std::vector<int64_t> sptr(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        int64_t w = 0;
        for (int l = 0; l < 32 && s * 32 + l < n; ++l) w = std::max<int64_t>(w, rp[s * 32 + l + 1] - rp[s * 32 + l] - 1);
        w += w & 1;
        sptr[s + 1] = sptr[s] + 32 * w;
    }
    std::vector<int32_t> scol(sptr[ns]);
    std::vector<double> sval(sptr[ns], 0.0);
    for (int64_t s = 0; s < ns; ++s) {
        const int w = (int)((sptr[s + 1] - sptr[s]) >> 5);
        for (int l = 0; l < 32; ++l) {
            const int64_t i = s * 32 + l;
            int k = 0;
            if (i < n)
                for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
                    if (ci[q] == i) {
                        dinv[i] = 1.0 / v[q];
                        continue;
                    }
                    scol[sell_pos(sptr[s], k, l)] = ci[q];
                    sval[sell_pos(sptr[s], k, l)] = v[q];
                    ++k;
                }
            for (; k < w; ++k) scol[sell_pos(sptr[s], k, l)] = (int32_t)std::min<int64_t>(i, n - 1);
        }
    }
    SsorHost h;
    if (ssor_layout(n, ns, sptr.data(), scol.data(), sval.data(), h) != NN_OK) return 3;
    // every off-diagonal in exactly one part; padding lanes carry -1
    int64_t parts = 0;
    for (double x : h.lval) parts += x != 0.0;
    for (double x : h.uval) parts += x != 0.0;
    if (parts != nnz - n) return 4;
    // the sweeps; scratch starts as NaN, so a read of an unwritten entry shows
    std::vector<double> y(n, NAN), z(n, NAN);
    for (int c = 0; c < h.ncolors; ++c)
        for (int64_t s = h.cslice[c]; s < h.cslice[c + 1]; ++s)
            for (int lane = 0; lane < 32; ++lane) {
                const int32_t i = h.row[s * 32 + lane];
                const int64_t e0 = h.lptr[s], w = (h.lptr[s + 1] - e0) >> 5;
                double t = 0.0;
                for (int64_t k = 0; k < w; ++k) t = std::fma(h.lval[e0 + 32 * k + lane], y[h.lcol[e0 + 32 * k + lane]], t);
                if (i >= 0) y[i] = fm[i] ? dinv[i] * std::fma(-om, t, r[i]) : 0.0;
            }
    const double sc = om * (2.0 - om);
    for (int c = h.ncolors - 1; c >= 0; --c)
        for (int64_t s = h.cslice[c]; s < h.cslice[c + 1]; ++s)
            for (int lane = 0; lane < 32; ++lane) {
                const int32_t i = h.row[s * 32 + lane];
                const int64_t e0 = h.uptr[s], w = (h.uptr[s + 1] - e0) >> 5;
                double t = 0.0;
                for (int64_t k = 0; k < w; ++k) t = std::fma(h.uval[e0 + 32 * k + lane], z[h.ucol[e0 + 32 * k + lane]], t);
                if (i >= 0) z[i] = fm[i] ? std::fma(sc, y[i], -om * dinv[i] * t) : 0.0;
            }
    FILE *g = fopen(argv[2], "wb");
    if (!g) return 2;
    fwrite(z.data(), sizeof(double), n, g);
    fwrite(h.color.data(), sizeof(int32_t), n, g);
    fclose(g);
    return 0;
}
