// SSOR preconditioning, host side: the DSatur colouring of A's pattern, the
// colour-ordered SELL-32 storage of A's lower and upper parts that the
// sweeps of ssor.cuh read, and the stand-alone application of a
// preconditioner (nn_precond_apply) through the solve kernels' sweep code.
#include <algorithm>
#include <cstring>
#include <queue>
#include <vector>
#include "internal.h"
#include "ops.cuh"
#include "ssor.cuh"

namespace nnqp {

// DSatur (Brelaz, "New methods to color the vertices of a graph", Comm. ACM
// 22, 1979): the uncoloured vertex of largest saturation degree (number of
// distinct colours among its neighbours) takes the smallest colour none of
// its neighbours has; ties go to the larger degree, then to the smaller
// index.  A max-heap of (saturation, degree, -index) with lazy deletion:
// a vertex is pushed again whenever its saturation grows, and a popped entry
// whose saturation is out of date, or whose vertex is coloured, is skipped.
nn_status dsatur_color(int64_t n, const int64_t *rowptr, const int32_t *col, int32_t *color, int *ncolors) {
    struct Item {
        int sat, deg;
        int64_t v;
        bool operator<(const Item &o) const {   // "lower priority than"
            if (sat != o.sat) return sat < o.sat;
            if (deg != o.deg) return deg < o.deg;
            return v > o.v;
        }
    };
    std::vector<uint64_t> seen((size_t)n, 0);   // colours among the neighbours (bit k = colour k)
    std::vector<int> deg((size_t)n, 0);
    for (int64_t i = 0; i < n; ++i) {
        int d = 0;
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) d += col[q] != i;
        deg[(size_t)i] = d;
        color[i] = -1;
    }
    std::vector<Item> init;
    init.reserve((size_t)n);
    for (int64_t i = 0; i < n; ++i) init.push_back(Item{0, deg[(size_t)i], i});
    std::priority_queue<Item> heap(std::less<Item>(), std::move(init));
    int k = 0;
    while (!heap.empty()) {
        const Item t = heap.top();
        heap.pop();
        const int64_t v = t.v;
        if (color[v] >= 0 || t.sat != __builtin_popcountll(seen[(size_t)v])) continue;
        const uint64_t used = seen[(size_t)v];
        if (used == ~0ull) {
            set_error("nn_color_dsatur: more than 64 colours needed (vertex %lld)", (long long)v);
            return NN_ERR_INVALID_ARG;
        }
        const int c = __builtin_ctzll(~used);
        color[v] = c;
        k = std::max(k, c + 1);
        for (int64_t q = rowptr[v]; q < rowptr[v + 1]; ++q) {
            const int64_t j = col[q];
            if (j == v || color[j] >= 0) continue;
            const uint64_t bit = 1ull << c;
            if (seen[(size_t)j] & bit) continue;
            seen[(size_t)j] |= bit;
            heap.push(Item{__builtin_popcountll(seen[(size_t)j]), deg[(size_t)j], j});
        }
    }
    *ncolors = k;
    return NN_OK;
}

nn_status ssor_layout(int64_t n, int64_t ns, const int64_t *sptr, const int32_t *scol, const double *sval,
                      SsorHost &h) {
    // A's off-diagonal entries, row by row, from its pair-interleaved SELL-32
    // storage (sell_idx; padding slots carry the row's own column)
    std::vector<int64_t> rp((size_t)n + 1, 0);
    for (int64_t sl = 0; sl < ns; ++sl) {
        const int w = (int)((sptr[sl + 1] - sptr[sl]) >> 5);
        for (int l = 0; l < 32 && sl * 32 + l < n; ++l) {
            const int64_t i = sl * 32 + l;
            for (int k = 0; k < w; ++k) rp[(size_t)i + 1] += scol[sell_idx(sptr[sl], k, l)] != i;
        }
    }
    for (int64_t i = 0; i < n; ++i) rp[(size_t)i + 1] += rp[(size_t)i];
    std::vector<int32_t> oc((size_t)rp[(size_t)n]);
    std::vector<double> ov((size_t)rp[(size_t)n]);
    for (int64_t sl = 0; sl < ns; ++sl) {
        const int w = (int)((sptr[sl + 1] - sptr[sl]) >> 5);
        for (int l = 0; l < 32 && sl * 32 + l < n; ++l) {
            const int64_t i = sl * 32 + l;
            int64_t q = rp[(size_t)i];
            for (int k = 0; k < w; ++k) {
                const int64_t e = sell_idx(sptr[sl], k, l);
                if (scol[e] == i) continue;
                oc[(size_t)q] = scol[e];
                ov[(size_t)q] = sval[e];
                ++q;
            }
        }
    }
    std::vector<int32_t> &color = h.color;
    color.assign((size_t)n, -1);
    int C = 0;
    NN_TRY(dsatur_color(n, rp.data(), oc.data(), color.data(), &C));
    // rows of each colour, ascending; slices of 32
    std::vector<std::vector<int32_t>> rows((size_t)C);
    for (int64_t i = 0; i < n; ++i) rows[(size_t)color[(size_t)i]].push_back((int32_t)i);
    h.ncolors = C;
    h.cslice.assign((size_t)C + 1, 0);
    for (int c = 0; c < C; ++c) h.cslice[(size_t)c + 1] = h.cslice[(size_t)c] + ((int64_t)rows[(size_t)c].size() + 31) / 32;
    const int64_t nsl = h.cslice[(size_t)C];
    h.row.assign((size_t)nsl * 32, -1);
    h.lptr.assign((size_t)nsl + 1, 0);
    h.uptr.assign((size_t)nsl + 1, 0);
    // entries of each row by part; a neighbour of the same colour exists only
    // if the pattern is not symmetric
    auto parts = [&](int32_t i, int64_t &nl, int64_t &nu) {
        nl = nu = 0;
        for (int64_t q = rp[(size_t)i]; q < rp[(size_t)i + 1]; ++q) {
            const int cj = color[(size_t)oc[(size_t)q]], ci = color[(size_t)i];
            if (cj == ci) return false;
            (cj < ci ? nl : nu) += 1;
        }
        return true;
    };
    for (int c = 0; c < C; ++c) {
        const std::vector<int32_t> &rc = rows[(size_t)c];
        for (int64_t sl = h.cslice[(size_t)c]; sl < h.cslice[(size_t)c + 1]; ++sl) {
            int64_t wl = 0, wu = 0;
            for (int l = 0; l < 32; ++l) {
                const int64_t k = (sl - h.cslice[(size_t)c]) * 32 + l;
                if (k >= (int64_t)rc.size()) break;
                const int32_t i = rc[(size_t)k];
                int64_t nl, nu;
                if (!parts(i, nl, nu)) {
                    set_error("SSOR set-up: row %d is coupled to a row of its own colour (pattern not symmetric)", i);
                    return NN_ERR_INVALID_ARG;
                }
                h.row[(size_t)(sl * 32 + l)] = i;
                wl = std::max(wl, nl);
                wu = std::max(wu, nu);
            }
            h.lptr[(size_t)sl + 1] = h.lptr[(size_t)sl] + 32 * wl;
            h.uptr[(size_t)sl + 1] = h.uptr[(size_t)sl] + 32 * wu;
        }
    }
    h.lcol.assign((size_t)h.lptr[(size_t)nsl], rows[0][0]);
    h.ucol.assign((size_t)h.uptr[(size_t)nsl], rows[(size_t)C - 1][0]);
    h.lval.assign((size_t)h.lptr[(size_t)nsl], 0.0);
    h.uval.assign((size_t)h.uptr[(size_t)nsl], 0.0);
    for (int64_t sl = 0; sl < nsl; ++sl)
        for (int l = 0; l < 32; ++l) {
            const int32_t i = h.row[(size_t)(sl * 32 + l)];
            if (i < 0) continue;
            int64_t kl = 0, ku = 0;
            for (int64_t q = rp[(size_t)i]; q < rp[(size_t)i + 1]; ++q) {
                const int32_t j = oc[(size_t)q];
                if (color[(size_t)j] < color[(size_t)i]) {
                    const size_t e = (size_t)(h.lptr[(size_t)sl] + 32 * kl++ + l);
                    h.lcol[e] = j;
                    h.lval[e] = ov[(size_t)q];
                } else {
                    const size_t e = (size_t)(h.uptr[(size_t)sl] + 32 * ku++ + l);
                    h.ucol[e] = j;
                    h.uval[e] = ov[(size_t)q];
                }
            }
        }
    return NN_OK;
}

nn_status ssor_setup(nn_system *s, cudaStream_t st) {
    if (s->ssor.ncolors > 0) return NN_OK;
    const int64_t n = s->NF;
    if (n < 1) return NN_OK;   // nothing to order (no free unknowns)
    const int64_t ns = s->A64.nslices, stored = s->A64.stored;
    SsorHost h;
    {
        std::vector<int64_t> sptr((size_t)ns + 1);
        std::vector<int32_t> scol((size_t)stored);
        std::vector<double> sval((size_t)stored);
        NN_CUDA_TRY(cudaMemcpyAsync(sptr.data(), s->A64.sptr, sizeof(int64_t) * (ns + 1), cudaMemcpyDeviceToHost, st));
        NN_CUDA_TRY(cudaMemcpyAsync(scol.data(), s->A64.col, sizeof(int32_t) * stored, cudaMemcpyDeviceToHost, st));
        NN_CUDA_TRY(cudaMemcpyAsync(sval.data(), s->A64.val, sizeof(double) * stored, cudaMemcpyDeviceToHost, st));
        NN_CUDA_TRY(cudaStreamSynchronize(st));
        NN_TRY(ssor_layout(n, ns, sptr.data(), scol.data(), sval.data(), h));
    }
    // device copies, owned by the system
    int64_t *d_cslice, *d_lptr, *d_uptr;
    int32_t *d_row, *d_lcol, *d_ucol;
    double *d_lval, *d_uval;
    DevArena &A = s->arena;
    NN_TRY(A.alloc(&d_cslice, h.cslice.size(), st));
    NN_TRY(A.alloc(&d_row, h.row.size(), st));
    NN_TRY(A.alloc(&d_lptr, h.lptr.size(), st));
    NN_TRY(A.alloc(&d_uptr, h.uptr.size(), st));
    NN_TRY(A.alloc(&d_lcol, h.lcol.size(), st));
    NN_TRY(A.alloc(&d_ucol, h.ucol.size(), st));
    NN_TRY(A.alloc(&d_lval, h.lval.size(), st));
    NN_TRY(A.alloc(&d_uval, h.uval.size(), st));
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    NN_CUDA_TRY(up(d_cslice, h.cslice.data(), sizeof(int64_t) * h.cslice.size()));
    NN_CUDA_TRY(up(d_row, h.row.data(), sizeof(int32_t) * h.row.size()));
    NN_CUDA_TRY(up(d_lptr, h.lptr.data(), sizeof(int64_t) * h.lptr.size()));
    NN_CUDA_TRY(up(d_uptr, h.uptr.data(), sizeof(int64_t) * h.uptr.size()));
    NN_CUDA_TRY(up(d_lcol, h.lcol.data(), sizeof(int32_t) * h.lcol.size()));
    NN_CUDA_TRY(up(d_ucol, h.ucol.data(), sizeof(int32_t) * h.ucol.size()));
    NN_CUDA_TRY(up(d_lval, h.lval.data(), sizeof(double) * h.lval.size()));
    NN_CUDA_TRY(up(d_uval, h.uval.data(), sizeof(double) * h.uval.size()));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    // the parts stream from HBM on every application once they exceed about
    // a third of L2 (the threshold of the solve's own operator)
    const bool stream = 12.0 * (double)(h.lval.size() + h.uval.size()) > 48.0 * (1 << 20);
    s->ssor = SsorF64{h.ncolors, stream, 1.0, d_cslice, d_row, d_lptr, d_uptr, d_lcol, d_ucol, d_lval, d_uval};
    s->ssor_slices = (int64_t)h.lptr.size() - 1;
    s->ssor_color.swap(h.color);
    return NN_OK;
}

namespace {

struct PcArgs {
    SsorF64 S;
    int kind;
    int64_t n;
    const uint8_t *fm;
    const double *dinv, *r;
    double *y, *z;
    GridBarrier *bar;
    unsigned long long timeout_ns;
};

// z = P r with the solve kernels' code (cooperative launch for SSOR: its
// colours are separated by grid barriers).
__global__ void __launch_bounds__(256) k_precond_apply(PcArgs a) {
    __shared__ RedSmem sm;
    if (a.kind == NN_PC_JACOBI) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
            a.z[i] = (a.fm == nullptr || a.fm[i]) ? a.dinv[i] * a.r[i] : 0.0;
        return;
    }
    GridTeam T{a.bar, nullptr, (int)gridDim.x, a.timeout_ns, 0, 0, &sm};
    ssor_apply(T, a.S, a.fm, a.dinv, a.r, a.y, a.z, [](int64_t, double) {});
}

}  // namespace
}  // namespace nnqp

using namespace nnqp;

extern "C" {

nn_status nn_color_dsatur(int64_t n, const int64_t *rowptr, const int32_t *col, int32_t *color, int *ncolors) {
    clear_error();
    if (n < 0 || !rowptr || !col || (n > 0 && !color) || !ncolors) {
        set_error("nn_color_dsatur: need n >= 0, rowptr, col, color and ncolors");
        return NN_ERR_INVALID_ARG;
    }
    if (rowptr[0] != 0) {
        set_error("nn_color_dsatur: rowptr[0] must be 0");
        return NN_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) {
            set_error("nn_color_dsatur: rowptr must not decrease (row %lld)", (long long)i);
            return NN_ERR_INVALID_ARG;
        }
    for (int64_t q = 0; q < rowptr[n]; ++q)
        if (col[q] < 0 || col[q] >= n) {
            set_error("nn_color_dsatur: column %d at entry %lld is outside [0, %lld)", col[q], (long long)q,
                      (long long)n);
            return NN_ERR_INVALID_ARG;
        }
    if (n == 0) {
        *ncolors = 0;
        return NN_OK;
    }
    return dsatur_color(n, rowptr, col, color, ncolors);
}

nn_status nn_precond_setup(nn_system *s, void *stream) {
    clear_error();
    if (!s) {
        set_error("nn_precond_setup: NULL system");
        return NN_ERR_INVALID_ARG;
    }
    return ssor_setup(s, (cudaStream_t)stream);
}

nn_status nn_precond_apply(nn_system *s, int precond, double omega, const uint8_t *face, const double *r, double *z,
                           void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (!s || !r || !z || r == z || (precond != NN_PC_JACOBI && precond != NN_PC_SSOR) ||
        (precond == NN_PC_SSOR && !(omega > 0.0 && omega < 2.0))) {
        set_error("nn_precond_apply: need a system, distinct r and z, precond JACOBI or SSOR, 0 < omega < 2");
        return NN_ERR_INVALID_ARG;
    }
    if (s->NF == 0) return NN_OK;
    if (precond == NN_PC_SSOR) NN_TRY(ssor_setup(s, st));
    DevArena tmp;
    struct Release {
        DevArena &a;
        cudaStream_t st;
        ~Release() { a.release(st); }
    } rel{tmp, st};
    PcArgs a{};
    a.S = s->ssor;
    a.S.omega = omega;
    a.kind = precond;
    a.n = s->NF;
    a.fm = face;
    a.dinv = s->dinv64;
    a.r = r;
    a.z = z;
    a.timeout_ns = 5000000000ull;
    NN_TRY(tmp.alloc(&a.y, (size_t)s->NF, st));
    NN_TRY(tmp.alloc(&a.bar, 1, st));
    NN_CUDA_TRY(cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), st));
    int dev = 0, sms = 1, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    NN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_precond_apply, 256, 0));
    const int64_t need = precond == NN_PC_SSOR ? (s->ssor_slices + 7) / 8 : (s->NF + 255) / 256;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(per, 1) * sms));
    void *args[] = {&a};
    cudaError_t le = cudaLaunchCooperativeKernel((const void *)k_precond_apply, dim3(blocks), dim3(256), args, 0, st);
    count_launch();
    if (le != cudaSuccess) {
        set_error("nn_precond_apply: cooperative launch of %d blocks failed: %s", blocks, cudaGetErrorString(le));
        return NN_ERR_CUDA;
    }
    GridBarrier hb;
    NN_CUDA_TRY(cudaMemcpyAsync(&hb, a.bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb.error) {
        set_error("nn_precond_apply: a grid barrier gave up (wait #%d)", hb.where);
        return (nn_status)hb.error;
    }
    return NN_OK;
}

}  // extern "C"
