// Batched solves: many independent QPs of uneven size in ONE persistent
// launch.  Every thread block takes the next instance (largest first) from
// a device work counter and solves it alone with block-level barriers and
// reductions, so no block ever waits on another.  The solver is the same
// GPCG (and mixed-precision refinement) code as the single-system path,
// instantiated for a one-block team.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>
#include "internal.h"
#include "gpcg.cuh"
#include "refine.cuh"

namespace nnqp {

struct BatchInst {
    int64_t n, N, nslices;
    const int64_t *sptr;
    const int32_t *col;
    const double *val;
    const double *diag;
    const double *dinv64;
    const float *val32;
    const float *rsum32;
    const float *dinv32;
    const double *b0;
    const int32_t *free_node;
    const uint8_t *dmask;
    const double *dval;
    double lo, hi, den;
    double *c;          // full node vector: warm start in, solution out
    double *w64;        // 10 n doubles
    float *w32;         // 12 n floats (mixed)
};

constexpr int kBatchCounters = 9;

template <int TPB, int MIXED>
__global__ void __launch_bounds__(TPB) k_batch(const BatchInst *__restrict__ insts, const int *__restrict__ order,
                                               int count, unsigned *next, GpcgCtl ctl, double rtol,
                                               double inner_rtol, int max_ref, int64_t *counters, double *scalars) {
    __shared__ RedSmem sm;
    __shared__ int s_q;
    BlockTeam T{&sm};
    for (;;) {
        if (threadIdx.x == 0) s_q = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= count) return;
        const int id = order[q];
        const BatchInst I = insts[id];
        const int64_t n = I.n;
        const Rows R{0, I.nslices, n};
        double *x = I.w64;
        R.each([&](int64_t i) { x[i] = I.c[I.free_node[i]]; });
        __syncthreads();
        const SellF64 A{n, I.nslices, I.sptr, I.col, I.val, I.diag};
        int64_t cnt[kBatchCounters] = {0};
        double gp2 = 0.0;
        int status;
        if (MIXED) {
            float *w = I.w32;
            GpcgVecs<float> v{w, w + n, w + 2 * n, w + 3 * n, w + 4 * n, w + 5 * n, w + 6 * n, w + 7 * n, w + 8 * n,
                              w + 9 * n, I.dinv32};
            const SellF32Diff A32{n, I.nslices, I.sptr, I.col, I.val32, I.rsum32};
            double *w6 = I.w64;
            GpcgVecs<double> v64{x, w6 + n, w6 + 2 * n, w6 + 3 * n, w6 + 4 * n, w6 + 5 * n, w6 + 6 * n,
                                 w6 + 7 * n, w6 + 8 * n, I.b0, I.dinv64};
            MixedStats ms;
            status = mixed_solve(T, R, A, A32, I.lo, I.hi, I.b0, x, v, w + 9 * n, w + 10 * n, w + 11 * n, v64,
                                 rtol * I.den, inner_rtol, max_ref, ctl.max_spmv, inner_product_cap(n), ctl, ctl,
                                 ms);
            cnt[1] = ms.spmv64;
            cnt[2] = ms.spmv32;
            cnt[3] = ms.cg;
            cnt[4] = ms.phases;
            cnt[5] = ms.refinements;
            cnt[6] = ms.vec64;
            cnt[7] = ms.vec32;
            cnt[8] = ms.fallback;
            gp2 = ms.gp2;
        } else {
            double *w = I.w64;
            GpcgVecs<double> v{w, w + n, w + 2 * n, w + 3 * n, w + 4 * n, w + 5 * n, w + 6 * n, w + 7 * n,
                               w + 8 * n, I.b0, I.dinv64};
            GpcgCtl c = ctl;
            c.tol = rtol * I.den;
            c.face_tol = 0.5 * c.tol;
            GpcgStats gs;
            status = gpcg_solve(T, R, A, Bounds<double>{I.lo, I.hi, nullptr, nullptr}, v, c, gs);
            x = v.x;
            cnt[1] = gs.spmv;
            cnt[3] = gs.cg;
            cnt[4] = gs.phases;
            cnt[6] = gs.vec;
            gp2 = gs.gp2;
        }
        R.each([&](int64_t i) { I.c[I.free_node[i]] = x[i]; });
        for (int64_t v = threadIdx.x; v < I.N; v += blockDim.x)
            if (I.dmask[v]) I.c[v] = I.dval[v];
        if (threadIdx.x == 0) {
            cnt[0] = status;
            for (int k = 0; k < kBatchCounters; ++k) counters[(int64_t)id * kBatchCounters + k] = cnt[k];
            scalars[2 * id] = gp2;
            scalars[2 * id + 1] = I.den;
        }
        __syncthreads();
    }
}

namespace {

using BatchKernel = void (*)(const BatchInst *, const int *, int, unsigned *, GpcgCtl, double, double, int,
                             int64_t *, double *);

BatchKernel pick(int tpb, bool mixed) {
    switch (tpb) {
        case 128: return mixed ? k_batch<128, 1> : k_batch<128, 0>;
        case 512: return mixed ? k_batch<512, 1> : k_batch<512, 0>;
        default: return mixed ? k_batch<256, 1> : k_batch<256, 0>;
    }
}

int g_tuned_tpb = 0;   // process-wide choice of the autotuner (0: default 256)

double bytes_spmv(int64_t nnz, int64_t n, int sv, int sx) {
    return (double)nnz * (sv + 4) + 4.0 * (n + 1) + 2.0 * sx * n;
}

struct Scratch {
    DevArena a;
    cudaStream_t st;
    ~Scratch() { a.release(st); }
};

double den_of(const nn_system *s) {
    if (s->b0norm > 0.0) return s->b0norm;
    double m = 1.0;
    if (std::isfinite(s->lo)) m = std::max(m, std::fabs(s->lo));
    if (std::isfinite(s->hi)) m = std::max(m, std::fabs(s->hi));
    double d = s->anorm_inf * m;
    return d > 0 ? d : 1.0;
}

}  // namespace

nn_status check_opts(const nn_solve_opts *o);

// Runs the batch kernel; returns elapsed device milliseconds in *ms.
static nn_status run_batch(int count, nn_system *const *systems, double *const *c, const nn_solve_opts *o,
                           cudaStream_t st, int tpb, nn_solve_info *infos, float *ms_out) {
    const bool mixed = o->precision == NN_PREC_MIXED;
    if (o->solver != NN_SOLVER_GPCG || o->format != NN_FMT_SELL) {
        set_error("nn_batch_solve runs GPCG on the SELL format");
        return NN_ERR_INVALID_ARG;
    }
    std::vector<BatchInst> h(count);
    size_t w64 = 0, w32 = 0;
    for (int i = 0; i < count; ++i) {
        const nn_system *s = systems[i];
        if (!s || !c[i]) {
            set_error("nn_batch_solve: NULL system or vector at %d", i);
            return NN_ERR_INVALID_ARG;
        }
        if (s->dt > 0.0) {
            set_error("nn_batch_solve: system %d is transient", i);
            return NN_ERR_INVALID_ARG;
        }
        if (mixed && !s->has_mixed) {
            set_error("nn_batch_solve: system %d has no FP32 copy", i);
            return NN_ERR_INVALID_ARG;
        }
        w64 += (size_t)10 * s->NF;
        if (mixed) w32 += (size_t)12 * s->NF;
    }
    Scratch S;
    S.st = st;
    double *d64;
    float *d32 = nullptr;
    NN_TRY(S.a.alloc(&d64, w64, st));
    if (mixed) NN_TRY(S.a.alloc(&d32, w32, st));
    size_t o64 = 0, o32 = 0;
    for (int i = 0; i < count; ++i) {
        const nn_system *s = systems[i];
        BatchInst &b = h[i];
        b.n = s->NF;
        b.N = s->N;
        b.nslices = s->A64.nslices;
        b.sptr = s->A64.sptr;
        b.col = s->A64.col;
        b.val = s->A64.val;
        b.diag = s->diag64;
        b.dinv64 = s->dinv64;
        b.val32 = s->A32.val;
        b.rsum32 = s->rsum32;
        b.dinv32 = s->dinv32;
        b.b0 = s->b0;
        b.free_node = s->free_node;
        b.dmask = s->dmask;
        b.dval = s->dval;
        b.lo = s->lo;
        b.hi = s->hi;
        b.den = den_of(s);
        b.c = c[i];
        b.w64 = d64 + o64;
        o64 += (size_t)10 * s->NF;
        if (mixed) {
            b.w32 = d32 + o32;
            o32 += (size_t)12 * s->NF;
        } else {
            b.w32 = nullptr;
        }
    }
    // largest first
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return systems[a]->nnzF > systems[b]->nnzF; });
    BatchInst *dinst;
    int *dorder;
    unsigned *dnext;
    int64_t *dcnt;
    double *dsc;
    NN_TRY(S.a.alloc(&dinst, count, st));
    NN_TRY(S.a.alloc(&dorder, count, st));
    NN_TRY(S.a.alloc(&dnext, 1, st));
    NN_TRY(S.a.alloc(&dcnt, (size_t)count * kBatchCounters, st));
    NN_TRY(S.a.alloc(&dsc, (size_t)2 * count, st));
    NN_CUDA_TRY(cudaMemcpyAsync(dinst, h.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, st));
    NN_CUDA_TRY(cudaMemcpyAsync(dorder, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
    NN_CUDA_TRY(cudaMemsetAsync(dnext, 0, sizeof(unsigned), st));
    NN_CUDA_TRY(cudaMemsetAsync(dcnt, 0, sizeof(int64_t) * count * kBatchCounters, st));
    GpcgCtl ctl;
    ctl.tol = 0;
    ctl.face_tol = 0;
    ctl.max_spmv = o->max_iter;
    ctl.gp_max = 50;
    ctl.cg_max = 1 << 30;
    ctl.eta1 = 0.1;
    ctl.eta2 = 1e-3;
    ctl.mu = 1e-4;
    ctl.cg_variant = 0;
    ctl.cg_bound_stop = 0;
    if (const char *e = getenv("NNQP_BATCH_CG_VARIANT")) ctl.cg_variant = atoi(e);
    if (const char *e = getenv("NNQP_CG_BOUND_STOP")) ctl.cg_bound_stop = atoi(e);
    if (const char *e = getenv("NNQP_GP_MAX")) ctl.gp_max = atoi(e);
    if (const char *e = getenv("NNQP_ETA2")) ctl.eta2 = atof(e);
    BatchKernel k = pick(tpb, mixed);
    int per = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, tpb, 0);
    const int grid = std::max(1, std::min(count, std::max(per, 1) * sms));
    cudaEvent_t e0, e1;
    NN_CUDA_TRY(cudaEventCreate(&e0));
    NN_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    (k<<<grid, tpb, 0, st>>>(dinst, dorder, count, dnext, ctl, o->rtol, o->inner_rtol, 200, dcnt, dsc),
     count_launch());
    cudaEventRecord(e1, st);
    std::vector<int64_t> hc((size_t)count * kBatchCounters);
    std::vector<double> hs((size_t)2 * count);
    NN_CUDA_TRY(cudaMemcpyAsync(hc.data(), dcnt, sizeof(int64_t) * hc.size(), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaMemcpyAsync(hs.data(), dsc, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    NN_CUDA_TRY(cudaGetLastError());
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_out) *ms_out = ms;
    nn_status worst = NN_OK;
    for (int i = 0; i < count; ++i) {
        const int64_t *q = &hc[(size_t)i * kBatchCounters];
        nn_solve_info inf;
        std::memset(&inf, 0, sizeof(inf));
        inf.status = (int)q[0];
        inf.spmv64 = q[1];
        inf.spmv = q[1] + q[2];
        inf.cg_iters = q[3];
        inf.iterations = q[4];
        inf.refinements = q[5];
        inf.fp64_fallback = q[8];
        inf.kkt_rel = std::sqrt(hs[2 * i]) / hs[2 * i + 1];
        inf.kkt_inf = NAN;
        inf.objective = NAN;
        inf.time_ms = i == 0 ? ms : 0.0;
        const nn_system *s = systems[i];
        inf.bytes_algo = q[1] * bytes_spmv(s->nnzF, s->NF, 8, 8) + q[2] * bytes_spmv(s->nnzF, s->NF, 4, 4) +
                         (double)q[6] * 8.0 * s->NF + (double)q[7] * 4.0 * s->NF;
        if (infos) infos[i] = inf;
        if (inf.status != NN_OK && worst == NN_OK) worst = (nn_status)inf.status;
    }
    if (worst == NN_ERR_NOT_CONVERGED) set_error("some batch instances reached the iteration cap");
    return worst;
}

}  // namespace nnqp

using namespace nnqp;

extern "C" {

nn_status nn_batch_solve(int count, nn_system *const *systems, double *const *c, const nn_solve_opts *o,
                         void *stream, nn_solve_info *infos) {
    clear_error();
    nn_solve_opts d;
    nn_solve_opts_default(&d);
    if (!o) o = &d;
    NN_TRY(check_opts(o));
    if (count < 1 || !systems || !c) {
        set_error("nn_batch_solve: count >= 1 and arrays are required");
        return NN_ERR_INVALID_ARG;
    }
    const int tpb = g_tuned_tpb ? g_tuned_tpb : 256;
    return run_batch(count, systems, c, o, (cudaStream_t)stream, tpb, infos, nullptr);
}

nn_status nn_batch_autotune(int count, nn_system *const *systems, const nn_solve_opts *o, void *stream,
                            int *best_threads) {
    clear_error();
    nn_solve_opts d;
    nn_solve_opts_default(&d);
    if (!o) o = &d;
    NN_TRY(check_opts(o));
    if (count < 1 || !systems) {
        set_error("nn_batch_autotune: count >= 1 and systems are required");
        return NN_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // a sample of up to 64 instances, each solved for a short fixed budget of
    // products from zero; the shape with the most products per second wins
    const int ns = std::min(count, 64);
    std::vector<nn_system *> sample(ns);
    for (int i = 0; i < ns; ++i) sample[i] = systems[(int64_t)i * count / ns];
    Scratch S;
    S.st = st;
    std::vector<double *> cs(ns);
    for (int i = 0; i < ns; ++i) {
        NN_TRY(S.a.alloc(&cs[i], sample[i]->N, st));
    }
    nn_solve_opts t = *o;
    t.max_iter = 120;
    const int cands[3] = {128, 256, 512};
    double best = -1.0;
    int best_tpb = 256;
    std::vector<nn_solve_info> inf(ns);
    for (int rep = 0; rep < 2; ++rep) {
        for (int cidx = 0; cidx < 3; ++cidx) {
            for (int i = 0; i < ns; ++i) NN_CUDA_TRY(cudaMemsetAsync(cs[i], 0, sizeof(double) * sample[i]->N, st));
            float ms = 0.0f;
            nn_status r = run_batch(ns, sample.data(), cs.data(), &t, st, cands[cidx], inf.data(), &ms);
            if (r != NN_OK && r != NN_ERR_NOT_CONVERGED) return r;
            double work = 0.0;
            for (int i = 0; i < ns; ++i) work += (double)inf[i].spmv * (double)sample[i]->nnzF;
            const double rate = work / std::max(ms, 1e-3f);
            if (rep == 1 && rate > best) {
                best = rate;
                best_tpb = cands[cidx];
            }
        }
    }
    g_tuned_tpb = best_tpb;
    if (best_threads) *best_threads = best_tpb;
    clear_error();
    return NN_OK;
}

}  // extern "C"
