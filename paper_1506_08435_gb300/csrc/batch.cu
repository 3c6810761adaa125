// Batched solves, host side: per-instance scratch, the launch shape (threads
// per block x CTAs per instance), the autotuner and the per-instance records.
// The kernels are in batch.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>
#include "internal.h"
#include "batch.cuh"

namespace nnqp {

namespace {

BatchKernel pick_kernel(bool mixed, int tpb, int cluster, int cgv) {
    return mixed ? batch_kernel_mixed(tpb, cluster, cgv) : batch_kernel_fp64(tpb, cluster, cgv);
}

// Launch shape of the batch kernel: threads per block and CTAs per
// instance (1 = one block per instance, > 1 = a cluster per instance).
struct BatchShape {
    int tpb = 256;
    int cluster = 1;
};
BatchShape g_tuned;          // process-wide choice of the autotuner
bool g_have_tuned = false;

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
                           cudaStream_t st, BatchShape shape, nn_solve_info *infos, float *ms_out) {
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
        w64 += (size_t)11 * s->NF;
        if (mixed) w32 += (size_t)13 * s->NF;
    }
    Scratch S;
    S.st = st;
    double *d64;
    float *d32 = nullptr;
    uint8_t *dfm;
    NN_TRY(S.a.alloc(&d64, w64, st));
    if (mixed) NN_TRY(S.a.alloc(&d32, w32, st));
    NN_TRY(S.a.alloc(&dfm, w64 / 11, st));
    size_t o64 = 0, o32 = 0, ofm = 0;
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
        o64 += (size_t)11 * s->NF;
        b.fm = dfm + ofm;
        ofm += (size_t)s->NF;
        if (mixed) {
            b.w32 = d32 + o32;
            o32 += (size_t)13 * s->NF;
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
    ctl.keep_p = 0;
    if (const char *e = getenv("NNQP_BATCH_CG_VARIANT")) ctl.cg_variant = atoi(e);
    if (const char *e = getenv("NNQP_CG_BOUND_STOP")) ctl.cg_bound_stop = atoi(e);
    if (const char *e = getenv("NNQP_GP_MAX")) ctl.gp_max = atoi(e);
    if (const char *e = getenv("NNQP_ETA1")) ctl.eta1 = atof(e);
    if (const char *e = getenv("NNQP_ETA2")) ctl.eta2 = atof(e);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tpb = shape.cluster > 1 ? 256 : shape.tpb;
    BatchKernel k = pick_kernel(mixed, tpb, shape.cluster, ctl.cg_variant);
    if (!k) {
        set_error("nn_batch_solve: no kernel for %d threads x %d CTAs, CG variant %d", tpb, shape.cluster,
                  ctl.cg_variant);
        return NN_ERR_INVALID_ARG;
    }
    cudaEvent_t e0, e1;
    NN_CUDA_TRY(cudaEventCreate(&e0));
    NN_CUDA_TRY(cudaEventCreate(&e1));
    if (shape.cluster <= 1) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, tpb, 0);
        const int grid = std::max(1, std::min(count, std::max(per, 1) * sms));
        cudaEventRecord(e0, st);
        (k<<<grid, tpb, 0, st>>>(dinst, dorder, count, dnext, ctl, o->rtol, o->inner_rtol, 200, dcnt, dsc),
         count_launch());
    } else {
        const int C = shape.cluster;
        if (C > 8) NN_CUDA_TRY(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(256);
        cfg.gridDim = dim3(C * std::max(1, sms / C));
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        NN_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, (const void *)k, &cfg));
        if (nclusters < 1) {
            set_error("nn_batch_solve: clusters of %d CTAs cannot be scheduled on this device", C);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return NN_ERR_INVALID_ARG;
        }
        cfg.gridDim = dim3(C * std::min(count, nclusters));
        cudaEventRecord(e0, st);
        NN_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, (const BatchInst *)dinst, (const int *)dorder, count, dnext, ctl,
                                       o->rtol, o->inner_rtol, 200, dcnt, dsc));
        count_launch();
    }
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
    if (o->precond != NN_PC_JACOBI) {
        set_error("batched solves use the Jacobi preconditioner");
        return NN_ERR_INVALID_ARG;
    }
    if (count < 1 || !systems || !c) {
        set_error("nn_batch_solve: count >= 1 and arrays are required");
        return NN_ERR_INVALID_ARG;
    }
    BatchShape shape;
    if (g_have_tuned) shape = g_tuned;
    // NNQP_BATCH_SHAPE="<threads>x<ctas>" overrides the shape (tests, sweeps)
    if (const char *e = getenv("NNQP_BATCH_SHAPE")) {
        int t = 0, c = 0;
        if (sscanf(e, "%dx%d", &t, &c) == 2 && (t == 128 || t == 256 || t == 512) && c >= 1 && c <= kMaxCluster &&
            (c & (c - 1)) == 0) {
            shape.tpb = c > 1 ? 256 : t;
            shape.cluster = c;
        }
    }
    return run_batch(count, systems, c, o, (cudaStream_t)stream, shape, infos, nullptr);
}

nn_status nn_batch_autotune(int count, nn_system *const *systems, const nn_solve_opts *o, void *stream,
                            int *best_shape) {
    clear_error();
    nn_solve_opts d;
    nn_solve_opts_default(&d);
    if (!o) o = &d;
    NN_TRY(check_opts(o));
    if (o->precond != NN_PC_JACOBI) {
        set_error("batched solves use the Jacobi preconditioner");
        return NN_ERR_INVALID_ARG;
    }
    if (count < 1 || !systems) {
        set_error("nn_batch_autotune: count >= 1 and systems are required");
        return NN_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // Every candidate shape solves the whole batch to the requested tolerance
    // and the shape with the shortest elapsed time wins: the makespan depends
    // on how many instances run side by side as much as on how fast each one
    // runs, so a sample of the batch misjudges it (measured: a quarter of the
    // batch picked 16 CTAs per instance, 19% slower on the whole batch than 8).
    // One block per instance is a candidate only for batches of small
    // instances; clusters win as soon as an instance has thousands of rows.
    std::vector<nn_system *> sample(systems, systems + count);
    int64_t largest = 0;
    for (int i = 0; i < count; ++i) largest = std::max<int64_t>(largest, systems[i]->NF);
    const int ns = (int)sample.size();
    Scratch S;
    S.st = st;
    std::vector<double *> cs(ns);
    for (int i = 0; i < ns; ++i) NN_TRY(S.a.alloc(&cs[i], sample[i]->N, st));
    nn_solve_opts t = *o;
    std::vector<BatchShape> cands;
    if (largest <= 8192) {
        cands = {{256, 1}, {512, 1}, {256, 4}, {256, 8}};
    } else {
        cands = {{256, 4}, {256, 8}, {256, 16}};
    }
    float best = 1e30f;
    BatchShape pick_shape;
    std::vector<nn_solve_info> inf(ns);
    for (const BatchShape &sh : cands) {
        for (int i = 0; i < ns; ++i) NN_CUDA_TRY(cudaMemsetAsync(cs[i], 0, sizeof(double) * sample[i]->N, st));
        float ms = 0.0f;
        nn_status r = run_batch(ns, sample.data(), cs.data(), &t, st, sh, inf.data(), &ms);
        if (r == NN_ERR_INVALID_ARG) continue;   // shape not schedulable here
        if (r != NN_OK && r != NN_ERR_NOT_CONVERGED) return r;
        if (ms < best) {
            best = ms;
            pick_shape = sh;
        }
    }
    g_tuned = pick_shape;
    g_have_tuned = true;
    if (best_shape) *best_shape = pick_shape.tpb * 100 + pick_shape.cluster;
    clear_error();
    return NN_OK;
}

}  // extern "C"
