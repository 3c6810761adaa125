// Single-system solves, host side: scratch, grid sizing and the cooperative
// launch of the persistent solve kernels (grid.cuh), the projected L-BFGS
// and TRON driver kernels, the FP64 KKT measure and the stand-alone products.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include "internal.h"
#include "grid.cuh"
#include "lbfgs.cuh"
#include "tron.cuh"

namespace nnqp {

// The same driver with the projected L-BFGS solver (FP64, SELL).
__global__ void __launch_bounds__(kSolveThreads) k_lbfgs_grid(GridArgs a) {
    __shared__ RedSmem sm;
    __shared__ LbSmem lsm;
    GridTeam T{a.bar, a.partials, (int)gridDim.x + a.bar_extra, a.timeout_ns, 0, 0, &sm};
    const Rows R = rows_of_block(a.n, a.nslices, blockIdx.x, gridDim.x);
    double *x0 = a.v64[0];
    R.each([&](int64_t i) { x0[i] = a.c_in[a.free_node[i]]; });
    if (!T.sync()) return;
    const int nsteps = a.mode == MODE_TRANSIENT ? a.nsteps : 1;
    for (int step = 0; step < nsteps; ++step) {
        int64_t cnt[kCounters] = {0};
        double den = a.b0norm;
        double *b = const_cast<double *>(a.b0);
        if (a.mode == MODE_TRANSIENT) {
            if (!transient_rhs(T, R, a, x0, b, den)) return;
            transient_predict<GridTeam>(R, a, x0, step);
            cnt[1] += 1;
        }
        if (!(den > 0.0)) den = a.den_fallback;
        double *x = x0, *g = a.v64[1], *w = a.v64[7], *gw = a.v64[8];
        LbCtl c{a.rtol * den, a.ctl.max_spmv, a.m, a.ctl.mu, a.h0};
        LbStats ls;
        const int status = lbfgs_solve(T, R, a.A, a.lo, a.hi, b, x, g, a.v64[2], w, gw, a.S, a.Y, a.n, c, ls, lsm);
        if (status == ST_TIMEOUT) return;
        if (x != x0) {
            R.each([&](int64_t i) { x0[i] = x[i]; });
            if (!T.sync()) return;
        }
        cnt[1] += ls.spmv;
        cnt[4] = ls.iters;
        cnt[6] = ls.vec;
        cnt[10] = ls.resets;
        if (!step_outputs(T, R, a, x0, step, nsteps, status, cnt, ls.gp2, den)) return;
    }
}

// The same driver with the trust-region Newton solver (FP64, SELL).
__global__ void __launch_bounds__(kSolveThreads, 2) k_tron_grid(GridArgs a) {
    __shared__ RedSmem sm;
    GridTeam T{a.bar, a.partials, (int)gridDim.x + a.bar_extra, a.timeout_ns, 0, 0, &sm};
    const Rows R = rows_of_block(a.n, a.nslices, blockIdx.x, gridDim.x);
    double *x0 = a.v64[0];
    R.each([&](int64_t i) { x0[i] = a.c_in[a.free_node[i]]; });
    if (!T.sync()) return;
    const int nsteps = a.mode == MODE_TRANSIENT ? a.nsteps : 1;
    const Bounds<double> B{a.lo, a.hi, nullptr, nullptr};
    for (int step = 0; step < nsteps; ++step) {
        int64_t cnt[kCounters] = {0};
        double den = a.b0norm;
        double *b = const_cast<double *>(a.b0);
        if (a.mode == MODE_TRANSIENT) {
            if (!transient_rhs(T, R, a, x0, b, den)) return;
            transient_predict<GridTeam>(R, a, x0, step);
            cnt[1] += 1;
            cnt[12] += 4;
        }
        if (!(den > 0.0)) den = a.den_fallback;
        const SsorF64 pcv = a.pc;
        TronVecs v{x0, a.v64[1], a.v64[7], a.v64[8], a.v64[2], a.v64[3], a.v64[4], a.v64[5], a.v64[6],
                   a.v64[10], b, a.dinv64, a.fmask, a.pc.ncolors > 0 ? &pcv : nullptr};
        const TronCtl c{a.rtol * den, 0.5 * a.rtol * den, a.ksp_rtol, a.ctl.max_spmv, 50};
        TronStats ts;
        const int status = tron_solve(T, R, a.A, B, v, c, ts);
        if (status == ST_TIMEOUT) return;
        if (v.x != x0) {
            const double *xs = v.x;
            R.each([&](int64_t i) { x0[i] = xs[i]; });
            if (!T.sync()) return;
        }
        cnt[1] += ts.spmv;
        cnt[3] = ts.cg;
        cnt[4] = ts.iters;
        cnt[6] = ts.vec;
        cnt[10] = ts.pc;
        cnt[12] += ts.fl;
        if (!step_outputs(T, R, a, x0, step, nsteps, status, cnt, ts.gp2, den)) return;
    }
}

__global__ void k_fill_dirichlet(int64_t N, const uint8_t *dmask, const double *dval, double *c, int nrep,
                                 int64_t stride) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= N || !dmask[v]) return;
    for (int r = 0; r < nrep; ++r) c[r * stride + v] = dval[v];
}

// ------------------------------------------------------------------ KKT (FP64)

// g = A x - b with b = b0 (+ M x_prev / dt); partial sums per block of
// |gP|^2, max |gP|, |b|^2, max |b|, x'Ax - 2 b'x, infeasible count.
__global__ void __launch_bounds__(256) k_kkt(SellF64 A, SellF64 M, int transient, double inv_dt,
                                             const double *b0, const double *x, const double *xprev,
                                             double lo, double hi, double *part) {
    __shared__ double sm[8][6];
    const Rows R = rows_of_block(A.n, A.nslices, blockIdx.x, gridDim.x);
    double s[6] = {0, 0, 0, 0, 0, 0};
    A.apply(R, x, [&](int64_t i, double ax) {
        double bi = b0[i];
        if (transient) bi += M.row_product(i, xprev) * inv_dt;   // (M x_prev)_i, row-wise
        const double xi = x[i];
        const double g = ax - bi;
        const double gp = proj_grad(xi, g, lo, hi);
        s[0] += gp * gp;
        s[1] = fmax(s[1], fabs(gp));
        s[2] += bi * bi;
        s[3] = fmax(s[3], fabs(bi));
        s[4] += xi * (ax - 2.0 * bi);
        s[5] += (xi >= lo && xi <= hi) ? 0.0 : 1.0;
    });
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
        s[1] = fmax(s[1], __shfl_xor_sync(0xffffffffu, s[1], o));
        s[2] += __shfl_xor_sync(0xffffffffu, s[2], o);
        s[3] = fmax(s[3], __shfl_xor_sync(0xffffffffu, s[3], o));
        s[4] += __shfl_xor_sync(0xffffffffu, s[4], o);
        s[5] += __shfl_xor_sync(0xffffffffu, s[5], o);
    }
    if (lane == 0)
        for (int k = 0; k < 6; ++k) sm[warp][k] = s[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t[0] += sm[w][0];
            t[1] = fmax(t[1], sm[w][1]);
            t[2] += sm[w][2];
            t[3] = fmax(t[3], sm[w][3]);
            t[4] += sm[w][4];
            t[5] += sm[w][5];
        }
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = t[k];
    }
}

__global__ void k_gather_free(int64_t n, const int32_t *free_node, const double *c, double *x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = c[free_node[i]];
}

// y = A x as a standalone product (FP64 SELL or CSR, or the FP32 operator).
__global__ void __launch_bounds__(256) k_spmv64(SellF64 A, const double *x, double *y) {
    const Rows R = rows_of_block(A.n, A.nslices, blockIdx.x, gridDim.x);
    A.apply(R, x, [&](int64_t i, double v) { y[i] = v; });
}
__global__ void __launch_bounds__(256) k_spmvcsr(CsrF64 A, const double *x, double *y) {
    const Rows R = rows_of_block(A.n, A.nslices, blockIdx.x, gridDim.x);
    A.apply(R, x, [&](int64_t i, double v) { y[i] = v; });
}
__global__ void k_to_f32(int64_t n, const double *x, float *y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}
__global__ void __launch_bounds__(256) k_spmv32(SellF32Diff A, const float *x, double *y) {
    const Rows R = rows_of_block(A.n, A.nslices, blockIdx.x, gridDim.x);
    A.apply(R, x, [&](int64_t i, float v) { y[i] = (double)v; });
}

// ------------------------------------------------------------------ host side

namespace {

// Operators larger than this stream through L2 (evict-first loads, slice prefetch).
constexpr double kStreamBytes = 48.0 * (1 << 20);
// Most shared memory a block's staged operator slices may take.
constexpr size_t kSmemOperatorBytes = 192 * 1024;
// Shared-memory budget of the streamed FP32 operator's slots per block: one
// 768-thread block per SM, 24 warps x 2 slots of 32 rows x up to 16 entries
// x 8 bytes, plus a 2 KB header.
constexpr size_t kTmaSmemBytes = 196 * 1024;
// Threads per block of the large-system grids (one block per SM), and of
// the large mixed grid where the streamed operator does not apply.
constexpr int kLargeThreads = 768;
constexpr int kLargeThreadsLoads = 512;
// Threads per block of the projected L-BFGS kernel (128 was measured too:
// faster on the 50^2 problem, slower on the 40^3 transient run).
constexpr int kLbfgsThreads = 256;

SellF64 view64(const nn_system *s) {
    return SellF64{s->NF, s->A64.nslices, s->A64.sptr, s->A64.col, s->A64.val, s->diag64,
                   (double)s->nnzF * 12.0 > kStreamBytes};
}
SellF64 viewM(const nn_system *s) {
    return SellF64{s->NF, s->M64.nslices, s->M64.sptr, s->M64.col, s->M64.val, s->mdiag64};
}
SellF32Diff view32(const nn_system *s) {
    return SellF32Diff{s->NF, s->A32.nslices, s->A32.sptr, s->A32.col, s->A32.val, s->rsum32,
                       (double)s->nnzF * 8.0 > kStreamBytes};
}
CsrF64 viewcsr(const nn_system *s) { return CsrF64{s->NF, s->A64.nslices, s->arow, s->acol, s->aval}; }

double den_fallback(const nn_system *s) {
    double m = 1.0;
    if (std::isfinite(s->lo)) m = std::max(m, std::fabs(s->lo));
    if (std::isfinite(s->hi)) m = std::max(m, std::fabs(s->hi));
    double d = s->anorm_inf * m;
    return d > 0 ? d : 1.0;
}

int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

template <typename K>
int max_coresident(K kern, int tpb = kSolveThreads) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, tpb, 0);
    return std::max(per, 1) * device_sms();
}

GridKernel grid_kernel(int mode, int fmt, int cgv, int tpb = kSolveThreads) {
    switch (mode) {
        case MODE_TRANSIENT: return grid_kernel_transient(fmt, cgv, tpb);
        case MODE_MIXED: return grid_kernel_mixed(fmt, cgv, tpb);
        case MODE_MIXED_TR: return grid_kernel_mixed_transient(fmt, cgv, tpb);
        default: return grid_kernel_steady(fmt, cgv, tpb);
    }
}

// algorithmic bytes of one product (paper's MatMult model, Sec. 4):
// nnz (s_v + 4) + 4 (n + 1) + s_x n (x read) + s_x n (y written)
double bytes_spmv(int64_t nnz, int64_t n, int sv, int sx) {
    return (double)nnz * (sv + 4) + 4.0 * (n + 1) + 2.0 * sx * n;
}

struct Scratch {
    DevArena a;
    cudaStream_t st;
    ~Scratch() { a.release(st); }
};

}  // namespace

// algorithmic bytes of one SSOR application (ssor.cuh): every off-diagonal
// entry once (value + column), the row ids of both sweeps, and per row the
// forward sweep's r, 1/a_ii, face byte, y written and y gathered, the
// backward sweep's y, 1/a_ii, face byte, z written and z gathered
double bytes_ssor(int64_t nnz, int64_t n) { return 12.0 * (double)(nnz - n) + 74.0 * (double)n; }

// its operations: a multiply-add per off-diagonal entry, 7 per row
double flops_ssor(int64_t nnz, int64_t n) { return 2.0 * (double)(nnz - n) + 7.0 * (double)n; }

void fill_info(const nn_system *s, const int64_t *cnt, const double *sc, int precision, int precond,
               nn_solve_info *info) {
    std::memset(info, 0, sizeof(*info));
    info->status = (int)cnt[0];
    info->spmv64 = cnt[1];
    info->spmv = cnt[1] + cnt[2];
    info->cg_iters = cnt[3];
    info->iterations = cnt[4];
    info->refinements = cnt[5];
    info->active_lo = cnt[8];
    info->active_hi = cnt[9];
    info->fp64_fallback = cnt[11];
    info->pc_applies = precond == NN_PC_SSOR ? cnt[10] : 0;   // (slot 10 holds L-BFGS resets otherwise)
    info->flops64_algo = 2.0 * cnt[1] * (double)s->nnzF + (double)cnt[12] * s->NF +
                         (double)info->pc_applies * flops_ssor(s->nnzF, s->NF);
    info->flops_algo = info->flops64_algo + 2.0 * cnt[2] * (double)s->nnzF + (double)cnt[13] * s->NF;
    info->kkt_rel = std::sqrt(sc[0]) / sc[1];
    info->kkt_inf = NAN;
    info->objective = NAN;
    info->bytes_algo = cnt[1] * bytes_spmv(s->nnzF, s->NF, 8, 8) + cnt[2] * bytes_spmv(s->nnzF, s->NF, 4, 4) +
                       (double)cnt[6] * 8.0 * s->NF + (double)cnt[7] * 4.0 * s->NF +
                       (double)info->pc_applies * bytes_ssor(s->nnzF, s->NF);
    (void)precision;
}

// Everything one persistent solve launch needs, built once: arguments,
// scratch, kernel, grid and shared memory.  A plan can be launched many times
// (stream-ordered, without host synchronisation) and its results read after.
struct GridPlan {
    nn_system *s = nullptr;
    nn_solve_opts o{};
    int mode = 0, nsteps = 1;
    GridArgs a{};
    GridKernel kern = nullptr;
    int want = 1, tpb = kSolveThreads;
    size_t dyn_smem = 0;
    DevArena arena;
};

// Builds plan P (its scratch is allocated on stream st).  force_tpb = 256 or
// 512 fixes the threads per block (serving decides the launch shape before
// admission); 0 lets the size decide.
nn_status plan_build(nn_system *s, const nn_solve_opts *o, int mode, int nsteps, cudaStream_t st, GridPlan &P,
                     int force_tpb = 0) {
    const int64_t n = s->NF, N = s->N;
    const bool mixed = mode_mixed(mode);
    const int fmt = o->format;
    if (mixed && !s->has_mixed) {
        set_error("mixed precision needs a system assembled with build_mixed = 1");
        return NN_ERR_INVALID_ARG;
    }
    if (mode_transient(mode) && !(s->dt > 0.0)) {
        set_error("transient solve on a steady system (dt = 0)");
        return NN_ERR_INVALID_ARG;
    }
    if (!mode_transient(mode) && s->dt > 0.0) {
        set_error("steady solve on a transient system: use nn_step or nn_transient");
        return NN_ERR_INVALID_ARG;
    }
    if (fmt == NN_FMT_CSR && mixed) {
        set_error("CSR format is available in FP64 only");
        return NN_ERR_INVALID_ARG;
    }
    const bool ssor = o->precond == NN_PC_SSOR;
    if (ssor && (mixed || fmt != NN_FMT_SELL || o->solver == NN_SOLVER_LBFGS)) {
        set_error("the SSOR preconditioner runs in FP64 on the SELL format with GPCG or TRON");
        return NN_ERR_INVALID_ARG;
    }
    if (ssor) NN_TRY(ssor_setup(s, st));
    P.s = s;
    P.o = *o;
    P.mode = mode;
    P.nsteps = nsteps;
    DevArena &SA = P.arena;
    GridArgs &a = P.a;
    std::memset(&a, 0, sizeof(a));
    a.mode = mode;
    a.n = n;
    a.N = N;
    a.nslices = s->A64.nslices;
    a.A = view64(s);
    a.Acsr = viewcsr(s);
    if (s->has_mixed) a.A32 = view32(s);
    if (s->dt > 0.0) a.M = viewM(s);
    a.lo = s->lo;
    a.hi = s->hi;
    a.inv_dt = s->dt > 0.0 ? 1.0 / s->dt : 0.0;
    a.b0 = s->b0;
    a.dinv64 = s->dinv64;
    a.dinv32 = s->dinv32;
    a.free_node = s->free_node;
    a.nsteps = nsteps;
    for (int k = 0; k < 11; ++k) NN_TRY(SA.alloc(&a.v64[k], n, st));
    NN_TRY(SA.alloc(&a.fmask, n, st));
    if (mixed)
        for (int k = 0; k < 13; ++k) NN_TRY(SA.alloc(&a.v32[k], n, st));
    a.ctl.max_spmv = o->max_iter;
    // gradient-projection steps per phase: a warm-started time step has few
    // active-set changes to find, and short GP phases win there (measured on
    // the 40^3 transient run: 3 steps -10% products); steady solves from zero
    // need the long phases
    a.ctl.gp_max = mode_transient(mode) ? 3 : 50;
    a.ctl.cg_max = 1 << 30;
    a.ctl.eta1 = 0.1;
    a.ctl.eta2 = 1e-3;
    a.ctl.mu = 1e-4;
    // CG form: the pipelined one (one barrier per iteration) where barrier
    // latency bounds the solve; the textbook one on large systems, where the
    // passes stream HBM and the pipelined form's extra vector streams cost
    // more than its saved barriers (measured: 40^3 transient 71.6 -> 64.4 ms,
    // 50^2 steady 4.5 -> 4.0 ms; 150^3 steady 4.12 -> 4.31 s)
    // NNQP_FORCE_LARGE=1 runs a system of any size the way the largest ones
    // run (streamed operator, textbook CG, the full co-resident grid of
    // 256-thread blocks): it lets the tests check that path against the
    // oracle at sizes the oracle solves in seconds
    const char *fl = getenv("NNQP_FORCE_LARGE");
    const bool force_large = o->solver == NN_SOLVER_GPCG && fl && fl[0] == '1';
    a.ctl.cg_variant = n < (1 << 20) && !force_large ? 2 : 0;
    if (fmt == NN_FMT_CSR && a.ctl.cg_variant == 2) a.ctl.cg_variant = 1;   // CSR kernels: forms 0 and 1
    a.ctl.cg_bound_stop = 0;
    if (const char *e = getenv("NNQP_CG_VARIANT")) a.ctl.cg_variant = atoi(e);
    if (const char *e = getenv("NNQP_CG_BOUND_STOP")) a.ctl.cg_bound_stop = atoi(e);
    if (ssor) {
        // the textbook CG form with the SSOR sweeps in place of D^-1
        a.pc = s->ssor;
        a.pc.omega = o->ssor_omega;
        if (o->solver == NN_SOLVER_GPCG) a.ctl.cg_variant = 3;
    }
    // the search direction stays in L2 for the product that gathers it
    // (measured on the 150^3 solve: FP64 182.9 -> 176.7 us per product,
    // mixed 107.9 -> 106.5 us; no effect where the vectors fit L2 anyway)
    a.ctl.keep_p = 1;
    if (const char *e = getenv("NNQP_KEEP_P")) a.ctl.keep_p = atoi(e);
    if (const char *e = getenv("NNQP_GP_MAX")) a.ctl.gp_max = atoi(e);
    if (const char *e = getenv("NNQP_ETA1")) a.ctl.eta1 = atof(e);
    if (const char *e = getenv("NNQP_ETA2")) a.ctl.eta2 = atof(e);
    a.rtol = o->rtol;
    a.den_fallback = den_fallback(s);
    a.b0norm = s->b0norm;
    a.inner_rtol = o->inner_rtol;
    a.inner_cap = inner_product_cap(n);
    if (const char *e = getenv("NNQP_INNER_CAP")) a.inner_cap = std::max<int64_t>(1, atoll(e));
    a.max_ref = 200;
    a.timeout_ns = (unsigned long long)(o->wait_timeout_s * 1e9);
    // grid
    const bool lbfgs = o->solver == NN_SOLVER_LBFGS;
    const bool tron = o->solver == NN_SOLVER_TRON;
    if ((lbfgs || tron) && (mixed || fmt == NN_FMT_CSR)) {
        set_error("the projected L-BFGS and TRON solvers run in FP64 on the SELL format");
        return NN_ERR_INVALID_ARG;
    }
    a.ksp_rtol = o->ksp_rtol;
    if (lbfgs) {
        a.m = std::min(o->lbfgs_m, kLbMaxM);
        a.h0 = 1.0 / s->anorm_inf;
        NN_TRY(SA.alloc(&a.S, (size_t)(a.m + 1) * n, st));
        NN_TRY(SA.alloc(&a.Y, (size_t)(a.m + 1) * n, st));
    }
    a.predict = o->extrapolate;
    if (mode_transient(mode) && a.predict) NN_TRY(SA.alloc(&a.xprev, n, st));
    if (mode_transient(mode) && a.predict == 2) NN_TRY(SA.alloc(&a.xprev2, n, st));
    // Grid: one slice per warp at least.  Systems that a grid of one block
    // per SM covers in a few slices per warp run one block per SM (fewer
    // barrier arrivals) of 512 threads (one slice per warp: all loads of a
    // pass in flight at once); larger systems run the full co-resident grid
    // of 256-thread blocks (more loads in flight per SM).
    const int sms = device_sms();
    const int64_t slices = s->A64.nslices;
    int tpb = kSolveThreads;
    const bool driver = lbfgs || tron;   // solvers with a kernel of their own
    // Large systems (more than 32 slices per SM) run one 768-thread block
    // per SM with the textbook CG form: the warps of three 256-thread blocks,
    // a third of the barrier arrivals and reduction partials.  (Served
    // requests of that size take the whole device, so they may too.)  Mixed
    // solves of that size take the 768-thread kernel with the streamed FP32
    // operator (the only one built at that size; below, the 512-thread
    // load-based kernel where the streamed operator does not apply).
    const bool large = !driver && (slices > (int64_t)4 * 8 * sms || force_large);
    if (!driver && slices <= (int64_t)4 * 8 * sms && slices > (int64_t)8 * sms / 2) tpb = 512;
    if (!driver && (force_tpb == 256 || force_tpb == 512)) tpb = force_tpb;
    if (large && (a.ctl.cg_variant == 0 || a.ctl.cg_variant == 3) && fmt == NN_FMT_SELL && force_tpb != 512)
        tpb = kLargeThreads;
    if (force_large) {
        a.A.stream = true;
        a.A32.stream = true;
    }
    if (const char *e = getenv("NNQP_GRID_THREADS")) tpb = atoi(e);
    GridKernel kern = lbfgs ? k_lbfgs_grid : tron ? k_tron_grid : grid_kernel(mode, fmt, a.ctl.cg_variant, tpb);
    // a launch shape built only with the streamed FP32 operator: that kernel
    // stands in for the sizing below and must be taken by the streaming
    // choice further down (checked there)
    bool tma_only = false;
    if (!kern && !driver && mixed && fmt == NN_FMT_SELL && a.ctl.cg_variant == 0) {
        kern = grid_kernel(mode, FMT_SELL_TMA, 0, tpb);
        tma_only = kern != nullptr;
    }
    if (!kern && !driver && tpb != kSolveThreads) {
        tpb = kSolveThreads;
        kern = grid_kernel(mode, fmt, a.ctl.cg_variant, tpb);
    }
    if (lbfgs) tpb = kLbfgsThreads;
    if (tron) tpb = kSolveThreads;
    if (!kern) {
        set_error("CG variant %d is not available for this mode and format", a.ctl.cg_variant);
        return NN_ERR_INVALID_ARG;
    }
    int maxg = max_coresident(kern, tpb);
    const int warps = tpb / 32;
    const int64_t by_rows = (slices + warps - 1) / warps;
    // at least 4 slices' rows per block spread over the SMs: a mid-size solve
    // runs one block on every SM (its FP64 passes use every SM's FP64 pipe)
    // rather than filling fewer blocks' warps (measured: 40^3 transient on
    // 131 -> 152 blocks 55.8 -> 52.3 ms; 50^2 steady on 10 -> 19 blocks
    // 3.72 -> 3.36 ms)
    const int64_t spread = std::max<int64_t>(by_rows, (slices + 3) / 4);
    int want = (int)std::min<int64_t>(spread, slices <= (int64_t)4 * 8 * sms ? (int64_t)sms : (int64_t)maxg);
    want = std::min(want, maxg);
    if (large) want = maxg;
    if (o->grid_blocks > 0) want = std::min(o->grid_blocks, maxg);
    want = std::max(want, 1);
    // Mid-size SELL solves keep each block's slices of the operator of the
    // inner products in shared memory when they fit (one block per SM).
    size_t dyn_smem = 0;
    const char *sm_env = getenv("NNQP_SMEM_OP");
    if (!driver && fmt == NN_FMT_SELL && tpb == 512 && !(sm_env && sm_env[0] == '0')) {
        if (s->sptr_host.empty()) {
            s->sptr_host.resize((size_t)slices + 1);
            NN_CUDA_TRY(cudaMemcpyAsync(s->sptr_host.data(), s->A64.sptr, sizeof(int64_t) * (slices + 1),
                                        cudaMemcpyDeviceToHost, st));
            NN_CUDA_TRY(cudaStreamSynchronize(st));
        }
        const int vbytes = mixed ? 4 : 8;
        int64_t most = 0;
        for (int b = 0; b < want; ++b) {
            const Rows rb = rows_of_block(n, slices, b, want);
            most = std::max(most, s->sptr_host[(size_t)rb.s1] - s->sptr_host[(size_t)rb.s0]);
        }
        const size_t bytes = (size_t)most * (4 + vbytes);
        GridKernel ks = grid_kernel(mode, FMT_SELL_SMEM, a.ctl.cg_variant, tpb);
        // the attribute is set to the same budget by every caller (solves on
        // other host threads may launch this kernel at the same time)
        if (ks && bytes > 0 && bytes <= kSmemOperatorBytes &&
            cudaFuncSetAttribute((const void *)ks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemOperatorBytes) == cudaSuccess) {
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ks, tpb, bytes);
            if (per * sms >= want) {
                kern = ks;
                dyn_smem = bytes;
                maxg = per * sms;
            }
        }
        cudaGetLastError();   // a refused attribute leaves the plain kernel in use
    }
    // Large mixed solves stream the FP32 operator of their inner products
    // through shared memory with bulk asynchronous copies (FMT 3), when the
    // slots of the block's 24 warps fit the budget.  NNQP_TMA_OP=0 keeps the
    // load-based operator.
    const char *tma_env = getenv("NNQP_TMA_OP");
    if (!driver && fmt == NN_FMT_SELL && mixed && tpb == kLargeThreads && a.ctl.cg_variant == 0 && a.A32.stream &&
        dyn_smem == 0 && !(tma_env && tma_env[0] == '0')) {
        if (s->sptr_host.empty()) {
            s->sptr_host.resize((size_t)slices + 1);
            NN_CUDA_TRY(cudaMemcpyAsync(s->sptr_host.data(), s->A64.sptr, sizeof(int64_t) * (slices + 1),
                                        cudaMemcpyDeviceToHost, st));
            NN_CUDA_TRY(cudaStreamSynchronize(st));
        }
        int64_t wmax = 0;
        for (int64_t k = 0; k < slices; ++k)
            wmax = std::max<int64_t>(wmax, (s->sptr_host[(size_t)k + 1] - s->sptr_host[(size_t)k]) >> 5);
        const int se = (int)(32 * std::max<int64_t>(wmax, 2));
        const size_t budget = kTmaSmemBytes;
        // as many slots per warp as the budget holds (2 .. 4): D - 1 slices
        // of every warp in flight
        int slots = SellF32DiffTma::kMaxSlots;
        while (slots > 2 && SellF32DiffTma::smem_bytes(tpb / 32, slots, se) > budget) --slots;
        if (const char *e = getenv("NNQP_TMA_SLOTS")) slots = std::min(std::max(atoi(e), 2), SellF32DiffTma::kMaxSlots);
        const size_t bytes = SellF32DiffTma::smem_bytes(tpb / 32, slots, se);
        GridKernel kt = grid_kernel(mode, FMT_SELL_TMA, 0, tpb);
        if (kt && bytes <= budget &&
            cudaFuncSetAttribute((const void *)kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget) ==
                cudaSuccess) {
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kt, tpb, bytes);
            if (per >= 1) {
                const bool full_grid = want >= maxg;
                kern = kt;
                dyn_smem = bytes;
                maxg = per * sms;
                want = full_grid ? maxg : std::min(want, maxg);
                a.tma_slot_entries = se;
                a.tma_slots = slots;
            }
        }
        cudaGetLastError();   // a refused attribute leaves the load-based kernel in use
    }
    if (tma_only && dyn_smem == 0) {
        // the streamed operator does not apply: the load-based kernel with
        // 512-thread blocks, one per SM
        tpb = kLargeThreadsLoads;
        kern = grid_kernel(mode, fmt, a.ctl.cg_variant, tpb);
        if (!kern) {
            set_error("no solve kernel for this mode at %d threads per block", tpb);
            return NN_ERR_INVALID_ARG;
        }
        maxg = max_coresident(kern, tpb);
        want = large ? maxg : std::min(want, maxg);
    }
    // NNQP_TEST_STALL_BARRIER=1 makes the grid barrier wait for one block
    // that does not exist, so every wait runs into its time limit: the test of
    // the bounded-wait path (no fault, the kernel returns TIMEOUT).
    const char *stall = getenv("NNQP_TEST_STALL_BARRIER");
    a.bar_extra = (stall && stall[0] == '1') ? 1 : 0;
    NN_TRY(SA.alloc(&a.bar, 1, st));
    NN_TRY(SA.alloc(&a.partials, (size_t)2 * kMaxRed * (want + a.bar_extra), st));
    NN_TRY(SA.alloc(&a.counters, (size_t)nsteps * kCounters, st));
    NN_TRY(SA.alloc(&a.scalars, (size_t)nsteps * kScalars, st));
    P.kern = kern;
    P.want = want;
    P.tpb = tpb;
    P.dyn_smem = dyn_smem;
    return NN_OK;
}

// Enqueues one launch of plan P on stream st: resets the barrier and the
// counters, runs the persistent kernel, writes the Dirichlet entries of the
// outputs.  No host synchronisation (capturable in a CUDA graph).
nn_status plan_enqueue(GridPlan &P, const double *c_in, double *c_out, double *c_hist, cudaStream_t st) {
    GridArgs &a = P.a;
    const int64_t N = P.s->N;
    a.c_in = c_in;
    a.c_out = c_out;
    a.c_hist = c_hist;
    NN_CUDA_TRY(cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), st));
    NN_CUDA_TRY(cudaMemsetAsync(a.counters, 0, sizeof(int64_t) * P.nsteps * kCounters, st));
    void *args[] = {&a};
    cudaError_t le = cudaLaunchCooperativeKernel((void *)P.kern, dim3(P.want), dim3(P.tpb), args, P.dyn_smem, st);
    count_launch();
    if (le != cudaSuccess) {
        set_error("cooperative launch of %d blocks failed: %s", P.want, cudaGetErrorString(le));
        return NN_ERR_CUDA;
    }
    (k_fill_dirichlet<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, P.s->dmask, P.s->dval, c_out, 1, 0),
     ::nnqp::count_launch());
    if (c_hist)
        (k_fill_dirichlet<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, P.s->dmask, P.s->dval, c_hist,
                                                                       P.nsteps, N),
         ::nnqp::count_launch());
    return NN_OK;
}

// Reads the records of the last launch of plan P (synchronises stream st).
nn_status plan_collect(GridPlan &P, cudaStream_t st, float ms, nn_solve_info *infos, int ninfos) {
    GridArgs &a = P.a;
    const int nsteps = P.nsteps;
    std::vector<int64_t> cnt((size_t)nsteps * kCounters);
    std::vector<double> sc((size_t)nsteps * kScalars);
    GridBarrier hb;
    NN_CUDA_TRY(cudaMemcpyAsync(cnt.data(), a.counters, sizeof(int64_t) * cnt.size(), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaMemcpyAsync(sc.data(), a.scalars, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaMemcpyAsync(&hb, a.bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb.error) {
        set_error("a device-side wait gave up after %.3g s (wait #%d)", P.o.wait_timeout_s, hb.where);
        return (nn_status)hb.error;
    }
    nn_status worst = NN_OK;
    for (int k = 0; k < nsteps; ++k) {
        nn_solve_info inf;
        fill_info(P.s, &cnt[(size_t)k * kCounters], &sc[(size_t)k * kScalars], mode_mixed(P.mode), P.o.precond,
                  &inf);
        if (k == 0) inf.time_ms = ms;
        if (infos && k < ninfos) infos[k] = inf;
        if (inf.status != NN_OK && worst == NN_OK) worst = (nn_status)inf.status;
    }
    if (worst == NN_ERR_NOT_CONVERGED) set_error("iteration cap reached before the KKT tolerance");
    else if (worst == NN_ERR_NUMERIC) set_error("NaN/Inf met in a reduction");
    return worst;
}

// Runs the persistent solve kernel once: plan, launch, records, release.
// c_in/c_out/c_hist are device arrays.
// force_tpb: as for plan_build; plan_bytes (optional) receives the plan's
// scratch bytes.
nn_status run_grid(nn_system *s, const nn_solve_opts *o, int mode, int nsteps, const double *c_in, double *c_out,
                   double *c_hist, cudaStream_t st, nn_solve_info *infos, int ninfos, int force_tpb = 0,
                   size_t *plan_bytes = nullptr) {
    GridPlan P;
    struct Release {
        GridPlan &p;
        cudaStream_t st;
        ~Release() { p.arena.release(st); }
    } rel{P, st};
    NN_TRY(plan_build(s, o, mode, nsteps, st, P, force_tpb));
    if (plan_bytes) *plan_bytes = P.arena.bytes;
    cudaEvent_t e0, e1;
    NN_CUDA_TRY(cudaEventCreate(&e0));
    NN_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    nn_status r = plan_enqueue(P, c_in, c_out, c_hist, st);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    if (r == NN_OK) {
        NN_CUDA_TRY(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != NN_OK) return r;
    return plan_collect(P, st, ms, infos, ninfos);
}

nn_status kkt_impl(const nn_system *s, const double *c, const double *c_prev, int memory, double out[4],
                   cudaStream_t st) {
    if (s->dt > 0.0 && !c_prev) {
        set_error("nn_kkt_residual: a transient system needs c_prev");
        return NN_ERR_INVALID_ARG;
    }
    Scratch S;
    S.st = st;
    const int64_t n = s->NF, N = s->N;
    double *cfull, *pfull = nullptr, *x, *xp = nullptr, *part;
    const int nb = (int)std::min<int64_t>(std::max<int64_t>((s->A64.nslices + 7) / 8, 1), 4096);
    NN_TRY(S.a.alloc(&x, n, st));
    NN_TRY(S.a.alloc(&part, (size_t)nb * 6, st));
    cudaMemcpyKind kind = memory == NN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    NN_TRY(S.a.alloc(&cfull, N, st));
    NN_CUDA_TRY(cudaMemcpyAsync(cfull, c, sizeof(double) * N, kind, st));
    (k_gather_free<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, s->free_node, cfull, x), ::nnqp::count_launch());
    if (s->dt > 0.0) {
        NN_TRY(S.a.alloc(&pfull, N, st));
        NN_TRY(S.a.alloc(&xp, n, st));
        NN_CUDA_TRY(cudaMemcpyAsync(pfull, c_prev, sizeof(double) * N, kind, st));
        (k_gather_free<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, s->free_node, pfull, xp), ::nnqp::count_launch());
    }
    SellF64 M = s->dt > 0.0 ? viewM(s) : view64(s);
    (k_kkt<<<nb, 256, 0, st>>>(view64(s), M, s->dt > 0.0, s->dt > 0.0 ? 1.0 / s->dt : 0.0, s->b0, x, xp, s->lo,
                              s->hi, part), ::nnqp::count_launch());
    std::vector<double> hp((size_t)nb * 6);
    NN_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b) {
        t[0] += hp[b * 6 + 0];
        t[1] = std::max(t[1], hp[b * 6 + 1]);
        t[2] += hp[b * 6 + 2];
        t[3] = std::max(t[3], hp[b * 6 + 3]);
        t[4] += hp[b * 6 + 4];
        t[5] += hp[b * 6 + 5];
    }
    double d2 = std::sqrt(t[2]), di = t[3];
    if (t[2] == 0.0) d2 = di = den_fallback(s);
    out[0] = std::sqrt(t[0]) / d2;
    out[1] = t[1] / di;
    out[2] = t[5] == 0.0 ? 1.0 : 0.0;
    out[3] = 0.5 * t[4];
    return NN_OK;
}

nn_status spmv_impl(const nn_system *s, const double *x, double *y, int format, int precision, cudaStream_t st) {
    const int nb = (int)std::max<int64_t>((s->A64.nslices + 7) / 8, 1);
    if ((format != NN_FMT_SELL && format != NN_FMT_CSR) || (precision != NN_PREC_FP64 && precision != NN_PREC_MIXED)) {
        set_error("nn_spmv: format must be NN_FMT_SELL or NN_FMT_CSR, precision NN_PREC_FP64 or NN_PREC_MIXED");
        return NN_ERR_INVALID_ARG;
    }
    if (precision == NN_PREC_MIXED && format != NN_FMT_SELL) {
        set_error("nn_spmv: the FP32-value operator is stored in SELL format only");
        return NN_ERR_INVALID_ARG;
    }
    if (precision == NN_PREC_MIXED && !s->has_mixed) {
        set_error("nn_spmv: system has no FP32 copy (build_mixed = 0)");
        return NN_ERR_INVALID_ARG;
    }
    // nn_assemble refuses systems without free unknowns; a zero-size grid
    // would be a launch error, so an empty product returns before any launch
    if (s->NF == 0) return NN_OK;
    if (precision == NN_PREC_MIXED) {
        Scratch S;
        S.st = st;
        float *x32;
        NN_TRY(S.a.alloc(&x32, s->NF, st));
        (k_to_f32<<<(unsigned)((s->NF + 255) / 256), 256, 0, st>>>(s->NF, x, x32), ::nnqp::count_launch());
        (k_spmv32<<<nb, 256, 0, st>>>(view32(s), x32, y), ::nnqp::count_launch());
        NN_CUDA_TRY(cudaGetLastError());
        return NN_OK;
    }
    if (format == NN_FMT_CSR) (k_spmvcsr<<<nb, 256, 0, st>>>(viewcsr(s), x, y), ::nnqp::count_launch());
    else (k_spmv64<<<nb, 256, 0, st>>>(view64(s), x, y), ::nnqp::count_launch());
    NN_CUDA_TRY(cudaGetLastError());
    return NN_OK;
}

// y = A_local x_ext for one shard of a row-sharded system: CSR rows with
// local column ids (device arrays; x_ext holds the owned entries followed by
// the ghosts).
nn_status csr_spmv_impl(int64_t nrows, const int64_t *rowptr, const int32_t *col, const double *val,
                        const double *x, double *y, cudaStream_t st) {
    if (nrows == 0) return NN_OK;
    const int64_t slices = (nrows + 31) / 32;
    const int nb = (int)std::max<int64_t>((slices + 7) / 8, 1);
    (k_spmvcsr<<<nb, 256, 0, st>>>(CsrF64{nrows, slices, rowptr, col, val}, x, y), count_launch());
    NN_CUDA_TRY(cudaGetLastError());
    return NN_OK;
}

// ------------------------------------------------------------------ no-allocation product
//
// nn_spmv_mixed_noalloc computes the same FP32-value product as nn_spmv with
// NN_PREC_MIXED, but keeps the FP32 copy of x in the file-scope array below
// instead of allocating it per call.  Maximum: kNoAllocMaxFree unknowns
// (16 MiB of FP32).  The array exists on every device that loads this
// library, for the life of the process; all calls share it, so calls that
// overlap on the GPU race on it.  Nothing in it has to start at zero: every
// call overwrites the first NF entries before reading them.

constexpr int64_t kNoAllocMaxFree = 1LL << 22;
static __device__ __align__(256) float g_noalloc_x32[kNoAllocMaxFree];

namespace {
std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
float *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device, looked up once
// per device with that device current (host code may not use the symbol itself).
static nn_status noalloc_scratch(float **out) {
    int dev = 0;
    NN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("nn_spmv_mixed_noalloc: device %d is beyond the supported %d devices", dev, kNoAllocMaxDevices);
        return NN_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_x32);
        if (e != cudaSuccess || !p) {
            set_error("nn_spmv_mixed_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return NN_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = (float *)p;
    }
    *out = g_noalloc_ptr[dev];
    return NN_OK;
}

nn_status spmv_mixed_noalloc_impl(const nn_system *s, const double *x, double *y, cudaStream_t st) {
    if (!s->has_mixed) {
        set_error("nn_spmv_mixed_noalloc: system has no FP32 copy (build_mixed = 0)");
        return NN_ERR_INVALID_ARG;
    }
    if (s->NF > kNoAllocMaxFree) {
        set_error("nn_spmv_mixed_noalloc: %lld unknowns exceed the static scratch limit of %lld",
                  (long long)s->NF, (long long)kNoAllocMaxFree);
        return NN_ERR_INVALID_ARG;
    }
    if (s->NF == 0) return NN_OK;   // as in spmv_impl: no launch for an empty product
    float *x32 = nullptr;
    NN_TRY(noalloc_scratch(&x32));
    const int nb = (int)std::max<int64_t>((s->A64.nslices + 7) / 8, 1);
    (k_to_f32<<<(unsigned)((s->NF + 255) / 256), 256, 0, st>>>(s->NF, x, x32), count_launch());
    (k_spmv32<<<nb, 256, 0, st>>>(view32(s), x32, y), count_launch());
    NN_CUDA_TRY(cudaGetLastError());
    return NN_OK;
}

// Host or device full vectors in and out of run_grid.
nn_status solve_entry(nn_system *s, const nn_solve_opts *o, int mode, int nsteps, const double *c_in,
                      double *c_out, double *c_hist, int memory, cudaStream_t st, nn_solve_info *infos,
                      int ninfos) {
    if (memory == NN_MEM_DEVICE) return run_grid(s, o, mode, nsteps, c_in, c_out, c_hist, st, infos, ninfos);
    Scratch S;
    S.st = st;
    double *din, *dout, *dhist = nullptr;
    NN_TRY(S.a.alloc(&din, s->N, st));
    NN_TRY(S.a.alloc(&dout, s->N, st));
    if (c_hist) NN_TRY(S.a.alloc(&dhist, (size_t)s->N * nsteps, st));
    NN_CUDA_TRY(cudaMemcpyAsync(din, c_in, sizeof(double) * s->N, cudaMemcpyHostToDevice, st));
    nn_status r = run_grid(s, o, mode, nsteps, din, dout, dhist, st, infos, ninfos);
    if (r == NN_OK || r == NN_ERR_NOT_CONVERGED || r == NN_ERR_NUMERIC) {
        NN_CUDA_TRY(cudaMemcpyAsync(c_out, dout, sizeof(double) * s->N, cudaMemcpyDeviceToHost, st));
        if (c_hist)
            NN_CUDA_TRY(cudaMemcpyAsync(c_hist, dhist, sizeof(double) * s->N * nsteps, cudaMemcpyDeviceToHost, st));
        NN_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return r;
}

// NN_PREC_AUTO: mixed precision where the FP32 operator streams from HBM.
bool auto_mixed(const nn_system *s) { return s->has_mixed && (double)s->nnzF * 8.0 > kStreamBytes; }

int mode_for(const nn_system *s, const nn_solve_opts *o) {
    const bool mixed = o->precision == NN_PREC_MIXED ||
                       (o->precision == NN_PREC_AUTO && o->precond != NN_PC_SSOR && auto_mixed(s));
    if (s->dt > 0.0) return mixed ? MODE_MIXED_TR : MODE_TRANSIENT;
    return mixed ? MODE_MIXED : MODE_STEADY;
}

// Co-resident 256-thread blocks per SM of the steady/mixed solve kernels
// (the smallest over modes and CG forms) and the SM count of the current
// device.
int solve_grid_blocks_per_sm(int *sms) {
    int c = 1 << 30;
    for (int mode : {MODE_STEADY, MODE_MIXED})
        for (int v = 0; v < 3; ++v)
            if (GridKernel k = grid_kernel(mode, NN_FMT_SELL, v)) c = std::min(c, max_coresident(k) / device_sms());
    if (sms) *sms = device_sms();
    return c;
}

// One steady solve with the launch shape fixed at admission (serving):
// tpb threads per block, at most grid_blocks blocks.  plan_bytes receives
// the solve's scratch bytes.
nn_status serve_solve(nn_system *s, const nn_solve_opts *o, const double *c_in_dev, double *c_out_dev,
                      cudaStream_t st, int tpb, int grid_blocks, nn_solve_info *info, size_t *plan_bytes) {
    nn_solve_opts q = *o;
    q.grid_blocks = grid_blocks;
    return run_grid(s, &q, mode_for(s, &q), 1, c_in_dev, c_out_dev, nullptr, st, info, info ? 1 : 0, tpb,
                    plan_bytes);
}

}  // namespace nnqp

// ---------------------------------------------------------------- reusable solve plans

namespace nnqp {
nn_status check_opts(const nn_solve_opts *o);
}

struct nn_plan {
    nnqp::GridPlan p;
    cudaStream_t st = nullptr;   // stream the scratch was allocated on
};

extern "C" {

nn_status nn_plan_create(nn_system *s, const nn_solve_opts *o, int nsteps, void *stream, nn_plan **out) {
    using namespace nnqp;
    clear_error();
    if (!s || !out) {
        set_error("nn_plan_create: NULL system or output");
        return NN_ERR_INVALID_ARG;
    }
    *out = nullptr;
    nn_solve_opts d;
    nn_solve_opts_default(&d);
    if (!o) o = &d;
    NN_TRY(check_opts(o));
    const int mode = mode_for(s, o);
    if (nsteps < 1 || (!mode_transient(mode) && nsteps != 1)) {
        set_error("nn_plan_create: nsteps must be 1 for a steady system, >= 1 for a transient one");
        return NN_ERR_INVALID_ARG;
    }
    nn_plan *pl = new (std::nothrow) nn_plan;
    if (!pl) {
        set_error("nn_plan_create: out of host memory");
        return NN_ERR_OOM;
    }
    pl->st = (cudaStream_t)stream;
    nn_status r = plan_build(s, o, mode, nsteps, pl->st, pl->p);
    if (r != NN_OK) {
        pl->p.arena.release(pl->st);
        cudaStreamSynchronize(pl->st);
        delete pl;
        return r;
    }
    *out = pl;
    return NN_OK;
}

nn_status nn_plan_launch(nn_plan *pl, const double *c_in, double *c_out, double *c_hist, void *stream) {
    using namespace nnqp;
    clear_error();
    if (!pl || !c_in || !c_out) {
        set_error("nn_plan_launch: NULL plan or vector");
        return NN_ERR_INVALID_ARG;
    }
    return plan_enqueue(pl->p, c_in, c_out, c_hist, (cudaStream_t)stream);
}

nn_status nn_plan_result(nn_plan *pl, void *stream, nn_solve_info *infos, int ninfos) {
    using namespace nnqp;
    clear_error();
    if (!pl) {
        set_error("nn_plan_result: NULL plan");
        return NN_ERR_INVALID_ARG;
    }
    nn_status r = plan_collect(pl->p, (cudaStream_t)stream, 0.0f, infos, ninfos);
    for (int k = 0; infos && k < ninfos && k < pl->p.nsteps; ++k) infos[k].time_ms = NAN;
    return r;
}

void nn_plan_destroy(nn_plan *pl) {
    if (!pl) return;
    pl->p.arena.release(pl->st);
    cudaStreamSynchronize(pl->st);
    delete pl;
}

}  // extern "C"
