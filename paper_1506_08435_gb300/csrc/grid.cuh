// The persistent solve kernel of one system: one cooperative launch runs a
// whole QP solve (steady), a whole backward-Euler run (transient: one
// warm-started QP per step, Sec. 2.2.2 and Algorithm 1), or a mixed-precision
// refinement loop (steady or per step), with no host round trip between
// iterations.  The kernel is a template over (format, mode, CG variant); each
// mode's instantiations are compiled in a translation unit of their own
// (solve_grid_*.cu), which also returns them by (format, variant).
#pragma once
#include <stdint.h>
#include "internal.h"
#include "gpcg.cuh"
#include "refine.cuh"

namespace nnqp {

constexpr int kSolveThreads = 256;
constexpr int kCounters = 14;   // per-step int64 counters written by the kernel
constexpr int kScalars = 4;     // per-step double results

enum { MODE_STEADY = 0, MODE_TRANSIENT = 1, MODE_MIXED = 2, MODE_MIXED_TR = 3 };
__host__ __device__ constexpr bool mode_transient(int m) { return m == MODE_TRANSIENT || m == MODE_MIXED_TR; }
__host__ __device__ constexpr bool mode_mixed(int m) { return m == MODE_MIXED || m == MODE_MIXED_TR; }
// Blocks per SM the kernel is compiled for: the transient drivers run one
// block per SM on mid-size systems and get the larger register budget.
__host__ __device__ constexpr int mode_min_blocks(int m) { return mode_transient(m) ? 2 : 3; }
// CG form of the FP32 inner solves of a mixed mode whose FP64 form is cgv:
// steady solves from zero do not take the pipelined form (its recurrences
// drift in FP32 over thousands of iterations: the inner solves of 1e5 - 1e6
// unknown steady problems stalled at ~10x the FP64 product count) but the
// Chronopoulos-Gear form, with the same single fused reduction; the short,
// warm-started inner solves of backward-Euler steps keep the pipelined one.
__host__ __device__ constexpr int inner_cg_form(int mode, int cgv) {
    return (mode == MODE_MIXED && cgv == 2) ? 1 : cgv;
}

struct GridArgs {
    int mode;
    int64_t n, N, nslices;
    SellF64 A;
    CsrF64 Acsr;
    SellF32Diff A32;
    SellF64 M;
    double lo, hi, inv_dt;
    const double *b0;
    const double *dinv64;
    const float *dinv32;
    const int32_t *free_node;
    const double *c_in;     // full node vector (warm start)
    double *c_out;          // full node vector (result), free entries written
    double *c_hist;         // [nsteps][N] or null
    int nsteps;
    double *v64[11];        // x g p q r z s w gw b m2
    float *v32[13];         // d g p q r z s w gw r32 l32 h32 m2
    GpcgCtl ctl;
    double rtol, den_fallback, b0norm, inner_rtol;
    int64_t inner_cap;      // mixed: products allowed to one FP32 inner solve
    int max_ref;
    GridBarrier *bar;
    double *partials;
    unsigned long long timeout_ns;
    int bar_extra;          // arrivals the barrier waits for beyond the grid (0; 1 only in the stall test)
    int64_t *counters;      // [nsteps][kCounters]
    double *scalars;        // [nsteps][kScalars]
    // projected L-BFGS
    double *S, *Y;          // (m+1) slots of n doubles each
    int m;
    double h0;
    // TRON: relative tolerance of each subspace CG
    double ksp_rtol;
    // transient: initial iterate of step n+1 (option extrapolate): 1 = the box
    // projection of the linear extrapolation 2 c^(n) - c^(n-1), 2 = of the
    // quadratic one 3 c^(n) - 3 c^(n-1) + c^(n-2); 0 = c^(n)
    int predict;
    double *xprev;          // [n] c^(n-1) at the free nodes
    double *xprev2;         // [n] c^(n-2) (quadratic extrapolation)
    uint8_t *fmask;         // [n] face mask of the CG phases
    int tma_slot_entries;   // FMT 3: 32 x the widest slice (slot size of the streamed operator)
    int tma_slots;          // FMT 3: slots per warp
    SsorF64 pc;             // SSOR ordering and omega (CG form 3, TRON with ncolors > 0)
};

// Initial iterate of a backward-Euler step: linear extrapolation of the last
// two states, projected onto the box (the QP itself is unchanged; only the
// starting point of its iteration moves).
template <class Team>
__device__ void transient_predict(const Rows &R, const GridArgs &a, double *x, int step) {
    if (!a.predict) return;
    R.each([&](int64_t i) {
        const double xn = x[i];
        const double x1 = a.xprev[i];
        if (a.predict == 2 && step > 1) {
            x[i] = clampv(3.0 * (xn - x1) + a.xprev2[i], a.lo, a.hi);
        } else if (step > 0) {
            x[i] = clampv(xn + (xn - x1), a.lo, a.hi);
        }
        if (a.predict == 2) a.xprev2[i] = x1;
        a.xprev[i] = xn;
    });
}

// b of one backward-Euler step: b0 + M x / dt (Sec. 2.2.2, with c^(n));
// returns ||b||_2 through den.
template <class Team>
__device__ bool transient_rhs(Team &T, const Rows &R, const GridArgs &a, const double *x, double *&b, double &den) {
    double *bt = a.v64[9];
    double acc[1] = {0.0};
    a.M.apply(R, x, [&](int64_t i, double mx) {
        const double bi = a.b0[i] + mx * a.inv_dt;
        bt[i] = bi;
        acc[0] += bi * bi;
    });
    if (!T.reduce(acc)) return false;
    den = sqrt(acc[0]);
    b = bt;
    return true;
}

// Scatter of the step result to the full-node outputs and the per-step record.
template <class Team>
__device__ bool step_outputs(Team &T, const Rows &R, const GridArgs &a, const double *x, int step, int nsteps,
                             int status, int64_t (&cnt)[kCounters], double gp2, double den) {
    double acc[2] = {0.0, 0.0};
    double *hist = a.c_hist ? a.c_hist + (int64_t)step * a.N : nullptr;
    R.each([&](int64_t i) {
        const double xi = x[i];
        const int32_t v = a.free_node[i];
        if (hist) hist[v] = xi;
        if (step == nsteps - 1) a.c_out[v] = xi;
        acc[0] += xi <= a.lo ? 1.0 : 0.0;
        acc[1] += xi >= a.hi ? 1.0 : 0.0;
    });
    if (!T.reduce(acc)) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cnt[0] = status;
        cnt[8] = (int64_t)acc[0];
        cnt[9] = (int64_t)acc[1];
        for (int k = 0; k < kCounters; ++k) a.counters[(int64_t)step * kCounters + k] = cnt[k];
        a.scalars[step * kScalars + 0] = gp2;
        a.scalars[step * kScalars + 1] = den;
    }
    return true;
}

// One instantiation per (format, mode) so that each kernel carries only the
// code of its own path (register allocation is per kernel).
// TPB threads per block: 256 (several blocks per SM), 512 (one block per SM
// on mid-size systems: one slice per warp, so the loads of a pass are all in
// flight at once) or 768 (one block of 24 warps per SM on large systems: the
// warps of three 256-thread blocks with a third of the barrier arrivals and
// reduction partials).
// FMT: 0 = SELL, 1 = CSR (FP64), 2 = SELL with the block's slices of the
// operator that the inner products use (FP64 A, or FP32 A in the mixed
// modes) held in shared memory for the whole launch: staged once, then every
// product reads its columns and values on chip and only gathers x from L2
// (mid-size systems, whose slices per block fit in shared memory);
// 3 (mixed modes) = the FP32 operator of the inner products streamed through
// shared memory by bulk asynchronous copies, D slices in flight per warp
// (operators far larger than L2).
template <int FMT, int MODE, int CGV, int TPB>
__global__ void __launch_bounds__(TPB, TPB >= 512 ? 1 : mode_min_blocks(MODE)) k_solve_grid(GridArgs a) {
    __shared__ RedSmem sm;
    extern __shared__ __align__(16) unsigned char op_smem[];
    GridTeam T{a.bar, a.partials, (int)gridDim.x + a.bar_extra, a.timeout_ns, 0, 0, &sm};
    const Rows R = rows_of_block(a.n, a.nslices, blockIdx.x, gridDim.x);
    double *x = a.v64[0];
    R.each([&](int64_t i) { x[i] = a.c_in[a.free_node[i]]; });
    SellF64Local Aloc{};
    SellF32DiffLocal A32loc{};
    SellF32DiffTma A32tma{};
    if constexpr (FMT == 3) {
        static_assert(mode_mixed(MODE), "the streamed FP32 operator serves the mixed modes");
        A32tma.n = a.A32.n;
        A32tma.nslices = a.A32.nslices;
        A32tma.sptr = a.A32.sptr;
        A32tma.col = a.A32.col;
        A32tma.val = a.A32.val;
        A32tma.rsum = a.A32.rsum;
        A32tma.slot_entries = a.tma_slot_entries;
        A32tma.D = a.tma_slots;
        A32tma.error = &a.bar->error;
        A32tma.setup(op_smem);
    }
    if constexpr (FMT == 2) {
        // stage entries [e0, e1) of this block's slices: columns, then values
        constexpr bool MIX = mode_mixed(MODE);
        const int64_t e0 = a.A.sptr[R.s0], e1 = a.A.sptr[R.s1];
        const int64_t ne = e1 - e0;   // a multiple of 64 (32-row slices, even widths)
        int32_t *scol = reinterpret_cast<int32_t *>(op_smem);
        unsigned char *sv = op_smem + ne * 4;
        const int4 *gc = reinterpret_cast<const int4 *>(a.A.col + e0);
        for (int64_t q = threadIdx.x; q < ne / 4; q += blockDim.x) reinterpret_cast<int4 *>(scol)[q] = __ldg(gc + q);
        const int vbytes = MIX ? 4 : 8;
        const int4 *gv = MIX ? reinterpret_cast<const int4 *>(a.A32.val + e0) : reinterpret_cast<const int4 *>(a.A.val + e0);
        for (int64_t q = threadIdx.x; q < ne * vbytes / 16; q += blockDim.x) reinterpret_cast<int4 *>(sv)[q] = __ldg(gv + q);
        if constexpr (MIX)
            A32loc = SellF32DiffLocal{a.A32.n, a.A32.nslices, a.A32.sptr, scol, reinterpret_cast<const float *>(sv),
                                      a.A32.rsum, false, e0};
        else
            Aloc = SellF64Local{a.A.n, a.A.nslices, a.A.sptr, scol, reinterpret_cast<const double *>(sv), a.A.diag,
                                false, e0};
    }
    if (!T.sync()) return;
    const int nsteps = mode_transient(MODE) ? a.nsteps : 1;
    for (int step = 0; step < nsteps; ++step) {
        int status = ST_OK;
        int64_t cnt[kCounters] = {0};
        double den = a.b0norm, gp2 = 0.0;
        double *b = const_cast<double *>(a.b0);
        if (mode_transient(MODE)) {
            if (!transient_rhs(T, R, a, x, b, den)) return;
            cnt[1] += 1;   // products with M (FP64)
            cnt[12] += 4;
            transient_predict<GridTeam>(R, a, x, step);   // own rows; the solve's first pass syncs
        }
        if (!(den > 0.0)) den = a.den_fallback;
        if constexpr (mode_mixed(MODE)) {
            GpcgVecs<float> v{a.v32[0], a.v32[1], a.v32[2], a.v32[3], a.v32[4], a.v32[5],
                              a.v32[6], a.v32[7], a.v32[8], a.v32[9], a.dinv32, a.fmask, a.v32[12]};
            GpcgVecs<double> v64{x, a.v64[1], a.v64[2], a.v64[3], a.v64[4], a.v64[5],
                                 a.v64[6], a.v64[7], a.v64[8], b, a.dinv64, a.fmask, a.v64[10]};
            MixedStats ms;
            if constexpr (FMT == 2)
                status = mixed_solve<CGV, inner_cg_form(MODE, CGV), true>(T, R, a.A, A32loc, a.lo, a.hi, b, x, v, a.v32[9], a.v32[10],
                                                 a.v32[11], v64, a.rtol * den, a.inner_rtol, a.max_ref,
                                                 a.ctl.max_spmv, a.inner_cap, a.ctl, a.ctl, ms);
            else if constexpr (FMT == 3)
                status = mixed_solve<CGV, inner_cg_form(MODE, CGV), (TPB < 512)>(T, R, a.A, A32tma, a.lo, a.hi, b, x, v, a.v32[9], a.v32[10],
                                                 a.v32[11], v64, a.rtol * den, a.inner_rtol, a.max_ref,
                                                 a.ctl.max_spmv, a.inner_cap, a.ctl, a.ctl, ms);
            else
                status = mixed_solve<CGV, inner_cg_form(MODE, CGV), true>(T, R, a.A, a.A32, a.lo, a.hi, b, x, v, a.v32[9], a.v32[10],
                                                 a.v32[11], v64, a.rtol * den, a.inner_rtol, a.max_ref,
                                                 a.ctl.max_spmv, a.inner_cap, a.ctl, a.ctl, ms);
            if (status == ST_TIMEOUT) return;
            cnt[1] += ms.spmv64;
            cnt[2] += ms.spmv32;
            cnt[3] = ms.cg;
            cnt[4] = ms.phases;
            cnt[5] = ms.refinements;
            cnt[6] = ms.vec64;
            cnt[7] = ms.vec32;
            cnt[11] = ms.fallback;
            cnt[12] += ms.fl64;
            cnt[13] += ms.fl32;
            gp2 = ms.gp2;
        } else {
            GpcgVecs<double> v{x, a.v64[1], a.v64[2], a.v64[3], a.v64[4], a.v64[5],
                               a.v64[6], a.v64[7], a.v64[8], b, a.dinv64, a.fmask, a.v64[10]};
            const SsorF64 pcv = a.pc;
            if constexpr (CGV == 3) v.pc = &pcv;
            GpcgCtl c = a.ctl;
            c.tol = a.rtol * den;
            c.face_tol = 0.5 * c.tol;
            GpcgStats gs;
            const Bounds<double> B{a.lo, a.hi, nullptr, nullptr};
            if constexpr (FMT == 0)
                status = gpcg_solve<GridTeam, SellF64, double, CGV>(T, R, a.A, B, v, c, gs);
            else if constexpr (FMT == 2)
                status = gpcg_solve<GridTeam, SellF64Local, double, CGV>(T, R, Aloc, B, v, c, gs);
            else
                status = gpcg_solve<GridTeam, CsrF64, double, CGV>(T, R, a.Acsr, B, v, c, gs);
            if (status == ST_TIMEOUT) return;
            x = v.x;
            // keep the solution in slot 0 so that the next step starts there
            if (x != a.v64[0]) {
                R.each([&](int64_t i) { a.v64[0][i] = x[i]; });
                x = a.v64[0];
                if (!T.sync()) return;
            }
            cnt[1] += gs.spmv;
            cnt[3] = gs.cg;
            cnt[4] = gs.phases;
            cnt[6] = gs.vec;
            cnt[10] = gs.pc;
            cnt[12] += gs.fl;
            gp2 = gs.gp2;
        }
        if (!step_outputs(T, R, a, x, step, nsteps, status, cnt, gp2, den)) return;
    }
}

using GridKernel = void (*)(GridArgs);

// Internal format codes: the shared-memory-resident SELL operator, and the
// FP32 SELL operator streamed through shared memory by bulk copies.
constexpr int FMT_SELL_SMEM = 2;
constexpr int FMT_SELL_TMA = 3;

// Kernel of one mode for format fmt (NN_FMT_SELL / NN_FMT_CSR /
// FMT_SELL_SMEM), CG variant cgv (0, 1, 2; 3 = textbook CG with the SSOR
// preconditioner, FP64 modes) and threads per block tpb (256, 512, 768);
// nullptr if that combination is not built.
GridKernel grid_kernel_steady(int fmt, int cgv, int tpb);
GridKernel grid_kernel_transient(int fmt, int cgv, int tpb);
GridKernel grid_kernel_mixed(int fmt, int cgv, int tpb);
GridKernel grid_kernel_mixed_transient(int fmt, int cgv, int tpb);
GridKernel grid_kernel_tma(int mode, int cgv, int tpb);

}  // namespace nnqp
