/*
 * nnqp.h -- C ABI of the GB300-native non-negative diffusion solver.
 *
 * Method: Chang, Karra & Nakshatrala, "An optimization-based framework for
 * ... non-negative ... anisotropic diffusion" (arXiv 1506.08435).
 *   - The Galerkin P1 discretisation of -div(D grad c) = f with Dirichlet
 *     data c^p on Gamma^D and zero-flux Neumann data elsewhere (Sec. 2.1,
 *     Sec. 2.1.2) gives K c = f with K symmetric positive definite.
 *   - The non-negative methodology replaces K c = f by the convex QP
 *       minimize 1/2 <c; K c> - <c; f>  subject to  lo <= c <= hi
 *     (Sec. 2.1.3 with lo = 0; Sec. 2.2.2 with c_min, c_max; Sec. 5 remark:
 *     the upper bound 1 is enforced as well).
 *   - Transient problems use backward Euler with the capacity matrix M:
 *       Kt = M/dt + K,  ft^(n+1) = f + M c^(n)/dt   (Sec. 2.2.2; the printed
 *     formula has c^(n+1) in ft, which is read as c^(n)),
 *     and the Jacobian (Kt) is assembled once (Sec. 3.2).
 *   - Dispersion tensor D = (a_T |v| + D_M) I + (a_L - a_T) v v^T / |v|
 *     from a cell-wise velocity (Sec. 5; Algorithm 1 takes the cell-wise
 *     velocity as input).
 *
 * Conventions for every entry point:
 *   - Return value: NN_OK or an nn_status error; nn_last_error() gives a
 *     thread-local message for the last failing call on this thread.
 *   - Streams are CUDA streams (cudaStream_t) passed as void*; NULL is the
 *     legacy default stream.  Calls are ordered on that stream; a call that
 *     returns results to host memory synchronizes that stream.
 *   - Memory flags (NN_MEM_HOST / NN_MEM_DEVICE) say where caller arrays
 *     live.  Caller arrays are borrowed for the duration of the call only;
 *     the library copies what it keeps.
 *   - Handles (nn_system, nn_server) are owned by the library and released
 *     with the matching *_destroy call.
 *   - Floating point is IEEE double unless stated; index arrays are int32
 *     (node and element ids < 2^31).
 *   - Invalid input is rejected on the host or by a device-side check that
 *     writes a status word; no entry point traps or asserts on the device.
 */
#ifndef NNQP_H
#define NNQP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NN_OK = 0,
    NN_ERR_INVALID_ARG = 1,    /* bad sizes, pointers, flags, connectivity */
    NN_ERR_INFEASIBLE = 2,     /* lo > hi, or a Dirichlet value outside [lo, hi] */
    NN_ERR_NOT_SPD = 3,        /* an element tensor D_e is not symmetric positive definite */
    NN_ERR_OOM = 4,            /* device allocation failed */
    NN_ERR_NOT_CONVERGED = 5,  /* iteration cap reached; best feasible iterate returned */
    NN_ERR_NUMERIC = 6,        /* NaN/Inf met in a reduction or in the input */
    NN_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
    NN_ERR_CUDA = 8,           /* a CUDA runtime call failed */
    NN_ERR_BUSY = 9,           /* serving: over budget and queue full / result not ready */
    NN_ERR_DEGENERATE = 10     /* an element has zero measure */
} nn_status;

enum { NN_MEM_HOST = 0, NN_MEM_DEVICE = 1 };
enum { NN_COEF_TENSOR = 0, NN_COEF_VELOCITY = 1 };
enum { NN_SOLVER_GPCG = 0, NN_SOLVER_LBFGS = 1, NN_SOLVER_TRON = 2 };
enum { NN_PREC_FP64 = 0, NN_PREC_MIXED = 1, NN_PREC_AUTO = 2 };
enum { NN_FMT_SELL = 0, NN_FMT_CSR = 1 };
enum { NN_PC_JACOBI = 0, NN_PC_SSOR = 1 };

/* Last error message of the calling thread ("" if none). */
const char *nn_last_error(void);
/* Library version string. */
const char *nn_version(void);
/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads); for accounting of device work, never reset. */
uint64_t nn_kernel_launches(void);
/* Number of device allocations this library has made in this process (all
 * devices, all threads: every buffer it takes from its stream-ordered memory
 * pool); for accounting, never reset. */
uint64_t nn_device_allocations(void);

/* ------------------------------------------------------------------ mesh */

/* Node and element counts of the structured P1 mesh of [0,1]^dim with
 * nx x ny (x nz) cells: 2D (nx+1)(ny+1) nodes, 2 nx ny triangles; 3D
 * (nx+1)(ny+1)(nz+1) nodes, 6 nx ny nz tetrahedra.  (The paper's P1
 * simplicial spaces, Sec. 2.1.3; the structured split is this library's
 * canonical mesh: its meshes are unstructured.)  Errors: INVALID_ARG. */
nn_status nn_mesh_counts(int dim, int nx, int ny, int nz, int64_t *n_nodes, int64_t *n_elems);

/* Writes the canonical structured mesh into caller DEVICE buffers
 * coords [n_nodes][dim] (FP64, node (i,j,k) at (i/nx, j/ny, k/nz), id
 * i + (nx+1)(j + (ny+1)k)) and conn [n_elems][dim+1] (int32):
 *   2D: square (i,j) -> T0 = (v00, v10, v11), T1 = (v00, v11, v01),
 *       element id 2(i + nx j) + t;
 *   3D: hexahedron h = i + nx(j + ny k) -> 6 Kuhn tetrahedra, one per axis
 *       permutation p in lexicographic order (xyz, xzy, yxz, yzx, zxy, zyx),
 *       vertices v0, v0+e_p0, v0+e_p0+e_p1, v0+e_p0+e_p1+e_p2, id 6h + p.
 * Stream-ordered, asynchronous.  Errors: INVALID_ARG, CUDA. */
nn_status nn_mesh_structured(int dim, int nx, int ny, int nz, double *coords, int32_t *conn, void *stream);

/* --------------------------------------------------------------- problem */

typedef struct {
    int dim;                        /* 2 or 3 */
    /* Mesh: either explicit arrays (coords != NULL) or the structured mesh
     * of nn_mesh_structured generated on the device (coords == NULL). */
    int64_t n_nodes, n_elems;       /* explicit mesh sizes (ignored if structured) */
    const double *coords;           /* [n_nodes][dim] */
    const int32_t *conn;            /* [n_elems][dim+1] */
    int nx, ny, nz;                 /* structured sizes (used when coords == NULL) */
    /* Element coefficient (cell-wise data, one value per element). */
    int coef_kind;                  /* NN_COEF_TENSOR: coef [E][3|6] = upper triangle of D_e
                                       (2D xx,xy,yy; 3D xx,xy,xz,yy,yz,zz);
                                       NN_COEF_VELOCITY: coef [E][dim] = v_e, D_e by the
                                       dispersion law with alpha_L, alpha_T, D_M */
    const double *coef;
    double alpha_L, alpha_T, D_M;
    const double *f_elem;           /* [E] source per element, or NULL for f = 0; the load is
                                       F_e[a] = f_e |e| / (dim+1) (one-point rule) */
    const uint8_t *dirichlet_mask;  /* [N] 1 = node on Gamma^D */
    const double *dirichlet_value;  /* [N] c^p at Dirichlet nodes (other entries ignored) */
    double lo, hi;                  /* bounds c_min, c_max (hi may be +INF, lo may be -INF) */
    double dt;                      /* 0: steady; > 0: backward Euler step with capacity M */
    int memory;                     /* NN_MEM_HOST or NN_MEM_DEVICE for every array above */
} nn_problem;

typedef struct nn_system nn_system;

typedef struct {
    int build_csr;                  /* also keep the reduced matrix in CSR (for NN_FMT_CSR) */
    int build_mixed;                /* also build the FP32-value copy (for NN_PREC_MIXED) */
    int keep_full;                  /* keep the full-node K, M, F (for nn_system_copy_out) */
    int lumped_mass;                /* 0 (default): consistent capacity matrix, as in the paper;
                                       1: its row-sum lumping, M_aa = |e|/(d+1) per element and
                                       vertex, no off-diagonal entries (an extension: with it,
                                       K + M/dt keeps the sign pattern of K) */
} nn_assemble_opts;

void nn_assemble_opts_default(nn_assemble_opts *o);

/* Assembles the system on the device (paper Sec. 3.2, Algorithm 1: the
 * Jacobian is computed once):
 *   CSR pattern of the node graph -> element matrices K_e = |e| G^T D_e G,
 *   consistent capacity M_e = |e|(1+delta_ab)/((d+1)(d+2)), loads F_e ->
 *   summed per node in element order (deterministic) -> Dirichlet
 *   elimination A = Kt_FF, b0 = F_F - K_FD c_D (free unknowns numbered in
 *   ascending node order) -> SELL-32 (and optional CSR / FP32) copies.
 * Host-side validation: dim, sizes, lo <= hi, Dirichlet values in [lo, hi]
 * (INFEASIBLE), NaN in coefficients (NUMERIC).  Device-side validation
 * (status word): connectivity range (INVALID_ARG), zero-measure element
 * (DEGENERATE), non-SPD D_e (NOT_SPD); a problem whose every node is a
 * Dirichlet node has no unknowns and is refused (INVALID_ARG: its solution is
 * the Dirichlet data).  Synchronizes the stream.
 * On success *out owns all device data; release with nn_system_destroy. */
nn_status nn_assemble(const nn_problem *p, const nn_assemble_opts *o, void *stream, nn_system **out);

void nn_system_destroy(nn_system *s);

typedef struct {
    int dim;
    int64_t n_nodes, n_elems, n_free;
    int64_t nnz_full;               /* nonzeros of the full-node K */
    int64_t nnz_free;               /* nonzeros of A = Kt_FF (diagonal included) */
    int64_t sell_slices, sell_stored; /* SELL-32 slices and stored off-diagonal slots */
    double lo, hi, dt;
    size_t device_bytes;            /* device memory held by the system */
    int ssor_colors;                /* colours of the SSOR ordering (0 before nn_precond_setup) */
} nn_system_desc;

nn_status nn_system_describe(const nn_system *s, nn_system_desc *d);

/* Copies one internal array into a caller buffer (for verification):
 *   0 K rowptr int64[N+1], 1 K col int32[nnz], 2 K val f64[nnz], 3 M val f64[nnz],
 *   4 F f64[N], 5 free->node int32[NF], 6 A rowptr int64[NF+1], 7 A col int32[nnzF],
 *   8 A val f64[nnzF], 9 b0 f64[NF], 10 coords f64[N*dim], 11 conn int32[E*(dim+1)],
 *   12 colour of each free unknown in the SSOR ordering int32[NF] (after nn_precond_setup).
 * Full-node arrays (0-4) need keep_full.  bytes must equal the array size.
 * Synchronizes the stream.  Errors: INVALID_ARG. */
nn_status nn_system_copy_out(const nn_system *s, int what, void *dst, size_t bytes, int dst_memory, void *stream);

/* ------------------------------------------------------------------ solve */

typedef struct {
    int solver;          /* NN_SOLVER_GPCG (gradient projection + CG, More & Toraldo),
                            NN_SOLVER_LBFGS (projected limited-memory quasi-Newton, BLMVM-like) or
                            NN_SOLVER_TRON (trust-region Newton for bounds, Lin & More 1999;
                            Sec. 3.1 and 5.1); L-BFGS and TRON run in FP64 on the SELL format */
    int precision;       /* NN_PREC_FP64, or NN_PREC_MIXED: FP32 values/vectors in inner solves,
                            FP64 residual, refinement and KKT, or NN_PREC_AUTO: MIXED for systems
                            whose FP32 operator exceeds 48 MB (it streams from HBM every product,
                            and FP32 values cut those bytes by a third) when the system has the
                            FP32 copy, FP64 otherwise (smaller solves are latency-bound and gain
                            nothing from FP32); batched solves take AUTO as FP64 */
    int format;          /* NN_FMT_SELL or NN_FMT_CSR (FP64 only) */
    double rtol;         /* stop when kkt_rel <= rtol (default 1e-10) */
    int64_t max_iter;    /* cap on matrix-vector products (default 200000) */
    int lbfgs_m;         /* L-BFGS memory (default 5, at most 16) */
    int grid_blocks;     /* persistent grid size; 0 = chosen from the size */
    double wait_timeout_s; /* bound on every device-side wait (default 5 s) */
    double inner_rtol;   /* mixed: relative tolerance of each inner solve (default 1e-4) */
    int extrapolate;     /* transient: first iterate of the QP of step n+1 (the QP and its
                            solution are unchanged, only the first iterate moves):
                            0 = c^(n); 1 = box projection of 2 c^(n) - c^(n-1);
                            2 (default) = box projection of 3 c^(n) - 3 c^(n-1) + c^(n-2)
                            (measured on the 40^3 run: 6,853 / 5,817 / 5,356 products) */
    double ksp_rtol;     /* TRON: the subspace steps of an iteration stop once the free-face
                            gradient is at most ksp_rtol times its value at the Cauchy point
                            (default 1e-1; the paper's TRON1/2/3 use 1e-1, 1e-2, 1e-3) */
    int precond;         /* preconditioner of the CG iterations (GPCG's CG phases, TRON's subspace
                            steps) on the current face F: NN_PC_JACOBI (default), z = D^-1 r, or
                            NN_PC_SSOR, z = M_F^-1 r with the multicolour symmetric SOR matrix
                            M = (D + omega L) D^-1 (D + omega U) / (omega (2 - omega)) of A_FF
                            (see nn_precond_apply).  The paper preconditions its CG with block
                            Jacobi/ILU(0) (Sec. 5, Sec. 5.1); SSOR is the triangular-sweep
                            preconditioner that a colouring makes parallel.  SSOR runs with
                            precision FP64 (AUTO is taken as FP64), the SELL format and the GPCG
                            or TRON solver; other combinations are INVALID_ARG.  The first solve
                            with SSOR builds the ordering (nn_precond_setup) if it is not built */
    double ssor_omega;   /* relaxation factor of NN_PC_SSOR, 0 < omega < 2 (default 1: symmetric
                            Gauss-Seidel) */
} nn_solve_opts;

void nn_solve_opts_default(nn_solve_opts *o);

typedef struct {
    int status;          /* nn_status of the solve */
    int64_t iterations;  /* outer iterations (GPCG phases or L-BFGS steps) */
    int64_t spmv;        /* matrix-vector products (all precisions) */
    int64_t spmv64;      /* of which FP64 */
    int64_t cg_iters;    /* CG iterations (GPCG) */
    int64_t refinements; /* mixed precision outer steps */
    double kkt_rel;      /* ||gP||_2 / ||b||_2 at exit (FP64) */
    double kkt_inf;      /* ||gP||_inf / ||b||_inf */
    double objective;    /* 1/2 x'Ax - b'x */
    double time_ms;      /* device time of the call (CUDA events) */
    double bytes_algo;   /* algorithmic bytes moved (perfect-cache model) */
    int64_t active_lo, active_hi; /* entries exactly at lo / hi */
    int64_t fp64_fallback; /* mixed: 1 if refinement stopped contracting and the solve
                              finished with FP64 iterations (the result still meets rtol) */
    double flops64_algo;   /* algorithmic FP64 operations: 2 nnz per FP64 product plus the
                              arithmetic of the fused vector passes */
    double flops_algo;     /* the same over all precisions */
    int64_t pc_applies;    /* SSOR preconditioner applications (0 with Jacobi); bytes_algo and the
                              flop counts include them */
} nn_solve_info;

/* Solves the steady QP  min 1/2 x'Ax - x'b0, lo <= x <= hi  over the free
 * unknowns (Sec. 2.1.3).  c [N] (full node vector, memory c_memory):
 * in = warm start (free entries; projected onto the box), out = solution
 * with Dirichlet entries = c^p.  All iterations run on the device in one
 * persistent launch.  Bounds are exact on output.  Returns NOT_CONVERGED
 * (best feasible iterate in c) if max_iter is reached, TIMEOUT if a device
 * wait gave up.  Synchronizes the stream.  For a transient system
 * (dt > 0) use nn_step / nn_transient. */
nn_status nn_qp_solve(nn_system *s, const nn_solve_opts *o, double *c, int c_memory, void *stream,
                      nn_solve_info *info);

/* One backward-Euler step (Sec. 2.2.2): solves the QP with
 * b = b0 + M_FF c_prev_F / dt (the c^(n) reading of ft), warm-started from
 * c_prev; writes c_next [N].  c_prev may equal c_next. */
nn_status nn_step(nn_system *s, const double *c_prev, double *c_next, int memory, const nn_solve_opts *o,
                  void *stream, nn_solve_info *info);

/* nsteps backward-Euler steps from c0 in ONE device launch; writes the
 * final state to c_final [N] and, if c_hist != NULL, every state to
 * c_hist [nsteps][N].  infos: NULL or [nsteps] per-step records (time_ms
 * is reported on the first record only).  With precision NN_PREC_MIXED
 * (system assembled with build_mixed = 1) every step's QP is solved by
 * FP32 inner solves refined in FP64; the right-hand side, the stopping
 * test and the stored states stay FP64. */
nn_status nn_transient(nn_system *s, const double *c0, int nsteps, double *c_final, double *c_hist, int memory,
                       const nn_solve_opts *o, void *stream, nn_solve_info *infos);

/* ------------------------------------------------------------- reusable plans
 * A plan holds everything one persistent solve launch of system s needs
 * (scratch vectors, barrier, counters, the chosen kernel, grid and shared
 * memory), so the same QP (Sec. 2.1.3; for a transient system nsteps
 * backward-Euler steps, Sec. 2.2.2) can be solved again and again without
 * allocation or host synchronisation: nn_plan_launch only enqueues work on
 * the stream, so launches can be issued back to back or captured into a
 * CUDA graph.  One plan serves one launch at a time (launches of the same
 * plan must be ordered on one stream).  The plan must not outlive s. */
typedef struct nn_plan nn_plan;

/* Builds a plan for options o (NULL = defaults); nsteps = 1 for a steady
 * system, >= 1 for a transient one.  Scratch is allocated on stream. */
nn_status nn_plan_create(nn_system *s, const nn_solve_opts *o, int nsteps, void *stream, nn_plan **out);

/* Enqueues one solve: c_in [N] warm start (device), c_out [N] solution
 * (device, may equal c_in), c_hist NULL or [nsteps][N] (transient).  Returns
 * without synchronising; launch errors are reported at once. */
nn_status nn_plan_launch(nn_plan *p, const double *c_in, double *c_out, double *c_hist, void *stream);

/* Waits for stream and returns the records of the plan's last launch
 * (infos: NULL or [ninfos]; time_ms is NaN: time launches with events).
 * Status as nn_qp_solve / nn_transient. */
nn_status nn_plan_result(nn_plan *p, void *stream, nn_solve_info *infos, int ninfos);

/* Frees the plan's scratch; call when its launches have completed. */
void nn_plan_destroy(nn_plan *p);

/* FP64 KKT measures of c (full node vector) for the system's QP; for a
 * transient system c_prev selects the step's right-hand side (NULL for
 * steady).  out[0] kkt_rel = ||gP||_2/||b||_2, out[1] ||gP||_inf/||b||_inf,
 * out[2] 1.0 if lo <= c_F <= hi exactly, out[3] objective.  If b = 0 the
 * denominators are ||A||_inf * max(|lo|, |hi| finite, 1).  Synchronizes. */
nn_status nn_kkt_residual(const nn_system *s, const double *c, const double *c_prev, int memory,
                          double out[4], void *stream);

/* y = A x on the free unknowns (x, y device [NF]); format NN_FMT_SELL or
 * NN_FMT_CSR; precision NN_PREC_FP64, or NN_PREC_MIXED for the FP32-value
 * operator (SELL only; x, y still FP64).  Stream-ordered, asynchronous. */
nn_status nn_spmv(const nn_system *s, const double *x, double *y, int format, int precision, void *stream);

/* y = A x with the FP32-value operator (the product of nn_spmv with
 * NN_FMT_SELL and NN_PREC_MIXED) WITHOUT allocating any device memory.
 * The paper has no counterpart; this entry point exists for callers that
 * must not allocate once they are running: for example a real-time loop
 * where cudaMalloc/cudaFree may synchronize the whole device and take an
 * unbounded time, or an application whose device memory is owned entirely
 * by another allocator and has no headroom.  nn_spmv(NN_PREC_MIXED)
 * allocates a temporary FP32 copy of x per call; this variant keeps that
 * copy in one fixed array inside the library instead.
 *   - x, y: device arrays of n_free doubles (as for nn_spmv); the system
 *     must have been assembled with build_mixed = 1.
 *   - Limit: n_free <= 4,194,304 (the array is 16 MiB of FP32).  Larger
 *     systems are rejected with NN_ERR_INVALID_ARG and a message.
 *   - Every GPU on which this library is loaded holds that 16 MiB array
 *     until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process; make that first call before any stream capture
 *     begins.  A cudaDeviceReset (or any other teardown of the device's
 *     primary context) unloads the array and leaves the kept address stale:
 *     a process that resets a device must not call this entry point on that
 *     device afterwards.
 *   - All calls share the one array and it keeps the last call's contents
 *     (each call overwrites what it reads, nothing has to start at zero).
 *     Calls whose kernels overlap on the GPU -- on different streams, or
 *     from different host threads -- race on it: order them on one stream
 *     or serialize them.
 *   - Launches two kernels on `stream`; no cudaMalloc, cudaFree or other
 *     allocating call.  Asynchronous. */
nn_status nn_spmv_mixed_noalloc(const nn_system *s, const double *x, double *y, void *stream);

/* ---------------------------------------------------- SSOR preconditioning
 * Symmetric SOR as the preconditioner of the CG iterations.  The paper's CG
 * runs with block Jacobi/ILU(0) (Sec. 5, Sec. 5.1; TRON1/2/3 use it too):
 * triangular sweeps over the unknowns in order.  Sweeps are sequential along
 * the ordering; with the unknowns ordered colour by colour (no two coupled
 * unknowns share a colour), each colour's rows depend only on other colours,
 * so a sweep is one parallel pass per colour.  With A_FF = D + L + U in that
 * ordering (L strictly lower), the preconditioner is
 *     M = (D + omega L) D^-1 (D + omega U) / (omega (2 - omega)),
 * symmetric positive definite for 0 < omega < 2 (omega = 1: symmetric
 * Gauss-Seidel), and z = M^-1 r is one forward and one backward SOR sweep
 * from z = 0. */

/* Greedy colouring by saturation degree (DSatur, Brelaz, Comm. ACM 22, 1979)
 * of the graph of an n x n pattern (host arrays rowptr int64 [n+1], col int32
 * [nnz]; diagonal entries ignored, the pattern must be symmetric): repeatedly
 * the uncoloured vertex with the most distinct colours among its neighbours
 * (ties: the larger degree, then the smaller index) takes the smallest colour
 * none of its neighbours has.  color int32 [n] receives the colours 0..k-1,
 * *ncolors = k.  On the structured meshes it finds 4 colours in 3D (the Kuhn
 * stencil's least number) and 3 in 2D.  Host only.  Errors: INVALID_ARG (bad
 * pattern, more than 64 colours). */
nn_status nn_color_dsatur(int64_t n, const int64_t *rowptr, const int32_t *col, int32_t *color, int *ncolors);

/* Builds the SSOR ordering of the system once: nn_color_dsatur of A's free
 * pattern, then the rows of each colour in ascending order, stored as
 * SELL-32 slices of their lower (earlier colour) and upper (later colour)
 * entries.  The device arrays (about the bytes of A's SELL operator) belong to
 * the system (nn_system_describe counts them).  No-op if already built.
 * The build changes the system: do not run it (or a first SSOR solve, which
 * calls it) while another call uses the same system.  Synchronizes the
 * stream.  Errors: OOM, CUDA, INVALID_ARG. */
nn_status nn_precond_setup(nn_system *s, void *stream);

/* z = P r for the preconditioner `precond` (NN_PC_JACOBI: P = D_F^-1;
 * NN_PC_SSOR: P = M_F^-1 above, relaxation omega) restricted to the face
 * F = {i : face[i] != 0} (face device uint8 [NF], or NULL for all free
 * unknowns); z_i = 0 outside F.  r, z device double [NF], distinct.  Runs
 * the solve kernels' sweep code in a launch of its own, so the tests can
 * compare it entry by entry with a plain implementation.  Builds the SSOR
 * ordering if needed.  Synchronizes the stream.  Errors: INVALID_ARG (unknown
 * precond, omega outside (0, 2), NULL vectors), TIMEOUT. */
nn_status nn_precond_apply(nn_system *s, int precond, double omega, const uint8_t *face, const double *r, double *z,
                           void *stream);

/* ------------------------------------------------------- row sharding
 * One QP spread over several ranks (one GPU each), as the paper scales one
 * problem by domain decomposition (PETSc/TAO over MPI, Sec. 3.1; strong
 * scaling, Sec. 5.1.2): rank r owns a contiguous range of the free unknowns
 * (a z-slab of the structured meshes, ranges balanced by nonzeros); a
 * product first gathers the ghost values its rows reference from their
 * owners, and a dot product is a local sum plus an all-reduce.  The plan is
 * computed on the host from the CSR pattern of A (nn_system_copy_out arrays
 * 6 and 7, or any CSR pattern with sorted columns), so every rank can build
 * its own and the plans agree.  The exchange itself belongs to the caller's
 * communicator (NCCL, MPI, ...); nn_shard_spmv is the local product. */
typedef struct {
    int rank, nranks;
    int64_t n;                      /* free unknowns of the whole system */
    int64_t row0, row1;             /* owned rows [row0, row1) */
    int64_t n_halo;                 /* ghosts: columns of owned rows outside [row0, row1) */
    int64_t nnz;                    /* nonzeros of the owned rows */
    int64_t n_send;                 /* (destination, owned id) pairs other ranks need as ghosts */
} nn_shard_desc;

/* Sizes of rank `rank`'s shard of the n x n pattern (host arrays rowptr
 * int64 [n+1], col int32 [nnz]).  Errors: INVALID_ARG. */
nn_status nn_shard_plan(int64_t n, const int64_t *rowptr, const int32_t *col, int nranks, int rank,
                        nn_shard_desc *d);

/* Fills caller host arrays of the shard (sizes from nn_shard_plan):
 *   local_rowptr int64 [row1 - row0 + 1], local_col int32 [nnz]: the owned
 *     rows with column c renumbered c - row0 if owned, else
 *     (row1 - row0) + h where h is its index in halo_ids;
 *   halo_ids int64 [n_halo] (ascending global ids), halo_owner int32 [n_halo];
 *   send_ids int64 [n_send], send_rank int32 [n_send]: the owned ids each
 *     other rank holds as ghosts, ordered by destination rank, then id.
 * The values of the local rows are A's values of rows row0..row1-1 in their
 * stored order.  Errors: INVALID_ARG. */
nn_status nn_shard_build(int64_t n, const int64_t *rowptr, const int32_t *col, int nranks, int rank,
                         int64_t *local_rowptr, int32_t *local_col, int64_t *halo_ids, int32_t *halo_owner,
                         int64_t *send_ids, int32_t *send_rank);

/* y = A_local x_ext on the device: local_rowptr/local_col/val of a shard
 * (device copies), x_ext [nrows + n_halo] = owned entries then ghosts, y
 * [nrows].  FP64.  Stream-ordered, asynchronous.  Errors: INVALID_ARG, CUDA. */
nn_status nn_shard_spmv(int64_t nrows, const int64_t *local_rowptr, const int32_t *local_col, const double *val,
                        const double *x_ext, double *y, void *stream);

/* --------------------------------------------------------------- batching */

/* Solves `count` independent steady systems in ONE persistent launch.
 * Each system is solved either by one thread block, or by one thread-block
 * cluster of 4/8/16 CTAs on as many SMs (hardware cluster barriers,
 * reductions through distributed shared memory); systems are taken largest
 * first from a device work counter.  The shape is the autotuner's choice
 * (nn_batch_autotune) or 256 threads x 1 CTA.  c[i] is the full node vector
 * of system i (device memory).  infos: NULL or [count].  Mixed precision
 * uses FP32 inner solves with FP64 refinement per system.  Synchronizes. */
nn_status nn_batch_solve(int count, nn_system *const *systems, double *const *c, const nn_solve_opts *o,
                         void *stream, nn_solve_info *infos);

/* Times candidate launch shapes (threads per block x CTAs per system:
 * 256x4, 256x8, 256x16; for batches whose largest system has at most 8192
 * free unknowns 256x1, 512x1, 256x4, 256x8) on the whole batch solved to the
 * requested tolerance, and keeps the fastest for later nn_batch_solve calls
 * in this process.  *best_shape receives threads * 100 + CTAs (e.g. 25608). */
nn_status nn_batch_autotune(int count, nn_system *const *systems, const nn_solve_opts *o, void *stream,
                            int *best_shape);

/* ---------------------------------------------------------------- serving */

typedef struct nn_server nn_server;

typedef struct {
    int max_inflight;       /* concurrent requests on the device (default 8) */
    int queue_capacity;     /* waiting requests before submit returns BUSY (default 100000) */
    int sm_share_blocks;    /* most persistent blocks of one request (0 = the whole co-resident
                               grid: large requests run alone, small ones side by side) */
    nn_solve_opts solve;    /* per-request solver options */
} nn_serve_opts;

typedef struct {
    int64_t submitted, completed, failed, rejected;
    double p50_ms, p99_ms, mean_ms;  /* latency submit -> result ready */
    double solves_per_s;             /* completed / (last completion - first submit) */
    size_t bytes_resident;           /* admission estimates of the requests admitted now */
    size_t bytes_peak;               /* largest sum of MEASURED device bytes over finished requests
                                        that held memory at the same time (each request's bytes:
                                        the most of its assembly with temporaries, or its system +
                                        solution + solve scratch) */
    size_t budget;
    int64_t inflight_peak;
    size_t bytes_reserved_peak;      /* largest sum of admission estimates (never above budget) */
    int64_t estimate_overruns;       /* finished requests whose measured bytes exceeded the estimate */
    double estimate_max_ratio;       /* largest measured / estimated bytes of a finished request */
    int64_t queued;                  /* requests waiting for admission now */
    int64_t inflight;                /* requests admitted and not finished now */
} nn_serve_stats_t;

void nn_serve_opts_default(nn_serve_opts *o);

/* Starts a serving loop on the current device: a host scheduler thread
 * admits queued requests while the estimated device bytes of the admitted
 * requests stay within hbm_budget_bytes, fewer than max_inflight run, and
 * the request's thread blocks are sure to be co-resident with those of the
 * running solves (each request's launch shape -- threads per block, blocks,
 * whether a block takes a whole SM -- is fixed when it is submitted and
 * charged against the SMs of the device; a request larger than about 32
 * slices of 32 rows per SM takes the whole device).  Each admitted request
 * is assembled and solved on its own stream, so solves of different requests
 * overlap on the device. */
nn_status nn_serve_create(size_t hbm_budget_bytes, const nn_serve_opts *o, nn_server **out);

/* Queues a steady problem (host arrays, copied before return) with its own
 * solver options o (NULL = the server's nn_serve_opts.solve; GPCG on the SELL
 * format, NN_PREC_FP64 or NN_PREC_MIXED).  Returns BUSY if the queue is full,
 * INVALID_ARG/INFEASIBLE for invalid problems or options, or INVALID_ARG if
 * the problem alone exceeds the budget. */
nn_status nn_serve_submit(nn_server *sv, const nn_problem *p, const nn_solve_opts *o, uint64_t *request_id);

/* NN_OK and the solution in c_out [N] (host) once request id finished
 * (the request is then released); BUSY while queued or running; the
 * request's failure status if it failed. */
nn_status nn_serve_poll(nn_server *sv, uint64_t id, double *c_out, nn_solve_info *info);

/* Blocks until every submitted request has finished. */
nn_status nn_serve_drain(nn_server *sv);

nn_status nn_serve_stats(nn_server *sv, nn_serve_stats_t *st);

void nn_serve_destroy(nn_server *sv);

#ifdef __cplusplus
}
#endif
#endif /* NNQP_H */
