// extern "C" entry points of libnnqp (declared in include/nnqp.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include "internal.h"

namespace nnqp {

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices];
bool g_pool_made[kMaxPoolDevices];
}  // namespace

cudaMemPool_t device_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_made[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
        uint64_t keep = 8ull << 30;   // bytes kept cached after frees
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
        g_pool_made[dev] = true;
    }
    return g_pools[dev];
}

static std::atomic<uint64_t> g_allocs{0};

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = device_pool();
    if (!pool) return cudaErrorMemoryAllocation;
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}



static thread_local char g_err[1024] = "";
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

nn_status assemble_impl(const nn_problem *p, const nn_assemble_opts *o, cudaStream_t st, nn_system **out);
nn_status mesh_structured_impl(int dim, int nx, int ny, int nz, double *coords, int32_t *conn, cudaStream_t st);
nn_status solve_entry(nn_system *s, const nn_solve_opts *o, int mode, int nsteps, const double *c_in,
                      double *c_out, double *c_hist, int memory, cudaStream_t st, nn_solve_info *infos,
                      int ninfos);
int mode_for(const nn_system *s, const nn_solve_opts *o);
nn_status kkt_impl(const nn_system *s, const double *c, const double *c_prev, int memory, double out[4],
                   cudaStream_t st);
nn_status spmv_impl(const nn_system *s, const double *x, double *y, int format, int precision, cudaStream_t st);
nn_status spmv_mixed_noalloc_impl(const nn_system *s, const double *x, double *y, cudaStream_t st);
nn_status csr_spmv_impl(int64_t nrows, const int64_t *rowptr, const int32_t *col, const double *val,
                        const double *x, double *y, cudaStream_t st);
nn_status check_opts(const nn_solve_opts *o);

nn_status check_opts(const nn_solve_opts *o) {
    if (!o) {
        set_error("solve options are NULL");
        return NN_ERR_INVALID_ARG;
    }
    if (o->solver != NN_SOLVER_GPCG && o->solver != NN_SOLVER_LBFGS && o->solver != NN_SOLVER_TRON) {
        set_error("unknown solver %d", o->solver);
        return NN_ERR_INVALID_ARG;
    }
    if (o->precision != NN_PREC_FP64 && o->precision != NN_PREC_MIXED && o->precision != NN_PREC_AUTO) {
        set_error("unknown precision %d", o->precision);
        return NN_ERR_INVALID_ARG;
    }
    if (o->format != NN_FMT_SELL && o->format != NN_FMT_CSR) {
        set_error("unknown format %d", o->format);
        return NN_ERR_INVALID_ARG;
    }
    if (!(o->rtol > 0.0) || o->max_iter < 1 || !(o->wait_timeout_s > 0.0) || o->lbfgs_m < 1 || o->lbfgs_m > 16 ||
        !(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || (o->extrapolate < 0 || o->extrapolate > 2) ||
        !(o->ksp_rtol > 0.0 && o->ksp_rtol < 1.0)) {
        set_error("invalid solve options (rtol > 0, max_iter >= 1, timeout > 0, 1 <= lbfgs_m <= 16, "
                  "0 < inner_rtol < 1, 0 <= extrapolate <= 2, 0 < ksp_rtol < 1)");
        return NN_ERR_INVALID_ARG;
    }
    if (o->precond != NN_PC_JACOBI && o->precond != NN_PC_SSOR) {
        set_error("unknown preconditioner %d", o->precond);
        return NN_ERR_INVALID_ARG;
    }
    if (o->precond == NN_PC_SSOR) {
        if (!(o->ssor_omega > 0.0 && o->ssor_omega < 2.0)) {
            set_error("SSOR needs 0 < omega < 2 (got %g)", o->ssor_omega);
            return NN_ERR_INVALID_ARG;
        }
        if (o->precision == NN_PREC_MIXED || o->format != NN_FMT_SELL || o->solver == NN_SOLVER_LBFGS) {
            set_error("the SSOR preconditioner runs in FP64 (or AUTO) on the SELL format with GPCG or TRON");
            return NN_ERR_INVALID_ARG;
        }
    }
    return NN_OK;
}

}  // namespace nnqp

using namespace nnqp;

static cudaStream_t S(void *s) { return (cudaStream_t)s; }

extern "C" {

const char *nn_last_error(void) { return g_err; }

const char *nn_version(void) { return "nnqp 0.1 (sm_103a)"; }

uint64_t nn_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

uint64_t nn_device_allocations(void) { return g_allocs.load(std::memory_order_relaxed); }

nn_status nn_mesh_counts(int dim, int nx, int ny, int nz, int64_t *n_nodes, int64_t *n_elems) {
    if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || (dim == 3 && nz < 1) || !n_nodes || !n_elems) {
        set_error("nn_mesh_counts: dim must be 2 or 3 and sizes >= 1");
        return NN_ERR_INVALID_ARG;
    }
    if (dim == 2) {
        *n_nodes = (int64_t)(nx + 1) * (ny + 1);
        *n_elems = 2LL * nx * ny;
    } else {
        *n_nodes = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
        *n_elems = 6LL * nx * ny * nz;
    }
    return NN_OK;
}

nn_status nn_mesh_structured(int dim, int nx, int ny, int nz, double *coords, int32_t *conn, void *stream) {
    clear_error();
    return mesh_structured_impl(dim, nx, ny, nz, coords, conn, S(stream));
}

void nn_assemble_opts_default(nn_assemble_opts *o) {
    if (!o) return;
    o->build_csr = 1;
    o->build_mixed = 1;
    o->keep_full = 1;
    o->lumped_mass = 0;
}

nn_status nn_assemble(const nn_problem *p, const nn_assemble_opts *o, void *stream, nn_system **out) {
    clear_error();
    if (!out) {
        set_error("nn_assemble: out is NULL");
        return NN_ERR_INVALID_ARG;
    }
    nn_assemble_opts d;
    nn_assemble_opts_default(&d);
    try {
        return assemble_impl(p, o ? o : &d, S(stream), out);
    } catch (const std::bad_alloc &) {
        set_error("nn_assemble: host allocation failed");
        return NN_ERR_OOM;
    }
}

void nn_system_destroy(nn_system *s) {
    if (!s) return;
    s->arena.release(nullptr);
    delete s;
}

nn_status nn_system_describe(const nn_system *s, nn_system_desc *d) {
    if (!s || !d) {
        set_error("nn_system_describe: NULL argument");
        return NN_ERR_INVALID_ARG;
    }
    d->dim = s->dim;
    d->n_nodes = s->N;
    d->n_elems = s->E;
    d->n_free = s->NF;
    d->nnz_full = s->nnz;
    d->nnz_free = s->nnzF;
    d->sell_slices = s->A64.nslices;
    d->sell_stored = s->A64.stored;
    d->lo = s->lo;
    d->hi = s->hi;
    d->dt = s->dt;
    d->device_bytes = s->arena.bytes;
    d->ssor_colors = s->ssor.ncolors;
    return NN_OK;
}

nn_status nn_system_copy_out(const nn_system *s, int what, void *dst, size_t bytes, int dst_memory, void *stream) {
    clear_error();
    if (!s || !dst) {
        set_error("nn_system_copy_out: NULL argument");
        return NN_ERR_INVALID_ARG;
    }
    const void *src = nullptr;
    size_t need = 0;
    switch (what) {
        case 0: src = s->rowptr; need = sizeof(int64_t) * (s->N + 1); break;
        case 1: src = s->col; need = sizeof(int32_t) * s->nnz; break;
        case 2: src = s->Kval; need = sizeof(double) * s->nnz; break;
        case 3: src = s->Mval; need = sizeof(double) * s->nnz; break;
        case 4: src = s->F; need = sizeof(double) * s->N; break;
        case 5: src = s->free_node; need = sizeof(int32_t) * s->NF; break;
        case 6: src = s->arow; need = sizeof(int64_t) * (s->NF + 1); break;
        case 7: src = s->acol; need = sizeof(int32_t) * s->nnzF; break;
        case 8: src = s->aval; need = sizeof(double) * s->nnzF; break;
        case 9: src = s->b0; need = sizeof(double) * s->NF; break;
        case 10: src = s->coords; need = sizeof(double) * s->N * s->dim; break;
        case 11: src = s->conn; need = sizeof(int32_t) * s->E * (s->dim + 1); break;
        case 12: {   // host array
            if (s->ssor_color.empty()) {
                set_error("nn_system_copy_out: the SSOR ordering is not built (nn_precond_setup)");
                return NN_ERR_INVALID_ARG;
            }
            need = sizeof(int32_t) * s->NF;
            if (bytes != need) {
                set_error("nn_system_copy_out: array 12 has %zu bytes, buffer has %zu", need, bytes);
                return NN_ERR_INVALID_ARG;
            }
            if (dst_memory == NN_MEM_DEVICE) {
                NN_CUDA_TRY(cudaMemcpyAsync(dst, s->ssor_color.data(), need, cudaMemcpyHostToDevice, S(stream)));
                NN_CUDA_TRY(cudaStreamSynchronize(S(stream)));
            } else {
                std::memcpy(dst, s->ssor_color.data(), need);
            }
            return NN_OK;
        }
        default: set_error("nn_system_copy_out: unknown array %d", what); return NN_ERR_INVALID_ARG;
    }
    if (!src) {
        set_error("nn_system_copy_out: array %d was not kept by this system", what);
        return NN_ERR_INVALID_ARG;
    }
    if (bytes != need) {
        set_error("nn_system_copy_out: array %d has %zu bytes, buffer has %zu", what, need, bytes);
        return NN_ERR_INVALID_ARG;
    }
    cudaMemcpyKind kind = dst_memory == NN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    NN_CUDA_TRY(cudaMemcpyAsync(dst, src, need, kind, S(stream)));
    NN_CUDA_TRY(cudaStreamSynchronize(S(stream)));
    return NN_OK;
}

void nn_solve_opts_default(nn_solve_opts *o) {
    if (!o) return;
    o->solver = NN_SOLVER_GPCG;
    o->precision = NN_PREC_FP64;
    o->format = NN_FMT_SELL;
    o->rtol = 1e-10;
    o->max_iter = 200000;
    o->lbfgs_m = 5;
    o->grid_blocks = 0;
    o->wait_timeout_s = 5.0;
    o->inner_rtol = 1e-4;
    o->extrapolate = 2;
    o->ksp_rtol = 1e-1;
    o->precond = NN_PC_JACOBI;
    o->ssor_omega = 1.0;
}

static nn_status solve_common(nn_system *s, const nn_solve_opts *o, int want_transient, int nsteps,
                              const double *c_in, double *c_out, double *c_hist, int memory, void *stream,
                              nn_solve_info *infos, int ninfos) {
    clear_error();
    nn_solve_opts d;
    nn_solve_opts_default(&d);
    if (!o) o = &d;
    if (!s || !c_in || !c_out) {
        set_error("NULL system or vector");
        return NN_ERR_INVALID_ARG;
    }
    NN_TRY(check_opts(o));
    if (memory != NN_MEM_HOST && memory != NN_MEM_DEVICE) {
        set_error("memory flag must be NN_MEM_HOST or NN_MEM_DEVICE");
        return NN_ERR_INVALID_ARG;
    }
    if (nsteps < 1) {
        set_error("nsteps must be >= 1");
        return NN_ERR_INVALID_ARG;
    }
    if (want_transient && !(s->dt > 0.0)) {
        set_error("this system is steady (dt = 0): use nn_qp_solve");
        return NN_ERR_INVALID_ARG;
    }
    if (!want_transient && s->dt > 0.0) {
        set_error("this system is transient (dt > 0): use nn_step or nn_transient");
        return NN_ERR_INVALID_ARG;
    }
    return solve_entry(s, o, mode_for(s, o), nsteps, c_in, c_out, c_hist, memory, S(stream), infos, ninfos);
}

nn_status nn_qp_solve(nn_system *s, const nn_solve_opts *o, double *c, int c_memory, void *stream,
                      nn_solve_info *info) {
    return solve_common(s, o, 0, 1, c, c, nullptr, c_memory, stream, info, info ? 1 : 0);
}

nn_status nn_step(nn_system *s, const double *c_prev, double *c_next, int memory, const nn_solve_opts *o,
                  void *stream, nn_solve_info *info) {
    return solve_common(s, o, 1, 1, c_prev, c_next, nullptr, memory, stream, info, info ? 1 : 0);
}

nn_status nn_transient(nn_system *s, const double *c0, int nsteps, double *c_final, double *c_hist, int memory,
                       const nn_solve_opts *o, void *stream, nn_solve_info *infos) {
    return solve_common(s, o, 1, nsteps, c0, c_final, c_hist, memory, stream, infos, infos ? nsteps : 0);
}

nn_status nn_kkt_residual(const nn_system *s, const double *c, const double *c_prev, int memory, double out[4],
                          void *stream) {
    clear_error();
    if (!s || !c || !out) {
        set_error("nn_kkt_residual: NULL argument");
        return NN_ERR_INVALID_ARG;
    }
    return kkt_impl(s, c, c_prev, memory, out, S(stream));
}

nn_status nn_spmv(const nn_system *s, const double *x, double *y, int format, int precision, void *stream) {
    clear_error();
    if (!s || ((!x || !y) && s->NF > 0)) {
        set_error("nn_spmv: NULL argument");
        return NN_ERR_INVALID_ARG;
    }
    return spmv_impl(s, x, y, format, precision, S(stream));
}

nn_status nn_shard_spmv(int64_t nrows, const int64_t *local_rowptr, const int32_t *local_col, const double *val,
                        const double *x_ext, double *y, void *stream) {
    clear_error();
    if (nrows < 0 || (nrows > 0 && (!local_rowptr || !local_col || !val || !x_ext || !y))) {
        set_error("nn_shard_spmv: nrows >= 0 and device arrays are required");
        return NN_ERR_INVALID_ARG;
    }
    return csr_spmv_impl(nrows, local_rowptr, local_col, val, x_ext, y, S(stream));
}

nn_status nn_spmv_mixed_noalloc(const nn_system *s, const double *x, double *y, void *stream) {
    clear_error();
    if (!s || ((!x || !y) && s->NF > 0)) {
        set_error("nn_spmv_mixed_noalloc: NULL argument");
        return NN_ERR_INVALID_ARG;
    }
    return spmv_mixed_noalloc_impl(s, x, y, S(stream));
}

}  // extern "C"
