// Internal host-side definitions shared by the translation units of libnnqp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <vector>
#include "../../include/nnqp.h"

namespace nnqp {

// Thread-local error message (nn_last_error).
void set_error(const char *fmt, ...);
void clear_error();
// Counts kernel launches made by the library (nn_kernel_launches).
void count_launch();

#define NN_CUDA_TRY(expr)                                                         \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) {                                                  \
            ::nnqp::set_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(_e),    \
                              __FILE__, __LINE__);                                \
            return _e == cudaErrorMemoryAllocation ? NN_ERR_OOM : NN_ERR_CUDA;    \
        }                                                                         \
    } while (0)

#define NN_TRY(expr)                      \
    do {                                  \
        nn_status _s = (expr);            \
        if (_s != NN_OK) return _s;       \
    } while (0)

// SELL-32 storage of the off-diagonal part of a square matrix: slice s holds
// rows [32s, 32s+32); its width w_s = max off-diagonal count of those rows,
// rounded up to even; entry k of row 32s+l is at
// sptr[s] + 64 (k/2) + 2l + (k%2) (pairs of entries interleaved by row,
// sell_idx in ops.cuh).  Padding slots carry the row's own column and value 0.
template <typename T>
struct SellMat {
    int64_t n = 0;
    int64_t nslices = 0;
    int64_t stored = 0;          // sptr[nslices]
    int64_t *sptr = nullptr;     // [nslices+1], shared between value copies
    int32_t *col = nullptr;      // [stored],    shared between value copies
    T *val = nullptr;            // [stored]
};

// Device view of the multicolour SSOR ordering of A = Kt_FF (nn_precond_setup).
// The rows of colour c fill slices cslice[c] .. cslice[c+1]-1 of 32 rows each,
// rows ascending; lane l of slice s is free unknown row[32s + l] (-1 = padding
// lane).  Entry k of that lane's lower part (columns of earlier colours) is at
// lptr[s] + 32k + l, of its upper part (later colours) at uptr[s] + 32k + l;
// slices are as wide as their longest row, the padding entries carry value 0
// and a column that the sweep has already written in that pass (the first row
// of colour 0 for lower parts, of the last colour for upper parts).
struct SsorF64 {
    int ncolors;
    bool stream;             // parts far larger than L2: evict-first loads
    double omega;
    const int64_t *cslice;   // [ncolors + 1]
    const int32_t *row;      // [32 * slices]
    const int64_t *lptr;     // [slices + 1]
    const int64_t *uptr;     // [slices + 1]
    const int32_t *lcol, *ucol;
    const double *lval, *uval;
};

// Device allocations owned by one object, released together.
// The library's stream-ordered memory pool on the current device.  Unlike
// the device's default pool it never makes one stream wait for another to
// reuse freed memory (no internal dependencies), so solves running on
// different streams (serving workers, user streams) stay concurrent; freed
// memory stays cached in the pool up to a release threshold.
cudaMemPool_t device_pool();

// Stream-ordered allocation from device_pool().
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st);

struct DevArena {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    template <typename T>
    nn_status alloc(T **out, size_t count, cudaStream_t st) {
        *out = nullptr;
        if (count == 0) count = 1;
        void *p = nullptr;
        cudaError_t e = pool_alloc(&p, count * sizeof(T), st);
        if (e != cudaSuccess) {
            set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? NN_ERR_OOM : NN_ERR_CUDA;
        }
        ptrs.push_back(p);
        bytes += count * sizeof(T);
        *out = (T *)p;
        return NN_OK;
    }
    void release(cudaStream_t st) {
        for (void *p : ptrs) cudaFreeAsync(p, st);
        ptrs.clear();
        bytes = 0;
    }
};

}  // namespace nnqp

struct nn_system {
    int dim = 0;
    int64_t N = 0, E = 0, NF = 0, nnz = 0, nnzF = 0;
    double lo = 0, hi = 0, dt = 0;
    nnqp::DevArena arena;
    // mesh
    double *coords = nullptr;
    int32_t *conn = nullptr;
    // full-node CSR (kept when keep_full)
    int64_t *rowptr = nullptr;
    int32_t *col = nullptr;
    double *Kval = nullptr, *Mval = nullptr, *F = nullptr;
    // Dirichlet data and the free numbering
    uint8_t *dmask = nullptr;       // [N]
    double *dval = nullptr;         // [N] c^p at Dirichlet nodes, 0 elsewhere
    int32_t *free_node = nullptr;   // [NF] node id of free unknown i (ascending)
    // reduced matrix A = Kt_FF: CSR (optional) and SELL-32
    int64_t *arow = nullptr;
    int32_t *acol = nullptr;
    double *aval = nullptr;
    nnqp::SellMat<double> A64;      // off-diagonals, FP64
    double *diag64 = nullptr;       // [NF]
    double *dinv64 = nullptr;       // [NF]
    nnqp::SellMat<float> A32;       // off-diagonals, FP32 (shares sptr/col with A64)
    std::vector<int64_t> sptr_host; // host copy of A64.sptr, made on first use (grid sizing)
    float *rsum32 = nullptr;        // [NF] row sums of A over free columns
    float *dinv32 = nullptr;        // [NF] 1 / (rsum - sum of FP32 off-diagonals)
    nnqp::SellMat<double> M64;      // transient: off-diagonals of M_FF (shares sptr/col)
    double *mdiag64 = nullptr;      // [NF]
    double *b0 = nullptr;           // [NF] F_F - K_FD c_D
    size_t assembly_peak_bytes = 0; // device bytes held at the end of assembly (system + temporaries)
    nnqp::SsorF64 ssor{};           // SSOR ordering (ncolors = 0 until nn_precond_setup)
    int64_t ssor_slices = 0;
    std::vector<int32_t> ssor_color; // colour of each free unknown (host)
    double anorm_inf = 0;           // ||A||_inf
    double b0norm = 0;              // ||b0||_2
    bool has_csr = false, has_mixed = false, has_full = false;
};

namespace nnqp {
// Host arrays of the SSOR ordering (the device view SsorF64 points at copies).
struct SsorHost {
    int ncolors = 0;
    std::vector<int32_t> color;                 // [n]
    std::vector<int64_t> cslice, lptr, uptr;    // [ncolors+1], [slices+1], [slices+1]
    std::vector<int32_t> row, lcol, ucol;
    std::vector<double> lval, uval;
};
// The ordering of the n x n matrix whose off-diagonals are held in
// pair-interleaved SELL-32 (ns slices, host copies of sptr / col / val).
nn_status ssor_layout(int64_t n, int64_t ns, const int64_t *sptr, const int32_t *scol, const double *sval,
                      SsorHost &h);
// Builds the SSOR ordering of s once (nn_precond_setup); synchronizes st.
nn_status ssor_setup(nn_system *s, cudaStream_t st);
// DSatur colouring of a symmetric pattern (nn_color_dsatur), without the
// argument checks.
nn_status dsatur_color(int64_t n, const int64_t *rowptr, const int32_t *col, int32_t *color, int *ncolors);
}  // namespace nnqp
