// Row sharding of one QP over several ranks (host planning).
//
// The paper scales one problem by domain decomposition over MPI ranks: each
// rank owns part of the unknowns, every matrix-vector product first scatters
// the ghost values its rows need from their owners, and every dot product is
// a local sum followed by an all-reduce (PETSc/TAO, Sec. 3.1; strong scaling
// of the cube with a hole, Sec. 5.1.2).  Here the unknowns are the free
// unknowns of A = Kt_FF in ascending node order; rank r owns one contiguous
// range of them.  On the structured meshes (node id i + (nx+1)(j + (ny+1)k))
// a contiguous range is a z-slab, so a rank's ghosts come from the slabs just
// below and above it.  Everything here works on a CSR pattern given by the
// caller, so the plan of every rank can be computed (and checked) anywhere.
#include <algorithm>
#include <cstring>
#include <vector>
#include "internal.h"

namespace nnqp {

namespace {

// Rows [row0, row1) of rank `rank`: contiguous ranges balanced by nonzeros
// (rank r takes the rows whose nonzero prefix falls in [r, r+1) nnz/nranks).
void rows_of_rank(int64_t n, const int64_t *rowptr, int nranks, int rank, int64_t *row0, int64_t *row1) {
    const int64_t nnz = rowptr[n];
    auto first_row_at = [&](int r) -> int64_t {
        if (r <= 0) return 0;
        if (r >= nranks) return n;
        const int64_t target = (nnz * (int64_t)r + nranks - 1) / nranks;
        return (int64_t)(std::lower_bound(rowptr, rowptr + n + 1, target) - rowptr);
    };
    *row0 = std::min(first_row_at(rank), n);
    *row1 = std::max(*row0, std::min(first_row_at(rank + 1), n));
}

// The rank whose range holds column c.
int owner_of(int64_t n, const int64_t *rowptr, int nranks, int64_t c) {
    for (int r = 0; r < nranks; ++r) {
        int64_t r0, r1;
        rows_of_rank(n, rowptr, nranks, r, &r0, &r1);
        if (c >= r0 && c < r1) return r;
    }
    return -1;
}

nn_status check_args(int64_t n, const int64_t *rowptr, const int32_t *col, int nranks, int rank) {
    if (n < 1 || !rowptr || !col || nranks < 1 || rank < 0 || rank >= nranks) {
        set_error("nn_shard: need n >= 1, rowptr, col, nranks >= 1 and 0 <= rank < nranks");
        return NN_ERR_INVALID_ARG;
    }
    if (rowptr[0] != 0) {
        set_error("nn_shard: rowptr[0] must be 0");
        return NN_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) {
            set_error("nn_shard: rowptr must not decrease (row %lld)", (long long)i);
            return NN_ERR_INVALID_ARG;
        }
    for (int64_t q = 0; q < rowptr[n]; ++q)
        if (col[q] < 0 || col[q] >= n) {
            set_error("nn_shard: column %d at entry %lld is outside [0, %lld)", col[q], (long long)q, (long long)n);
            return NN_ERR_INVALID_ARG;
        }
    return NN_OK;
}

// Ghost columns (ascending) of the rows [r0, r1).
std::vector<int64_t> ghosts_of(const int64_t *rowptr, const int32_t *col, int64_t r0, int64_t r1) {
    std::vector<int64_t> g;
    for (int64_t q = rowptr[r0]; q < rowptr[r1]; ++q)
        if (col[q] < r0 || col[q] >= r1) g.push_back(col[q]);
    std::sort(g.begin(), g.end());
    g.erase(std::unique(g.begin(), g.end()), g.end());
    return g;
}

// Owned unknowns of `rank` that other ranks hold as ghosts: (destination,
// id) pairs ordered by destination, then id.
std::vector<std::pair<int, int64_t>> sends_of(int64_t n, const int64_t *rowptr, const int32_t *col, int nranks,
                                              int rank) {
    int64_t r0, r1;
    rows_of_rank(n, rowptr, nranks, rank, &r0, &r1);
    std::vector<std::pair<int, int64_t>> s;
    for (int q = 0; q < nranks; ++q) {
        if (q == rank) continue;
        int64_t q0, q1;
        rows_of_rank(n, rowptr, nranks, q, &q0, &q1);
        for (int64_t c : ghosts_of(rowptr, col, q0, q1))
            if (c >= r0 && c < r1) s.push_back({q, c});
    }
    return s;
}

}  // namespace
}  // namespace nnqp

using namespace nnqp;

extern "C" {

nn_status nn_shard_plan(int64_t n, const int64_t *rowptr, const int32_t *col, int nranks, int rank,
                        nn_shard_desc *d) {
    clear_error();
    if (!d) {
        set_error("nn_shard_plan: NULL output");
        return NN_ERR_INVALID_ARG;
    }
    NN_TRY(check_args(n, rowptr, col, nranks, rank));
    std::memset(d, 0, sizeof(*d));
    d->rank = rank;
    d->nranks = nranks;
    d->n = n;
    rows_of_rank(n, rowptr, nranks, rank, &d->row0, &d->row1);
    d->nnz = rowptr[d->row1] - rowptr[d->row0];
    d->n_halo = (int64_t)ghosts_of(rowptr, col, d->row0, d->row1).size();
    d->n_send = (int64_t)sends_of(n, rowptr, col, nranks, rank).size();
    return NN_OK;
}

nn_status nn_shard_build(int64_t n, const int64_t *rowptr, const int32_t *col, int nranks, int rank,
                         int64_t *local_rowptr, int32_t *local_col, int64_t *halo_ids, int32_t *halo_owner,
                         int64_t *send_ids, int32_t *send_rank) {
    clear_error();
    NN_TRY(check_args(n, rowptr, col, nranks, rank));
    int64_t r0, r1;
    rows_of_rank(n, rowptr, nranks, rank, &r0, &r1);
    const int64_t nrows = r1 - r0;
    const std::vector<int64_t> g = ghosts_of(rowptr, col, r0, r1);
    const std::vector<std::pair<int, int64_t>> snd = sends_of(n, rowptr, col, nranks, rank);
    if (!local_rowptr || (rowptr[r1] > rowptr[r0] && !local_col) || (!g.empty() && (!halo_ids || !halo_owner)) ||
        (!snd.empty() && (!send_ids || !send_rank))) {
        set_error("nn_shard_build: an output array is NULL");
        return NN_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i <= nrows; ++i) local_rowptr[i] = rowptr[r0 + i] - rowptr[r0];
    for (int64_t q = rowptr[r0]; q < rowptr[r1]; ++q) {
        const int64_t c = col[q];
        local_col[q - rowptr[r0]] =
            (int32_t)(c >= r0 && c < r1 ? c - r0 : nrows + (std::lower_bound(g.begin(), g.end(), c) - g.begin()));
    }
    for (size_t h = 0; h < g.size(); ++h) {
        halo_ids[h] = g[h];
        halo_owner[h] = owner_of(n, rowptr, nranks, g[h]);
    }
    for (size_t k = 0; k < snd.size(); ++k) {
        send_rank[k] = snd[k].first;
        send_ids[k] = snd[k].second;
    }
    return NN_OK;
}

}  // extern "C"
