// Entry points whose device paths are not built yet: they fail loudly.
#include "internal.h"

namespace nnqp {
nn_status lbfgs_entry(nn_system *, const nn_solve_opts *, int, const double *, double *, double *, int,
                      cudaStream_t, nn_solve_info *, int) {
    set_error("projected L-BFGS is not built in this library version");
    return NN_ERR_INVALID_ARG;
}
}  // namespace nnqp

extern "C" {
nn_status nn_batch_solve(int, nn_system *const *, double *const *, const nn_solve_opts *, void *, nn_solve_info *) {
    nnqp::set_error("nn_batch_solve is not built in this library version");
    return NN_ERR_INVALID_ARG;
}
nn_status nn_batch_autotune(int, nn_system *const *, const nn_solve_opts *, void *, int *) {
    nnqp::set_error("nn_batch_autotune is not built in this library version");
    return NN_ERR_INVALID_ARG;
}
void nn_serve_opts_default(nn_serve_opts *o) {
    if (!o) return;
    o->max_inflight = 8;
    o->queue_capacity = 100000;
    o->sm_share_blocks = 0;
    nn_solve_opts_default(&o->solve);
}
nn_status nn_serve_create(size_t, const nn_serve_opts *, nn_server **) {
    nnqp::set_error("serving is not built in this library version");
    return NN_ERR_INVALID_ARG;
}
nn_status nn_serve_submit(nn_server *, const nn_problem *, uint64_t *) { return NN_ERR_INVALID_ARG; }
nn_status nn_serve_poll(nn_server *, uint64_t, double *, nn_solve_info *) { return NN_ERR_INVALID_ARG; }
nn_status nn_serve_drain(nn_server *) { return NN_ERR_INVALID_ARG; }
nn_status nn_serve_stats(nn_server *, nn_serve_stats_t *) { return NN_ERR_INVALID_ARG; }
void nn_serve_destroy(nn_server *) {}
}
