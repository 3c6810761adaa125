// Serving loop: continuous admission of steady QP requests.
//
// Requests are queued by nn_serve_submit (host arrays copied at once).  A
// scheduler thread admits the oldest queued request when (a) a worker slot
// is free, (b) its device-memory estimate fits in the HBM budget next to the
// requests already resident, and (c) its thread blocks are sure to be
// co-resident with those of the requests already running (admission.h: the
// launch shape of every request -- threads per block, blocks, and whether a
// block takes a whole SM -- is fixed at submit time and enforced at launch).
// Each worker owns a CUDA stream: it assembles the request's system, solves
// it in one persistent cooperative launch and copies the solution back, so
// the device work of different requests overlaps.  Large requests take the
// whole co-resident grid and run alone; small ones run side by side.  (One
// thread-block cluster per request was measured too: on 8-16 SMs a request's
// FP64 passes take 3-10x longer than on its grid share, and small requests
// gain nothing.)
//
// Memory: admission charges each request an upper estimate of its device
// bytes (estimate_bytes); the worker then measures what the request really
// holds (the assembled system, the assembly's temporaries, the solve's
// scratch and the solution vector) and the statistics report those measured
// bytes, plus every request whose measured bytes exceeded its estimate.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>
#include "internal.h"
#include "admission.h"

namespace nnqp {

nn_status assemble_impl(const nn_problem *p, const nn_assemble_opts *o, cudaStream_t st, nn_system **out);
nn_status check_opts(const nn_solve_opts *o);
nn_status serve_solve(nn_system *s, const nn_solve_opts *o, const double *c_in_dev, double *c_out_dev,
                      cudaStream_t st, int tpb, int grid_blocks, nn_solve_info *info, size_t *plan_bytes);
int solve_grid_blocks_per_sm(int *sms);

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    nn_problem p{};
    std::vector<double> coords, coef, fel, dval;
    std::vector<int32_t> conn;
    std::vector<uint8_t> dmask;
    int64_t N = 0, E = 0;
    nn_solve_opts opts{};         // this request's solver options
    size_t bytes = 0;             // admission estimate
    size_t measured = 0;          // device bytes the request really held
    RequestShape shape;
    Clock::time_point t_submit, t_start, t_done;   // t_start: a worker took it (device work begins)
    std::vector<double> result;
    nn_solve_info info{};
    nn_status status = NN_ERR_BUSY;
    std::string error;            // the worker's message when the request failed
    bool done = false;
};

struct Server {
    size_t budget = 0;
    nn_serve_opts opts{};
    int device = 0;
    BlockLedger ledger;           // blocks of the running solves, by class
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> table;
    std::deque<std::shared_ptr<Request>> ready;      // admitted, waiting for a worker
    uint64_t next_id = 1;
    size_t reserved = 0, reserved_peak = 0;   // admission estimates of the running requests
    struct Held { Clock::time_point t0, t1; size_t bytes; };
    std::vector<Held> held;                   // measured device bytes of every finished request
    int64_t overruns = 0;                     // requests whose measured bytes exceeded the estimate
    double worst_ratio = 0.0;                 // largest measured / estimate
    int inflight = 0;
    int64_t inflight_peak = 0;
    int64_t submitted = 0, completed = 0, failed = 0, rejected = 0;
    std::vector<double> lat_ms;
    Clock::time_point first_submit, last_done;
    bool have_first = false;
    bool stop = false;
    std::thread sched;
    std::vector<std::thread> workers;
};

namespace {

// Upper estimate of the device bytes one request holds while it runs (the
// most of: assembly with its temporaries -- element matrices, incidence
// lists, scans -- or the assembled system with the solve's vectors); the
// mixed path adds its FP32 operator values and vectors.  Checked against the
// measured bytes of every served request (estimate_overruns).
size_t estimate_bytes(int dim, int64_t N, int64_t E, bool mixed) {
    const double nnz = (dim == 3 ? 16.0 : 7.5) * (double)N;
    const double b = 52.0 * nnz + (mixed ? 360.0 : 300.0) * N + (dim == 3 ? 150.0 : 110.0) * E + (4 << 20);
    return (size_t)b;
}

// Whether a request needs the FP32 operator copy: mixed precision, or
// NN_PREC_AUTO on a system whose FP32 operator (about 16 or 7.5 nonzeros per
// node in 3D or 2D, 8 bytes each) exceeds the 48 MB streaming threshold.
bool uses_fp32(const nn_solve_opts &o, int dim, int64_t N) {
    if (o.precision == NN_PREC_MIXED) return true;
    const double nnz = (dim == 3 ? 16.0 : 7.5) * (double)N;
    return o.precision == NN_PREC_AUTO && nnz * 8.0 > 48.0 * (1 << 20);
}

void worker_loop(Server *sv) {
    cudaSetDevice(sv->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_sched.wait(lk, [&] { return sv->stop || !sv->ready.empty(); });
            if (sv->stop && sv->ready.empty()) break;
            r = sv->ready.front();
            sv->ready.pop_front();
            r->t_start = Clock::now();
        }
        nn_assemble_opts ao;
        nn_assemble_opts_default(&ao);
        ao.build_mixed = uses_fp32(r->opts, r->p.dim, r->N);
        nn_system *s = nullptr;
        nn_status stt = assemble_impl(&r->p, &ao, st, &s);
        double *dc = nullptr;
        size_t plan_bytes = 0, measured = 0;
        if (stt == NN_OK) {
            if (pool_alloc((void **)&dc, sizeof(double) * r->N, st) != cudaSuccess) stt = NN_ERR_OOM;
        }
        if (stt == NN_OK) {
            cudaMemsetAsync(dc, 0, sizeof(double) * r->N, st);
            stt = serve_solve(s, &r->opts, dc, dc, st, r->shape.tpb, r->shape.blocks, &r->info, &plan_bytes);
            // the most the request held at once: the assembly's peak (system +
            // temporaries), or the system + solution vector + solve scratch
            measured = std::max(s->assembly_peak_bytes, s->arena.bytes + sizeof(double) * r->N + plan_bytes);
            if (stt == NN_OK || stt == NN_ERR_NOT_CONVERGED) {
                r->result.resize(r->N);
                cudaError_t e = cudaMemcpyAsync(r->result.data(), dc, sizeof(double) * r->N,
                                                cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) {
                    set_error("serving: result copy failed: %s", cudaGetErrorString(e));
                    stt = NN_ERR_CUDA;
                }
            }
        }
        if (dc) cudaFreeAsync(dc, st);
        if (s) {
            s->arena.release(st);
            delete s;
        }
        cudaStreamSynchronize(st);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->status = stt;
            r->info.status = stt;
            if (stt != NN_OK && stt != NN_ERR_NOT_CONVERGED) r->error = nn_last_error();
            r->t_done = Clock::now();
            r->done = true;
            r->measured = measured;
            if (measured > r->bytes) ++sv->overruns;
            sv->worst_ratio = std::max(sv->worst_ratio, (double)measured / (double)r->bytes);
            if (measured > 0) sv->held.push_back({r->t_start, r->t_done, measured});
            sv->reserved -= r->bytes;
            sv->ledger.release(r->shape);
            --sv->inflight;
            if (stt == NN_OK) {
                ++sv->completed;
                sv->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
                sv->last_done = r->t_done;
            } else {
                ++sv->failed;
            }
            // drop the copied input arrays now; the result stays until polled
            r->coords.clear(); r->coef.clear(); r->fel.clear(); r->dval.clear(); r->conn.clear(); r->dmask.clear();
        }
        sv->cv_sched.notify_all();
        sv->cv_done.notify_all();
    }
    cudaStreamDestroy(st);
}

void sched_loop(Server *sv) {
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv_sched.wait(lk, [&] {
            if (sv->stop) return true;
            if (sv->queue.empty()) return false;
            const auto &r = sv->queue.front();
            return sv->inflight < sv->opts.max_inflight && sv->reserved + r->bytes <= sv->budget &&
                   sv->ledger.can_admit(r->shape);
        });
        if (sv->stop) break;
        auto r = sv->queue.front();
        sv->queue.pop_front();
        sv->reserved += r->bytes;
        sv->reserved_peak = std::max(sv->reserved_peak, sv->reserved);
        sv->ledger.admit(r->shape);
        ++sv->inflight;
        sv->inflight_peak = std::max<int64_t>(sv->inflight_peak, sv->inflight);
        sv->ready.push_back(r);
        sv->cv_sched.notify_all();
    }
}

}  // namespace
}  // namespace nnqp

using namespace nnqp;

struct nn_server {
    Server s;
};

extern "C" {

void nn_serve_opts_default(nn_serve_opts *o) {
    if (!o) return;
    o->max_inflight = 8;
    o->queue_capacity = 100000;
    o->sm_share_blocks = 0;
    nn_solve_opts_default(&o->solve);
}

nn_status nn_serve_create(size_t hbm_budget_bytes, const nn_serve_opts *o, nn_server **out) {
    clear_error();
    if (!out || hbm_budget_bytes == 0) {
        set_error("nn_serve_create: out and a nonzero budget are required");
        return NN_ERR_INVALID_ARG;
    }
    nn_serve_opts d;
    nn_serve_opts_default(&d);
    if (!o) o = &d;
    NN_TRY(check_opts(&o->solve));
    if (o->max_inflight < 1 || o->max_inflight > 64 || o->queue_capacity < 1 ||
        o->solve.solver != NN_SOLVER_GPCG || o->solve.format != NN_FMT_SELL || o->solve.precond != NN_PC_JACOBI) {
        set_error("nn_serve_create: 1 <= max_inflight <= 64, queue_capacity >= 1, GPCG on SELL with Jacobi");
        return NN_ERR_INVALID_ARG;
    }
    nn_server *h = new nn_server();
    Server *sv = &h->s;
    sv->budget = hbm_budget_bytes;
    sv->opts = *o;
    cudaGetDevice(&sv->device);
    int sms = 0;
    const int per = solve_grid_blocks_per_sm(&sms);
    sv->ledger.sms = sms;
    sv->ledger.small_per_sm = per;
    if (per < 1 || sms < 1 || per > 64) {
        delete h;
        set_error("nn_serve_create: cannot size the solve kernel on this device");
        return NN_ERR_CUDA;
    }
    sv->sched = std::thread(sched_loop, sv);
    for (int i = 0; i < o->max_inflight; ++i) sv->workers.emplace_back(worker_loop, sv);
    *out = h;
    return NN_OK;
}

nn_status nn_serve_submit(nn_server *h, const nn_problem *p, const nn_solve_opts *o, uint64_t *request_id) {
    clear_error();
    if (!h || !p || !request_id) {
        set_error("nn_serve_submit: NULL argument");
        return NN_ERR_INVALID_ARG;
    }
    Server *sv = &h->s;
    if (p->memory != NN_MEM_HOST) {
        set_error("nn_serve_submit: requests carry host arrays");
        return NN_ERR_INVALID_ARG;
    }
    if ((p->dim != 2 && p->dim != 3) || !p->coef || !p->dirichlet_mask || !p->dirichlet_value) {
        set_error("nn_serve_submit: dim 2|3, coef and Dirichlet arrays are required");
        return NN_ERR_INVALID_ARG;
    }
    if (std::isnan(p->lo) || std::isnan(p->hi) || p->lo > p->hi) {
        set_error("nn_serve_submit: bounds must satisfy lo <= hi");
        return NN_ERR_INFEASIBLE;
    }
    if (p->dt != 0.0) {
        set_error("nn_serve_submit: serving takes steady problems");
        return NN_ERR_INVALID_ARG;
    }
    if (!o) o = &sv->opts.solve;
    NN_TRY(check_opts(o));
    if (o->solver != NN_SOLVER_GPCG || o->format != NN_FMT_SELL || o->precond != NN_PC_JACOBI) {
        set_error("nn_serve_submit: served requests are solved by Jacobi-preconditioned GPCG on the SELL format");
        return NN_ERR_INVALID_ARG;
    }
    auto r = std::make_shared<Request>();
    r->opts = *o;
    const int dim = p->dim, nv = dim + 1;
    if (p->coords) {
        r->N = p->n_nodes;
        r->E = p->n_elems;
    } else {
        NN_TRY(nn_mesh_counts(dim, p->nx, p->ny, p->nz, &r->N, &r->E));
    }
    if (r->N < 1 || r->E < 1) {
        set_error("nn_serve_submit: empty mesh");
        return NN_ERR_INVALID_ARG;
    }
    r->bytes = estimate_bytes(dim, r->N, r->E, uses_fp32(r->opts, dim, r->N));
    if (r->bytes > sv->budget) {
        set_error("nn_serve_submit: the request alone (%zu bytes) exceeds the budget", r->bytes);
        return NN_ERR_INVALID_ARG;
    }
    // launch shape, fixed now (the free unknowns are at most the nodes):
    // large requests take the whole co-resident grid and run alone at full
    // speed (bandwidth- and FP64-bound solves gain nothing from sharing the
    // device, and blocks of other grids slow their barriers), small ones run
    // side by side
    r->shape = request_shape((r->N + 31) / 32, sv->ledger.sms, sv->ledger.small_per_sm, sv->opts.sm_share_blocks);
    if (!sv->ledger.fits_alone(r->shape)) {
        set_error("nn_serve_submit: the request's grid does not fit on the device");
        return NN_ERR_INVALID_ARG;
    }
    const int ncoef = p->coef_kind == NN_COEF_TENSOR ? (dim == 2 ? 3 : 6) : dim;
    r->coef.assign(p->coef, p->coef + (size_t)r->E * ncoef);
    if (p->f_elem) r->fel.assign(p->f_elem, p->f_elem + r->E);
    r->dmask.assign(p->dirichlet_mask, p->dirichlet_mask + r->N);
    r->dval.assign(p->dirichlet_value, p->dirichlet_value + r->N);
    if (p->coords) {
        r->coords.assign(p->coords, p->coords + (size_t)r->N * dim);
        r->conn.assign(p->conn, p->conn + (size_t)r->E * nv);
    }
    r->p = *p;
    r->p.coef = r->coef.data();
    r->p.f_elem = p->f_elem ? r->fel.data() : nullptr;
    r->p.dirichlet_mask = r->dmask.data();
    r->p.dirichlet_value = r->dval.data();
    r->p.coords = p->coords ? r->coords.data() : nullptr;
    r->p.conn = p->coords ? r->conn.data() : nullptr;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if ((int64_t)sv->queue.size() >= sv->opts.queue_capacity) {
            ++sv->rejected;
            set_error("nn_serve_submit: queue full");
            return NN_ERR_BUSY;
        }
        r->id = sv->next_id++;
        sv->table[r->id] = r;
        sv->queue.push_back(r);
        ++sv->submitted;
        if (!sv->have_first) {
            sv->first_submit = r->t_submit;
            sv->have_first = true;
        }
    }
    sv->cv_sched.notify_all();
    *request_id = r->id;
    return NN_OK;
}

nn_status nn_serve_poll(nn_server *h, uint64_t id, double *c_out, nn_solve_info *info) {
    clear_error();
    if (!h) {
        set_error("nn_serve_poll: NULL server");
        return NN_ERR_INVALID_ARG;
    }
    Server *sv = &h->s;
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->table.find(id);
        if (it == sv->table.end()) {
            set_error("nn_serve_poll: unknown request %llu", (unsigned long long)id);
            return NN_ERR_INVALID_ARG;
        }
        r = it->second;
        if (!r->done) return NN_ERR_BUSY;
        sv->table.erase(it);
    }
    if (info) *info = r->info;
    if (r->status != NN_OK && r->status != NN_ERR_NOT_CONVERGED) {
        set_error("request %llu failed with status %d: %s", (unsigned long long)id, (int)r->status,
                  r->error.c_str());
        return r->status;
    }
    if (c_out) std::memcpy(c_out, r->result.data(), sizeof(double) * r->N);
    return r->status;
}

nn_status nn_serve_drain(nn_server *h) {
    if (!h) return NN_ERR_INVALID_ARG;
    Server *sv = &h->s;
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_done.wait(lk, [&] { return sv->completed + sv->failed >= sv->submitted; });
    return NN_OK;
}

nn_status nn_serve_stats(nn_server *h, nn_serve_stats_t *st) {
    if (!h || !st) return NN_ERR_INVALID_ARG;
    Server *sv = &h->s;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = sv->submitted;
    st->completed = sv->completed;
    st->failed = sv->failed;
    st->rejected = sv->rejected;
    st->bytes_resident = sv->reserved;
    // largest sum of measured bytes over requests that held device memory at
    // the same time (a sweep over their [start, done] intervals)
    {
        std::vector<std::pair<Clock::time_point, int64_t>> ev;
        ev.reserve(sv->held.size() * 2);
        for (const auto &h : sv->held) {
            ev.push_back({h.t0, (int64_t)h.bytes});
            ev.push_back({h.t1, -(int64_t)h.bytes});
        }
        std::sort(ev.begin(), ev.end(), [](const auto &a, const auto &b) {
            return a.first < b.first || (a.first == b.first && a.second < b.second);
        });
        int64_t cur = 0, best = 0;
        for (const auto &e : ev) {
            cur += e.second;
            best = std::max(best, cur);
        }
        st->bytes_peak = (size_t)best;
    }
    st->budget = sv->budget;
    st->inflight_peak = sv->inflight_peak;
    st->bytes_reserved_peak = sv->reserved_peak;
    st->estimate_overruns = sv->overruns;
    st->estimate_max_ratio = sv->worst_ratio;
    st->queued = (int64_t)sv->queue.size();
    st->inflight = sv->inflight;
    if (!sv->lat_ms.empty()) {
        std::vector<double> v = sv->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const double pos = q * (v.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - i;
            return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        double s = 0;
        for (double x : v) s += x;
        st->mean_ms = s / v.size();
        const double span = std::chrono::duration<double>(sv->last_done - sv->first_submit).count();
        st->solves_per_s = span > 0 ? sv->completed / span : 0.0;
    }
    return NN_OK;
}

void nn_serve_destroy(nn_server *h) {
    if (!h) return;
    Server *sv = &h->s;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_sched.notify_all();
    if (sv->sched.joinable()) sv->sched.join();
    for (auto &t : sv->workers)
        if (t.joinable()) t.join();
    delete h;
}

}  // extern "C"
