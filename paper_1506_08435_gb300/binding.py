"""Thin ctypes binding of libnnqp (include/nnqp.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all
computation happens in the library's CUDA kernels.  Arrays may be numpy
arrays (host memory) or torch tensors (device or host memory); device
tensors are passed as raw device pointers together with the current torch
CUDA stream.  There is no CPU fallback: loading fails loudly if the library
has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, byref, c_double, c_int, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

from . import build as _build

NN_OK = 0
NN_ERR_INVALID_ARG = 1
NN_ERR_INFEASIBLE = 2
NN_ERR_NOT_SPD = 3
NN_ERR_OOM = 4
NN_ERR_NOT_CONVERGED = 5
NN_ERR_NUMERIC = 6
NN_ERR_TIMEOUT = 7
NN_ERR_CUDA = 8
NN_ERR_BUSY = 9
NN_ERR_DEGENERATE = 10
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "INFEASIBLE", 3: "NOT_SPD", 4: "OOM", 5: "NOT_CONVERGED",
                6: "NUMERIC", 7: "TIMEOUT", 8: "CUDA", 9: "BUSY", 10: "DEGENERATE"}

NN_MEM_HOST, NN_MEM_DEVICE = 0, 1
NN_COEF_TENSOR, NN_COEF_VELOCITY = 0, 1
NN_SOLVER_GPCG, NN_SOLVER_LBFGS, NN_SOLVER_TRON = 0, 1, 2
NN_PREC_FP64, NN_PREC_MIXED, NN_PREC_AUTO = 0, 1, 2
NN_FMT_SELL, NN_FMT_CSR = 0, 1
NN_PC_JACOBI, NN_PC_SSOR = 0, 1

COPY = dict(K_rowptr=0, K_col=1, K_val=2, M_val=3, F=4, free_node=5, A_rowptr=6, A_col=7, A_val=8, b0=9,
            coords=10, conn=11, ssor_color=12)


class NnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class nn_problem(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n_nodes", c_int64), ("n_elems", c_int64), ("coords", c_void_p),
                ("conn", c_void_p), ("nx", c_int), ("ny", c_int), ("nz", c_int), ("coef_kind", c_int),
                ("coef", c_void_p), ("alpha_L", c_double), ("alpha_T", c_double), ("D_M", c_double),
                ("f_elem", c_void_p), ("dirichlet_mask", c_void_p), ("dirichlet_value", c_void_p),
                ("lo", c_double), ("hi", c_double), ("dt", c_double), ("memory", c_int)]


class nn_assemble_opts(ctypes.Structure):
    _fields_ = [("build_csr", c_int), ("build_mixed", c_int), ("keep_full", c_int), ("lumped_mass", c_int)]


class nn_system_desc(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n_nodes", c_int64), ("n_elems", c_int64), ("n_free", c_int64),
                ("nnz_full", c_int64), ("nnz_free", c_int64), ("sell_slices", c_int64), ("sell_stored", c_int64),
                ("lo", c_double), ("hi", c_double), ("dt", c_double), ("device_bytes", c_size_t),
                ("ssor_colors", c_int)]


class nn_solve_opts(ctypes.Structure):
    _fields_ = [("solver", c_int), ("precision", c_int), ("format", c_int), ("rtol", c_double),
                ("max_iter", c_int64), ("lbfgs_m", c_int), ("grid_blocks", c_int), ("wait_timeout_s", c_double),
                ("inner_rtol", c_double), ("extrapolate", c_int), ("ksp_rtol", c_double), ("precond", c_int),
                ("ssor_omega", c_double)]


class nn_solve_info(ctypes.Structure):
    _fields_ = [("status", c_int), ("iterations", c_int64), ("spmv", c_int64), ("spmv64", c_int64),
                ("cg_iters", c_int64), ("refinements", c_int64), ("kkt_rel", c_double), ("kkt_inf", c_double),
                ("objective", c_double), ("time_ms", c_double), ("bytes_algo", c_double),
                ("active_lo", c_int64), ("active_hi", c_int64), ("fp64_fallback", c_int64),
                ("flops64_algo", c_double), ("flops_algo", c_double), ("pc_applies", c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class nn_serve_opts(ctypes.Structure):
    _fields_ = [("max_inflight", c_int), ("queue_capacity", c_int), ("sm_share_blocks", c_int),
                ("solve", nn_solve_opts)]


class nn_shard_desc(ctypes.Structure):
    _fields_ = [("rank", c_int), ("nranks", c_int), ("n", c_int64), ("row0", c_int64), ("row1", c_int64),
                ("n_halo", c_int64), ("nnz", c_int64), ("n_send", c_int64)]


class nn_serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64), ("rejected", c_int64),
                ("p50_ms", c_double), ("p99_ms", c_double), ("mean_ms", c_double), ("solves_per_s", c_double),
                ("bytes_resident", c_size_t), ("bytes_peak", c_size_t), ("budget", c_size_t),
                ("inflight_peak", c_int64), ("bytes_reserved_peak", c_size_t), ("estimate_overruns", c_int64),
                ("estimate_max_ratio", c_double), ("queued", c_int64), ("inflight", c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["nn_last_error", "nn_version", "nn_kernel_launches", "nn_device_allocations", "nn_mesh_counts", "nn_mesh_structured", "nn_assemble_opts_default",
           "nn_assemble", "nn_system_destroy", "nn_system_describe", "nn_system_copy_out",
           "nn_solve_opts_default", "nn_qp_solve", "nn_step", "nn_transient", "nn_kkt_residual", "nn_spmv",
           "nn_spmv_mixed_noalloc",
           "nn_batch_solve", "nn_batch_autotune", "nn_serve_opts_default", "nn_serve_create",
           "nn_serve_submit", "nn_serve_poll", "nn_serve_drain", "nn_serve_stats", "nn_serve_destroy",
           "nn_plan_create", "nn_plan_launch", "nn_plan_result", "nn_plan_destroy",
           "nn_shard_plan", "nn_shard_build", "nn_shard_spmv",
           "nn_color_dsatur", "nn_precond_setup", "nn_precond_apply"]

_lib = None


def library_path():
    return _build.OUT


def lib():
    """Loads libnnqp.so (building it first if sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    vp = c_void_p
    L.nn_last_error.restype = ctypes.c_char_p
    L.nn_version.restype = ctypes.c_char_p
    L.nn_kernel_launches.restype = c_uint64
    L.nn_device_allocations.restype = c_uint64
    L.nn_mesh_counts.argtypes = [c_int, c_int, c_int, c_int, POINTER(c_int64), POINTER(c_int64)]
    L.nn_mesh_structured.argtypes = [c_int, c_int, c_int, c_int, vp, vp, vp]
    L.nn_assemble_opts_default.argtypes = [POINTER(nn_assemble_opts)]
    L.nn_assemble_opts_default.restype = None
    L.nn_assemble.argtypes = [POINTER(nn_problem), POINTER(nn_assemble_opts), vp, POINTER(vp)]
    L.nn_system_destroy.argtypes = [vp]
    L.nn_system_destroy.restype = None
    L.nn_system_describe.argtypes = [vp, POINTER(nn_system_desc)]
    L.nn_system_copy_out.argtypes = [vp, c_int, vp, c_size_t, c_int, vp]
    L.nn_solve_opts_default.argtypes = [POINTER(nn_solve_opts)]
    L.nn_solve_opts_default.restype = None
    L.nn_qp_solve.argtypes = [vp, POINTER(nn_solve_opts), vp, c_int, vp, POINTER(nn_solve_info)]
    L.nn_step.argtypes = [vp, vp, vp, c_int, POINTER(nn_solve_opts), vp, POINTER(nn_solve_info)]
    L.nn_transient.argtypes = [vp, vp, c_int, vp, vp, c_int, POINTER(nn_solve_opts), vp, POINTER(nn_solve_info)]
    L.nn_plan_create.argtypes = [vp, POINTER(nn_solve_opts), c_int, vp, POINTER(vp)]
    L.nn_plan_launch.argtypes = [vp, vp, vp, vp, vp]
    L.nn_plan_result.argtypes = [vp, vp, POINTER(nn_solve_info), c_int]
    L.nn_plan_destroy.argtypes = [vp]
    L.nn_plan_destroy.restype = None
    L.nn_kkt_residual.argtypes = [vp, vp, vp, c_int, POINTER(c_double), vp]
    L.nn_spmv.argtypes = [vp, vp, vp, c_int, c_int, vp]
    L.nn_spmv_mixed_noalloc.argtypes = [vp, vp, vp, vp]
    L.nn_batch_solve.argtypes = [c_int, POINTER(vp), POINTER(vp), POINTER(nn_solve_opts), vp,
                                 POINTER(nn_solve_info)]
    L.nn_batch_autotune.argtypes = [c_int, POINTER(vp), POINTER(nn_solve_opts), vp, POINTER(c_int)]
    L.nn_serve_opts_default.argtypes = [POINTER(nn_serve_opts)]
    L.nn_serve_opts_default.restype = None
    L.nn_serve_create.argtypes = [c_size_t, POINTER(nn_serve_opts), POINTER(vp)]
    L.nn_serve_submit.argtypes = [vp, POINTER(nn_problem), POINTER(nn_solve_opts), POINTER(c_uint64)]
    L.nn_serve_poll.argtypes = [vp, c_uint64, vp, POINTER(nn_solve_info)]
    L.nn_serve_drain.argtypes = [vp]
    L.nn_serve_stats.argtypes = [vp, POINTER(nn_serve_stats_t)]
    L.nn_serve_destroy.argtypes = [vp]
    L.nn_serve_destroy.restype = None
    L.nn_shard_plan.argtypes = [c_int64, vp, vp, c_int, c_int, POINTER(nn_shard_desc)]
    L.nn_shard_build.argtypes = [c_int64, vp, vp, c_int, c_int, vp, vp, vp, vp, vp, vp]
    L.nn_shard_spmv.argtypes = [c_int64, vp, vp, vp, vp, vp, vp]
    L.nn_color_dsatur.argtypes = [c_int64, vp, vp, vp, POINTER(c_int)]
    L.nn_precond_setup.argtypes = [vp, vp]
    L.nn_precond_apply.argtypes = [vp, c_int, c_double, vp, vp, vp, vp]
    _lib = L
    return L


def last_error():
    return lib().nn_last_error().decode()


def _check(st, allow=()):
    if st != NN_OK and st not in allow:
        raise NnError(st, last_error())
    return st


# ---------------------------------------------------------------- marshalling helpers

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, memory flag) of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (NN_MEM_DEVICE if a.is_cuda else NN_MEM_HOST)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, NN_MEM_HOST


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch is optional for host-only calls
        pass
    return None


def solve_opts(**kw):
    o = nn_solve_opts()
    lib().nn_solve_opts_default(byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def assemble_opts(**kw):
    o = nn_assemble_opts()
    lib().nn_assemble_opts_default(byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Problem:
    """Owns the arrays behind an nn_problem for the duration of a call."""

    def __init__(self, spec, device=None):
        """spec: an nn_inputs.ProblemSpec (or any object with its fields).
        device: None -> numpy host arrays; a torch device -> tensors there."""
        if device is not None:
            import torch

            def conv(a, dt):
                return None if a is None else torch.as_tensor(np.ascontiguousarray(a, dt), device=device)
        else:
            def conv(a, dt):
                return None if a is None else np.ascontiguousarray(a, dt)
        self.coef = conv(spec.coef, np.float64)
        self.f_elem = conv(spec.f_elem, np.float64)
        self.dmask = conv(spec.dmask, np.uint8)
        self.dval = conv(spec.dval, np.float64)
        self.coords = conv(getattr(spec, "coords", None), np.float64)
        self.conn = conv(getattr(spec, "conn", None), np.int32)
        p = nn_problem()
        p.dim = spec.dim
        p.nx, p.ny, p.nz = spec.nx, spec.ny, spec.nz
        p.coef_kind = spec.coef_kind
        p.alpha_L, p.alpha_T, p.D_M = spec.aL, spec.aT, spec.DM
        p.lo, p.hi, p.dt = spec.lo, spec.hi, spec.dt
        p.coef, mem = _ptr(self.coef)
        p.f_elem = _ptr(self.f_elem)[0]
        p.dirichlet_mask = _ptr(self.dmask)[0]
        p.dirichlet_value = _ptr(self.dval)[0]
        if self.coords is not None:
            p.coords = _ptr(self.coords)[0]
            p.conn = _ptr(self.conn)[0]
            p.n_nodes = self.coords.shape[0]
            p.n_elems = self.conn.shape[0]
        p.memory = mem
        self.c = p


class System:
    """Owning wrapper of an nn_system* (destroyed with the object)."""

    def __init__(self, handle):
        self.handle = c_void_p(handle)

    def __del__(self):
        if getattr(self, "handle", None) is not None and self.handle.value and _lib is not None:
            _lib.nn_system_destroy(self.handle)
            self.handle = None

    def describe(self):
        return nn_system_describe(self)


# ---------------------------------------------------------------- entry points

def nn_version():
    return lib().nn_version().decode()


def nn_kernel_launches():
    return int(lib().nn_kernel_launches())


kernel_launches = nn_kernel_launches


def nn_device_allocations():
    return int(lib().nn_device_allocations())


def nn_mesh_counts(dim, nx, ny, nz=0):
    N, E = c_int64(), c_int64()
    _check(lib().nn_mesh_counts(dim, nx, ny, nz, byref(N), byref(E)))
    return N.value, E.value


def nn_mesh_structured(dim, nx, ny, nz, coords, conn, stream=None):
    _check(lib().nn_mesh_structured(dim, nx, ny, nz, _ptr(coords)[0], _ptr(conn)[0], _stream(stream)))


def nn_assemble(problem, opts=None, stream=None):
    if not isinstance(problem, Problem):
        problem = Problem(problem)
    h = c_void_p()
    o = opts if opts is not None else assemble_opts()
    _check(lib().nn_assemble(byref(problem.c), byref(o), _stream(stream), byref(h)))
    return System(h.value)


def nn_system_describe(sys):
    d = nn_system_desc()
    _check(lib().nn_system_describe(sys.handle, byref(d)))
    return {k: getattr(d, k) for k, _ in d._fields_}


def nn_system_copy_out(sys, what, dst, stream=None):
    ptr, mem = _ptr(dst)
    nbytes = dst.nbytes if not _is_torch(dst) else dst.numel() * dst.element_size()
    _check(lib().nn_system_copy_out(sys.handle, COPY.get(what, what), ptr, nbytes, mem, _stream(stream)))
    return dst


def _info(st, info):
    d = info.as_dict()
    d["status_name"] = STATUS_NAMES.get(d["status"], d["status"])
    return d


def nn_qp_solve(sys, c, opts=None, stream=None, allow=(NN_ERR_NOT_CONVERGED,)):
    info = nn_solve_info()
    ptr, mem = _ptr(c)
    o = opts if opts is not None else solve_opts()
    st = lib().nn_qp_solve(sys.handle, byref(o), ptr, mem, _stream(stream), byref(info))
    _check(st, allow)
    return _info(st, info)


def nn_step(sys, c_prev, c_next, opts=None, stream=None, allow=(NN_ERR_NOT_CONVERGED,)):
    info = nn_solve_info()
    p0, mem = _ptr(c_prev)
    p1, _ = _ptr(c_next)
    o = opts if opts is not None else solve_opts()
    st = lib().nn_step(sys.handle, p0, p1, mem, byref(o), _stream(stream), byref(info))
    _check(st, allow)
    return _info(st, info)


def nn_transient(sys, c0, nsteps, c_final, c_hist=None, opts=None, stream=None, allow=(NN_ERR_NOT_CONVERGED,)):
    infos = (nn_solve_info * nsteps)()
    p0, mem = _ptr(c0)
    o = opts if opts is not None else solve_opts()
    st = lib().nn_transient(sys.handle, p0, nsteps, _ptr(c_final)[0], _ptr(c_hist)[0] if c_hist is not None else None,
                            mem, byref(o), _stream(stream), infos)
    _check(st, allow)
    return [_info(st, i) for i in infos]


def nn_kkt_residual(sys, c, c_prev=None, stream=None):
    out = (c_double * 4)()
    p, mem = _ptr(c)
    pp = _ptr(c_prev)[0] if c_prev is not None else None
    _check(lib().nn_kkt_residual(sys.handle, p, pp, mem, out, _stream(stream)))
    return dict(kkt_rel=out[0], kkt_inf=out[1], bounds_ok=bool(out[2]), obj=out[3])


def nn_spmv(sys, x, y, format=NN_FMT_SELL, precision=NN_PREC_FP64, stream=None):
    _check(lib().nn_spmv(sys.handle, _ptr(x)[0], _ptr(y)[0], format, precision, _stream(stream)))
    return y


def nn_spmv_mixed_noalloc(sys, x, y, stream=None):
    """y = A x (FP32-value operator) using the library's fixed scratch array
    instead of a per-call allocation (see include/nnqp.h)."""
    _check(lib().nn_spmv_mixed_noalloc(sys.handle, _ptr(x)[0], _ptr(y)[0], _stream(stream)))
    return y


def nn_batch_solve(systems, cs, opts=None, stream=None, allow=(NN_ERR_NOT_CONVERGED,)):
    n = len(systems)
    hs = (c_void_p * n)(*[s.handle.value for s in systems])
    ps = (c_void_p * n)(*[_ptr(c)[0] for c in cs])
    infos = (nn_solve_info * n)()
    o = opts if opts is not None else solve_opts()
    st = lib().nn_batch_solve(n, hs, ps, byref(o), _stream(stream), infos)
    _check(st, allow)
    return [_info(st, i) for i in infos]


def nn_batch_autotune(systems, opts=None, stream=None):
    n = len(systems)
    hs = (c_void_p * n)(*[s.handle.value for s in systems])
    best = c_int()
    o = opts if opts is not None else solve_opts()
    _check(lib().nn_batch_autotune(n, hs, byref(o), _stream(stream), byref(best)))
    return best.value


class Plan:
    """A reusable solve of one system (nn_plan_*): launches enqueue work on a
    stream without allocating or synchronising (capturable in CUDA graphs)."""

    def __init__(self, sys, opts=None, nsteps=1, stream=None):
        self.sys = sys
        self.nsteps = nsteps
        h = c_void_p()
        o = opts if opts is not None else solve_opts()
        _check(lib().nn_plan_create(sys.handle, byref(o), nsteps, _stream(stream), byref(h)))
        self.handle = h

    def launch(self, c_in, c_out, c_hist=None, stream=None):
        _check(lib().nn_plan_launch(self.handle, _ptr(c_in)[0], _ptr(c_out)[0],
                                    _ptr(c_hist)[0] if c_hist is not None else None, _stream(stream)))

    def result(self, stream=None, allow=(NN_ERR_NOT_CONVERGED,)):
        infos = (nn_solve_info * self.nsteps)()
        st = lib().nn_plan_result(self.handle, _stream(stream), infos, self.nsteps)
        _check(st, allow)
        return [_info(st, i) for i in infos]

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().nn_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


def serve_opts(**kw):
    o = nn_serve_opts()
    lib().nn_serve_opts_default(byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Server:
    def __init__(self, handle):
        self.handle = c_void_p(handle)

    def __del__(self):
        if getattr(self, "handle", None) is not None and self.handle.value and _lib is not None:
            _lib.nn_serve_destroy(self.handle)
            self.handle = None


def nn_serve_create(budget_bytes, opts=None):
    h = c_void_p()
    o = opts if opts is not None else serve_opts()
    _check(lib().nn_serve_create(budget_bytes, byref(o), byref(h)))
    return Server(h.value)


def nn_serve_submit(server, problem, opts=None):
    """opts: this request's nn_solve_opts (None = the server's)."""
    if not isinstance(problem, Problem):
        problem = Problem(problem)
    rid = c_uint64()
    st = lib().nn_serve_submit(server.handle, byref(problem.c), byref(opts) if opts is not None else None,
                               byref(rid))
    _check(st)
    return rid.value


def nn_serve_poll(server, rid, c_out):
    info = nn_solve_info()
    st = lib().nn_serve_poll(server.handle, rid, _ptr(c_out)[0], byref(info))
    if st == NN_ERR_BUSY:
        return None
    _check(st, (NN_ERR_NOT_CONVERGED,))
    return _info(st, info)


def nn_serve_drain(server):
    _check(lib().nn_serve_drain(server.handle))


def nn_serve_stats(server):
    s = nn_serve_stats_t()
    _check(lib().nn_serve_stats(server.handle, byref(s)))
    return s.as_dict()


def nn_serve_destroy(server):
    if server.handle is not None and server.handle.value:
        lib().nn_serve_destroy(server.handle)
        server.handle = None


# ---------------------------------------------------------------- row sharding

def nn_shard_plan(rowptr, col, nranks, rank):
    """Shard sizes of rank `rank` for the CSR pattern (numpy int64 rowptr,
    int32 col, host)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    d = nn_shard_desc()
    _check(lib().nn_shard_plan(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, nranks, rank, byref(d)))
    return {k: getattr(d, k) for k, _ in d._fields_}


def nn_shard_build(rowptr, col, nranks, rank):
    """The shard's local CSR pattern, ghosts and send list (numpy arrays)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    d = nn_shard_plan(rowptr, col, nranks, rank)
    nrows = d["row1"] - d["row0"]
    out = dict(local_rowptr=np.zeros(nrows + 1, np.int64), local_col=np.zeros(max(d["nnz"], 1), np.int32),
               halo_ids=np.zeros(max(d["n_halo"], 1), np.int64), halo_owner=np.zeros(max(d["n_halo"], 1), np.int32),
               send_ids=np.zeros(max(d["n_send"], 1), np.int64), send_rank=np.zeros(max(d["n_send"], 1), np.int32))
    _check(lib().nn_shard_build(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, nranks, rank,
                                *[out[k].ctypes.data for k in ("local_rowptr", "local_col", "halo_ids", "halo_owner",
                                                               "send_ids", "send_rank")]))
    out["local_col"] = out["local_col"][:d["nnz"]]
    for k, m in (("halo_ids", "n_halo"), ("halo_owner", "n_halo"), ("send_ids", "n_send"), ("send_rank", "n_send")):
        out[k] = out[k][:d[m]]
    out.update(d)
    return out


def nn_shard_spmv(nrows, local_rowptr, local_col, val, x_ext, y, stream=None):
    """y = A_local x_ext on the device (torch tensors on the GPU)."""
    _check(lib().nn_shard_spmv(nrows, _ptr(local_rowptr)[0], _ptr(local_col)[0], _ptr(val)[0], _ptr(x_ext)[0],
                               _ptr(y)[0], _stream(stream)))
    return y


# ---------------------------------------------------------------- SSOR preconditioning

def nn_color_dsatur(rowptr, col):
    """DSatur colouring of the graph of a symmetric CSR pattern (numpy int64
    rowptr, int32 col, host): (colour int32 [n], number of colours)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    n = len(rowptr) - 1
    color = np.zeros(max(n, 1), np.int32)
    k = c_int()
    _check(lib().nn_color_dsatur(n, rowptr.ctypes.data, col.ctypes.data, color.ctypes.data, byref(k)))
    return color[:n], k.value


def nn_precond_setup(sys, stream=None):
    _check(lib().nn_precond_setup(sys.handle, _stream(stream)))


def nn_precond_apply(sys, r, z, precond=NN_PC_SSOR, omega=1.0, face=None, stream=None):
    """z = P r on the device (torch tensors): the solve kernels' Jacobi or
    multicolour SSOR preconditioner on the face (uint8 tensor or None)."""
    _check(lib().nn_precond_apply(sys.handle, precond, omega, _ptr(face)[0] if face is not None else None,
                                  _ptr(r)[0], _ptr(z)[0], _stream(stream)))
    return z
