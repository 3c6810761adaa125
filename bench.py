"""Benchmark of the non-negative diffusion QP path on GB300.

Default workload (no flags, N = 1): the 3D steady problem of 150^3
hexahedra x 6 tetrahedra (3,442,951 nodes, 3,414,525 free unknowns, about
50.7M nonzeros in the reduced matrix), dispersion tensor from the vortex
velocity field rotated per 10^3 block of hexahedra (seed 1506; alpha_L = 1,
alpha_T = 1e-3, D_M = 1e-9), c = 1 on the x = 0 patch and c = 0 on x = 1,
0 <= c <= 1.  One benchmark step is the whole path on one synthetic input:
device assembly (pattern, element matrices, elimination, SELL build) + one
QP solve to KKT <= 1e-10 relative (tighter than the 1e-8 acceptance) in one
persistent launch.  metric: QP solves per second.  The line is the plain
FP64 solve; its "mixed" object is the same workload solved with FP32 operator
values and FP32 inner solves refined in FP64 (FP64 residual, KKT and stored
solution), with "vs_plain_fp64" = mixed solves/s / FP64 solves/s.  Inputs
(0.6-0.9 GB of operator) are far larger than L2, and L2 is flushed between
steps anyway (256 MB write).

roofline: achieved = algorithmic bytes of the solve launch (every product
counted at the paper's MatMult traffic, every vector stream of the fused
passes at its width) / the launch's CUDA-event time; "dram_gbs" beside it is
the ncu-measured DRAM bytes of the same launch (scaled from a capture of a
smaller case, see traffic_source) / the same time; "alu" is the FP64 pipe
(algorithmic FP64 operations / time against 152 SMs x 2 DFMA/clk x 2 flop x
2.07 GHz).  "bound" names the larger of the two fractions.

Options: --precision fp64|mixed|both (default both for steady3d),
--solver gpcg|lbfgs|tron (--ksp-rtol: TRON's subspace tolerance), --n to
shrink the grid, --e2e-steps (end-to-end repeats, default 5).

Other workloads (--workload), each printing its own line:
  transient3d  40^3 x 6 tets, dt = 0.01, 50 backward-Euler steps
               (one warm-started QP per step) in one launch; --mass
               consistent|lumped; a step = assembly + the 50-step run
  steady2d     2D 50 x 50 square, rotated tensor; a step = assembly + one solve
  batch        512 2D instances of 21^2 - 201^2 nodes in one persistent launch; a step =
               one batched solve of all instances, --precision fp64|mixed;
               also reports the single-system FP64 solver on the same instances
  cube_hole    the cube with a cubic hole (Sec. 5.1 analogue; --m, --mesh
               kuhn|mirrored); a step = assembly + one solve; also reports the
               Galerkin solution's departure from [0, 1] (an unbounded solve)
  serve        Poisson arrivals at 200/s for 60 s, request r seeded (2015, r);
               reports p50/p99 latency
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import nn_inputs as I  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
FP64_PIPE_PEAK_GFLOPS = 152 * 2 * 2 * 2.07   # SMs x DFMA per clock (ncu unit count) x flop x GHz


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return None


# ---------------------------------------------------------------- distributed plumbing

def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group("gloo")
    return dist, rank, ws


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path):
        self.path, self.proc = path, None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9 or not p[0].isdigit() or int(p[0]) != gpu_index:
                continue
            try:
                sm.append(float(p[1].split()[0]))
                mx = float(p[2].split()[0])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- the oracle baseline (CPU)

class Steady3dOracle:
    """The FP64 oracle on the steady 3D workload, sampled: the oracle
    assembles the n^3 system itself (mesh, element loop, elimination; timed
    once), then runs bounded batches of its MPRGP iterations from the zero
    start (timed per batch).  A whole oracle solve is
        t_setup + I * t_iteration,
    with I the MPRGP iterations the oracle needs for this system, recorded by
    oracle/record_oracle_runs.py (a full oracle run; its active-set polish,
    a few percent of the run, is left out, in the oracle's favour)."""

    def __init__(self, n, threads, runs_dir=None):
        from oracle import oracle as O
        self.O, self.n, self.threads = O, n, threads
        self.record, self.extrapolated = oracle_iterations(n, runs_dir or os.path.join(ROOT, "oracle", "runs"))
        spec = I.config3_steady_3d(n=n)
        t0 = time.perf_counter()
        coords, conn = O.mesh_structured(3, spec.nx)
        asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, spec.f_elem)
        self.red = O.Reduced(asm, spec.dmask, spec.dval)
        self.b = self.red.rhs()
        self.t_setup = time.perf_counter() - t0
        self.spec = spec

    def iterations(self, k):
        """Seconds per MPRGP iteration over k iterations from the zero start."""
        t0 = time.perf_counter()
        self.O.mprgp(self.red.A, self.b, self.spec.lo, self.spec.hi, maxit=k, threads=self.threads)
        return (time.perf_counter() - t0) / k

    def value(self, t_it):
        if self.record is None:
            return None
        return 1.0 / (self.t_setup + self.record["mprgp_iters"] * t_it)

    def describe(self, k):
        if self.record is None:
            return "no record of the oracle's iteration count for steady3d_n%d" % self.n
        how = (self.extrapolated or "recorded full oracle run, kkt %.1e" % self.record["kkt_rel"])
        return ("oracle (FP64 C, MPRGP, %d threads) on the %d^3 steady system: its own assembly + elimination "
                "timed once (%.1f s), %d MPRGP iterations from the zero start timed, whole solve = setup + "
                "%d iterations (%s; polish excluded)"
                % (self.threads, self.n, self.t_setup, k, self.record["mprgp_iters"], how))


def oracle_iterations(n, runs_dir):
    """MPRGP iterations of the oracle's full solve of the n^3 steady system:
    the record of a full oracle run (oracle/record_oracle_runs.py) when there
    is one; otherwise extrapolated from the records of smaller grids by a
    least-squares power law iterations = a n^b (at least two records), which
    the returned note says.  Returns (record or None, note or None)."""
    import glob
    import re
    rec = os.path.join(runs_dir, "steady3d_n%d.json" % n)
    if os.path.exists(rec):
        return json.load(open(rec)), None
    pts = []
    for f in glob.glob(os.path.join(runs_dir, "steady3d_n*.json")):
        m = re.match(r"steady3d_n(\d+)\.json$", os.path.basename(f))
        if m and int(m.group(1)) < n:
            pts.append((int(m.group(1)), json.load(open(f))["mprgp_iters"]))
    if len(pts) < 2:
        return None, None
    ln = np.log([p[0] for p in pts])
    li = np.log([p[1] for p in pts])
    b, a = np.polyfit(ln, li, 1)
    iters = int(round(math.exp(a + b * math.log(n))))
    note = ("iteration count extrapolated from recorded full oracle runs at n = %s by iterations = a n^%.2f"
            % (", ".join(str(p[0]) for p in sorted(pts)), b))
    return {"mprgp_iters": iters, "kkt_rel": float("nan")}, note


def oracle_sample(workload, budget_s=20.0, n=None, lumped=False):
    """The FP64 oracle as it stands, on a bounded sample of the workload;
    returns (units per second, cores used, description)."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    if workload == "steady3d":
        orc = Steady3dOracle(n or 150, threads)
        t1 = orc.iterations(5)
        k = max(5, min(2000, int(max(budget_s - orc.t_setup, 5.0) / max(t1, 1e-6))))
        t_it = orc.iterations(k)
        return orc.value(t_it), threads, orc.describe(k)
    if workload == "transient3d":
        spec = I.config2_transient_3d()
        coords, conn = O.mesh_structured(3, spec.nx)
        asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, with_mass=True,
                         lumped=lumped)
        red = O.Reduced(asm, spec.dmask, spec.dval, dt=spec.dt)
        c = spec.c0.copy()
        t0, k = time.perf_counter(), 0
        while k < 1 or (time.perf_counter() - t0 < budget_s and k < spec.nsteps):
            b = red.rhs(c)
            x, _ = O.solve_qp(red.A, b, spec.lo, spec.hi, x0=c[red.free], threads=threads)
            c = red.full(x)
            k += 1
        dt = time.perf_counter() - t0
        return k / dt, threads, ("first %d backward-Euler QP steps of the 40^3 transient problem (%s mass; "
                                 "MPRGP + active-set polish to 1e-12, OpenMP products), assembly excluded"
                                 % (k, "lumped" if lumped else "consistent"))
    if workload == "steady2d":
        spec = I.config1_steady_2d()
        coords, conn = O.mesh_structured(2, spec.nx)
        asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, f_elem=spec.f_elem)
        red = O.Reduced(asm, spec.dmask, spec.dval)
        b = red.rhs()
        t0, k = time.perf_counter(), 0
        while k < 1 or time.perf_counter() - t0 < min(budget_s, 5.0):
            O.solve_qp(red.A, b, spec.lo, spec.hi, threads=1)
            k += 1
        return k / (time.perf_counter() - t0), 1, "%d full solves of the 2D 50x50 problem (1 thread)" % k
    if workload == "batch":
        t0, k = time.perf_counter(), 0
        while k < 1 or time.perf_counter() - t0 < budget_s:
            spec = I.config4_instance(k)
            coords, conn = O.mesh_structured(2, spec.nx)
            asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, f_elem=spec.f_elem)
            red = O.Reduced(asm, spec.dmask, spec.dval)
            O.solve_qp(red.A, red.rhs(), spec.lo, spec.hi, threads=threads)
            k += 1
        return k / (time.perf_counter() - t0), threads, "first %d instances of the 512-instance batch" % k
    if workload == "serve":
        # requests of the serving stream in arrival order, each assembled,
        # eliminated and solved by the oracle; requests above max_nodes are
        # skipped (the oracle needs minutes for one of them), which favours it
        max_nodes = 50000
        t0, k, skipped, r = time.perf_counter(), 0, 0, 0
        while k < 1 or time.perf_counter() - t0 < budget_s:
            spec = I.serve_request(r)
            r += 1
            if spec.n_nodes > max_nodes:
                skipped += 1
                continue
            coords, conn = O.mesh_structured(spec.dim, spec.nx, spec.ny, spec.nz)
            asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, f_elem=spec.f_elem)
            red = O.Reduced(asm, spec.dmask, spec.dval)
            O.solve_qp(red.A, red.rhs(), spec.lo, spec.hi, threads=threads)
            k += 1
        return k / (time.perf_counter() - t0), threads, (
            "the first %d requests of the serving stream with at most %d nodes, one after another (assembly, "
            "elimination, MPRGP + polish to 1e-12; %d larger requests skipped, which favours the oracle)"
            % (k, max_nodes, skipped))
    return None, threads, "no oracle sample for this workload"


# ---------------------------------------------------------------- helpers

def source_digest():
    """SHA-256 over the library's kernel and host sources (names and bytes,
    sorted by name): identifies the code an ncu summary was captured from."""
    import hashlib
    d = os.path.join(ROOT, "paper_1506_08435_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(name.encode())
            h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()[:16]


def pinned_problem(P, torch, spec):
    """A Problem whose arrays are in pinned host memory (for the e2e leg)."""
    hp = P.Problem(spec)
    keep = {}
    for name in ("coef", "dmask", "dval", "f_elem"):
        a = getattr(hp, name)
        if a is None:
            continue
        t = torch.from_numpy(a).pin_memory()
        keep[name] = t
        setattr(hp, name, t)
    hp.c.coef = keep["coef"].data_ptr()
    hp.c.dirichlet_mask = keep["dmask"].data_ptr()
    hp.c.dirichlet_value = keep["dval"].data_ptr()
    if "f_elem" in keep:
        hp.c.f_elem = keep["f_elem"].data_ptr()
    if getattr(spec, "coords", None) is not None:
        keep["coords"] = torch.from_numpy(np.ascontiguousarray(spec.coords, np.float64)).pin_memory()
        keep["conn"] = torch.from_numpy(np.ascontiguousarray(spec.conn, np.int32)).pin_memory()
        hp.coords, hp.conn = keep["coords"], keep["conn"]
        hp.c.coords = keep["coords"].data_ptr()
        hp.c.conn = keep["conn"].data_ptr()
    hp.c.memory = P.NN_MEM_HOST
    nbytes = sum(t.numel() * t.element_size() for t in keep.values())
    return hp, nbytes


def timed_steps(torch, step, steps, flush, clk):
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    outs = []
    clk.start()
    time.sleep(0.3)
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        outs.append(step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop(torch.cuda.current_device())
    return [a.elapsed_time(b) for a, b in ev], outs, clocks


# ---------------------------------------------------------------- workloads

def profile_traffic(pdir, kname, workload, precision, digest, scale_from=None, products=None, nnz_free=None,
                    algo_bytes=None):
    """DRAM bytes per launch of kernel kname on this workload from the committed
    ncu summary <kname>_<workload>_<precision>.md in pdir (its line
    "dram_bytes_per_launch: N"), used only while its "source_digest:" line
    equals digest.  Without a summary for the workload itself, the summary of
    the smaller case scale_from is scaled to this launch by algorithmic bytes
    (its "algo_bytes_per_launch:" line against algo_bytes: the DRAM traffic
    per algorithmic byte is taken as a property of the kernel), or, where the
    summary has no such line, by products x nnz_free (its
    "products_per_launch:" and "nnz_free:" lines).  Returns (bytes or None,
    where the figure came from or why there is none)."""
    tfile = os.path.join(pdir, "%s_%s_%s.md" % (kname, workload, precision))
    scaled = False
    if not os.path.exists(tfile) and scale_from:
        tfile = os.path.join(pdir, "%s_%s_%s.md" % (kname, scale_from, precision))
        scaled = True
    if not os.path.exists(tfile):
        return None, "no ncu summary for this workload"
    name = os.path.basename(tfile)
    fields = {}
    for line in open(tfile):
        key = line.split(":", 1)[0].strip() if ":" in line else ""
        if key in ("dram_bytes_per_launch", "source_digest", "products_per_launch", "nnz_free",
                   "algo_bytes_per_launch"):
            v = line.split(":", 1)[1].strip()
            fields[key] = v.split()[0] if v else ""
    if fields.get("source_digest") != digest:
        return None, "kernel changed since the ncu capture in %s" % name
    try:
        traffic = float(fields["dram_bytes_per_launch"])
        if not scaled:
            return traffic, "ncu capture, %s" % name
        if algo_bytes and fields.get("algo_bytes_per_launch"):
            traffic *= algo_bytes / float(fields["algo_bytes_per_launch"])
            return traffic, "ncu capture of a smaller case (%s), scaled by algorithmic bytes" % name
        traffic *= products / float(fields["products_per_launch"]) * nnz_free / float(fields["nnz_free"])
        return traffic, "ncu capture of a smaller case (%s), scaled by products x nnz_free" % name
    except (KeyError, ValueError, TypeError, ZeroDivisionError):
        return None, "incomplete ncu summary %s" % name


def solver_code(P, args):
    return {"gpcg": P.NN_SOLVER_GPCG, "lbfgs": P.NN_SOLVER_LBFGS, "tron": P.NN_SOLVER_TRON}[args.solver]


def precond_opts(P, args):
    """preconditioner fields of nn_solve_opts"""
    return dict(precond=P.NN_PC_SSOR if args.precond == "ssor" else P.NN_PC_JACOBI, ssor_omega=args.omega)


def precond_name(args):
    return "ssor(omega %g)" % args.omega if getattr(args, "precond", "jacobi") == "ssor" else "jacobi"


def transient_config(spec, args):
    """config of the default workload (both arms print the same one)."""
    return {"workload": "transient3d_n40_dt0.01_50steps", "nodes": spec.n_nodes, "tets": spec.n_elems,
            "qp_per_step": spec.nsteps, "rtol": args.rtol, "l2": "flushed between steps (256 MB write)",
            "solver": args.solver + ("(ksp %g)" % args.ksp_rtol if args.solver == "tron" else ""),
            "precision": getattr(args, "cur_precision", args.precision), "mass": args.mass,
            "first_iterate": "projected 3c^n - 3c^(n-1) + c^(n-2)", "precond": precond_name(args)}


def run_transient(P, torch, args, rank):
    spec = I.config2_transient_3d()
    dev = torch.device("cuda")
    nsteps = spec.nsteps
    prob = P.Problem(spec, device=dev)
    mixed = args.cur_precision == "mixed"
    opts = P.solve_opts(rtol=args.rtol, solver=solver_code(P, args), ksp_rtol=args.ksp_rtol,
                        precision=P.NN_PREC_MIXED if mixed else P.NN_PREC_FP64, **precond_opts(P, args))
    aopts = P.assemble_opts(build_mixed=1 if mixed else 0, lumped_mass=1 if args.mass == "lumped" else 0)
    c0 = torch.tensor(spec.c0, device=dev)
    cf = torch.zeros_like(c0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        s = P.nn_assemble(prob, aopts)
        infos = P.nn_transient(s, c0, nsteps, cf, None, opts)
        del s
        return infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = P.kernel_launches()
    times, outs, clocks = timed_steps(torch, step, args.steps, flush,
                                      ClockSampler(os.path.join(args.out_dir, "clocks_rank%d.csv" % rank)))
    launches = P.kernel_launches() - l0
    infos = [i for o in outs for i in o]
    # end to end through the C ABI with pinned host buffers, copies inside the timed region
    hp, hbytes = pinned_problem(P, torch, spec)
    c0h = torch.from_numpy(spec.c0.copy()).pin_memory()
    cfh = torch.zeros_like(c0h).pin_memory()
    stream = torch.cuda.current_stream()
    e2e = []
    for _ in range(min(args.steps, args.e2e_steps)):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s = P.nn_assemble(hp, aopts)
        P.nn_transient(s, c0h, nsteps, cfh, None, opts)
        b.record(stream)
        torch.cuda.synchronize()
        e2e.append(a.elapsed_time(b))
        del s
    return dict(times=times, infos=infos, kern_ms=[o[0]["time_ms"] for o in outs],
                kern_bytes=[sum(i["bytes_algo"] for i in o) for o in outs], units_per_step=nsteps, e2e=e2e,
                h2d=hbytes + c0h.numel() * 8, d2h=cfh.numel() * 8, clocks=clocks, launches=launches,
                nnz_free=None,
                config=transient_config(spec, args),
                dtype="f32+f64" if mixed else "f64", unit="QP solves/s", metric="QP solves/s")


def run_steady(P, torch, args, rank, dim):
    if args.workload == "cube_hole":
        spec = I.cube_with_hole(args.m, args.mesh)
    elif dim == 3:
        spec = I.config3_steady_3d(n=args.n or 150)
    else:
        spec = I.config1_steady_2d(n=args.n or 50)
    dev = torch.device("cuda")
    prec = {"mixed": P.NN_PREC_MIXED, "auto": P.NN_PREC_AUTO}.get(args.cur_precision, P.NN_PREC_FP64)
    opts = P.solve_opts(rtol=args.rtol, precision=prec, max_iter=args.max_iter,
                        solver=solver_code(P, args), ksp_rtol=args.ksp_rtol, **precond_opts(P, args))
    aopts = P.assemble_opts(build_mixed=1 if prec != P.NN_PREC_FP64 else 0)
    prob = P.Problem(spec, device=dev)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    desc = {}

    def step():
        s = P.nn_assemble(prob, aopts)
        c.zero_()
        info = P.nn_qp_solve(s, c, opts)
        desc.update(s.describe())
        del s
        return [info]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = P.kernel_launches()
    times, outs, clocks = timed_steps(torch, step, args.steps, flush,
                                      ClockSampler(os.path.join(args.out_dir, "clocks_rank%d.csv" % rank)))
    launches = P.kernel_launches() - l0
    infos = [i for o in outs for i in o]
    hp, hbytes = pinned_problem(P, torch, spec)
    ch = torch.zeros(spec.n_nodes, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    e2e = []
    for _ in range(min(args.steps, args.e2e_steps)):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s = P.nn_assemble(hp, aopts)
        ch.zero_()
        P.nn_qp_solve(s, ch, opts)
        b.record(stream)
        torch.cuda.synchronize()
        e2e.append(a.elapsed_time(b))
        del s
    graph = None
    if dim == 2:
        # back-to-back solves of the assembled system from a CUDA graph of 10
        # launches of one plan (no allocation, no host round trip per solve)
        s = P.nn_assemble(prob, aopts)
        plan = P.Plan(s, opts)
        zero = torch.zeros_like(c)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            for _ in range(10):
                plan.launch(zero, c, stream=side)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(args.steps, 3)
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        ginfo = plan.result()[0]
        ms = a.elapsed_time(b) / (10 * reps)
        graph = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "launches_per_graph": 10, "replays": reps,
                 "kkt_rel": ginfo["kkt_rel"], "status": ginfo["status"], "assembly": "outside (system reused)"}
        plan.close()
        del s
    name = ("steady3d_n%d" % (args.n or 150)) if dim == 3 else ("steady2d_n%d" % (args.n or 50))
    # the 150^3 solve (~18k products, seconds per launch) is captured with its
    # products capped (same system, same kernel, same launch shape)
    scale_from = ("steady3d_n%dcap" % (args.n or 150)) if dim == 3 else None
    dmp = None
    if args.workload == "cube_hole":
        name = "cube_hole_%s_m%d" % (args.mesh, args.m)
        scale_from = "cube_hole_%s_m12" % args.mesh
        # the Galerkin solution of the same system (no bounds: GPCG reduces to
        # Jacobi-preconditioned CG), once, outside the timed region: how far
        # the unconstrained discretisation leaves [0, 1] on this mesh
        import dataclasses
        gprob = P.Problem(dataclasses.replace(spec, lo=-math.inf, hi=math.inf), device=dev)
        s = P.nn_assemble(gprob, aopts)
        cg = torch.zeros(spec.n_nodes, dtype=torch.float64, device=dev)
        ginfo = P.nn_qp_solve(s, cg, P.solve_opts(rtol=args.rtol, max_iter=args.max_iter))
        cg = cg.cpu().numpy()
        bad = int(((cg < 0.0) | (cg > 1.0)).sum())
        dmp = {"galerkin_min": float(cg.min()), "galerkin_max": float(cg.max()), "nodes_violated": bad,
               "nodes": spec.n_nodes, "share": bad / spec.n_nodes, "galerkin_ms": ginfo["time_ms"],
               "galerkin_kkt_rel": ginfo["kkt_rel"]}
        del s
    return dict(times=times, infos=infos, kern_ms=[o[0]["time_ms"] for o in outs], graph=graph, dmp=dmp,
                kern_bytes=[o[0]["bytes_algo"] for o in outs], units_per_step=1, e2e=e2e,
                nnz_free=desc.get("nnz_free"), profile_scale_from=scale_from,
                h2d=hbytes + ch.numel() * 8, d2h=ch.numel() * 8, clocks=clocks, launches=launches,
                config=(steady3d_config(spec, args.n or 150, args) if args.workload == "steady3d" else
                        {"workload": name, "nodes": spec.n_nodes, "free": desc.get("n_free"),
                         "rtol": args.rtol,
                         "solver": args.solver + ("(ksp %g)" % args.ksp_rtol if args.solver == "tron" else ""),
                         "precision": args.cur_precision, "precond": precond_name(args),
                         "l2": "flushed between steps (256 MB write)"}),
                dtype="f64" if prec == P.NN_PREC_FP64 else "f32+f64", unit="QP solves/s", metric="QP solves/s")


def run_batch(P, torch, args, rank):
    count = args.count
    insts = I.config4_batch(count)
    dev = torch.device("cuda")
    prec = P.NN_PREC_MIXED if args.cur_precision == "mixed" else P.NN_PREC_FP64
    systems = [P.nn_assemble(P.Problem(sp, device=dev)) for sp in insts]
    cs = [torch.zeros(sp.n_nodes, dtype=torch.float64, device=dev) for sp in insts]
    opts = P.solve_opts(rtol=args.rtol, precision=prec)
    tuned = P.nn_batch_autotune(systems, opts)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        for c in cs:
            c.zero_()
        return P.nn_batch_solve(systems, cs, opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = P.kernel_launches()
    times, outs, clocks = timed_steps(torch, step, args.steps, flush,
                                      ClockSampler(os.path.join(args.out_dir, "clocks_rank%d.csv" % rank)))
    launches = P.kernel_launches() - l0
    infos = [i for o in outs for i in o]
    stream = torch.cuda.current_stream()
    # the same instances solved one after another by the single-system FP64
    # solver (one persistent launch each), once, for comparison
    seq_opts = P.solve_opts(rtol=args.rtol, precision=P.NN_PREC_FP64)
    for c in cs:
        c.zero_()
    flush.zero_()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for sy, c in zip(systems, cs):
        P.nn_qp_solve(sy, c, seq_opts)
    b.record(stream)
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    # end to end through the C ABI: every step assembles each instance from
    # pinned host buffers, copies the first iterates in, solves the batch and
    # reads the solutions back into pinned host memory
    hps = [pinned_problem(P, torch, sp) for sp in insts]
    c0h = [torch.zeros(sp.n_nodes, dtype=torch.float64).pin_memory() for sp in insts]
    outh = [torch.zeros(sp.n_nodes, dtype=torch.float64).pin_memory() for sp in insts]
    e2e = []
    for _ in range(min(args.steps, args.e2e_steps)):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ss = [P.nn_assemble(hp) for hp, _ in hps]
        for c, h in zip(cs, c0h):
            c.copy_(h, non_blocking=True)
        P.nn_batch_solve(ss, cs, opts)
        for h, c in zip(outh, cs):
            h.copy_(c, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e2e.append(a.elapsed_time(b))
        del ss
    h2d = sum(nb for _, nb in hps) + sum(h.numel() * 8 for h in c0h)
    d2h = sum(h.numel() * 8 for h in outh)
    return dict(times=times, infos=infos, kern_ms=[o[0]["time_ms"] for o in outs],
                kernel_name="k_batch_cluster" if tuned % 100 > 1 else "k_batch",
                kern_bytes=[sum(i["bytes_algo"] for i in o) for o in outs], units_per_step=count, e2e=e2e,
                h2d=h2d, d2h=d2h, clocks=clocks, launches=launches,
                sequential_fp64={"value": count / (seq_ms / 1e3), "unit": "QP solves/s", "ms": seq_ms,
                                 "how": "nn_qp_solve per instance, FP64, one after another"},
                config={"workload": "batch2d_%d" % count, "instances": count, "threads_per_block": tuned // 100, "ctas_per_instance": tuned % 100,
                        "precision": args.cur_precision, "rtol": args.rtol, "l2": "flushed between steps"},
                dtype="f64" if prec == P.NN_PREC_FP64 else "f32+f64", unit="QP solves/s", metric="QP solves/s")


def run_serve(P, torch, args, rank):
    """The serving stream as specified: Poisson arrivals at `rate` for
    `duration` s (seed 2015); arrival r carries request r, seeded (2015, r)
    (nn_inputs.serve_request).  The client sheds load like a bounded queue:
    an arrival that finds `queue` requests waiting (in the server's queue or
    still being generated) is refused and counted; otherwise its payload is
    generated by a pool of spawned processes and submitted.  Server latency is
    submit -> result; the client's generation time is reported beside it."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from collections import deque
    rate, duration = args.rate, args.duration
    arrivals = I.serve_arrivals(rate, duration)
    budget = int(args.budget_gb * (1 << 30))
    prec = {"mixed": P.NN_PREC_MIXED, "auto": P.NN_PREC_AUTO}.get(args.cur_precision, P.NN_PREC_FP64)
    sopts = P.solve_opts(precision=prec)
    workers = max(2, min(12, (os.cpu_count() or 4) - 2))
    gen = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    list(gen.map(I.serve_request, range(workers)))          # start the workers
    # warm-up: one small and one large request through a server of its own
    sv = P.nn_serve_create(budget, P.serve_opts(max_inflight=args.inflight, queue_capacity=args.queue, solve=sopts))
    for r in (0, 4):
        sp = I.serve_request(r)
        rid = P.nn_serve_submit(sv, P.Problem(sp))
        P.nn_serve_drain(sv)
        P.nn_serve_poll(sv, rid, np.zeros(sp.n_nodes))
    P.nn_serve_destroy(sv)
    sv = P.nn_serve_create(budget, P.serve_opts(max_inflight=args.inflight, queue_capacity=args.queue, solve=sopts))
    l0 = P.kernel_launches()
    pending = deque()          # (r, arrival time, future) in arrival order
    ids, kept, refused, late, gen_s = [], {}, 0, 0, []
    keep_first = 32

    def submit_ready(block=False):
        nonlocal late
        while pending and (block or pending[0][2].done()):
            r, ta, fut = pending.popleft()
            sp = fut.result()
            gen_s.append(time.perf_counter() - t0 - ta)
            try:
                ids.append((P.nn_serve_submit(sv, P.Problem(sp)), r, sp.n_nodes))
                if len(kept) < keep_first:
                    kept[r] = sp
            except P.NnError:
                late += 1

    t0 = time.perf_counter()
    for r, ta in enumerate(arrivals):
        while True:
            submit_ready()
            now = time.perf_counter() - t0
            if now >= ta:
                break
            time.sleep(min(ta - now, 0.002))
        if P.nn_serve_stats(sv)["queued"] + len(pending) >= args.queue:
            refused += 1
            continue
        pending.append((r, ta, gen.submit(I.serve_request, r)))
    submit_ready(block=True)
    window = time.perf_counter() - t0
    P.nn_serve_drain(sv)
    wall = time.perf_counter() - t0
    st = P.nn_serve_stats(sv)
    ok, failed, fallbacks, kkt_max = 0, [], 0, 0.0
    for rid, r, nn in ids:
        try:
            info = P.nn_serve_poll(sv, rid, np.zeros(nn))
        except P.NnError as e:
            failed.append(str(e))
            continue
        ok += info is not None and info["status"] == 0
        if info is not None:
            fallbacks += int(info["fp64_fallback"])
            kkt_max = max(kkt_max, info["kkt_rel"])
    P.nn_serve_destroy(sv)
    gen.shutdown()
    launches = P.kernel_launches() - l0
    # the plain FP64 path on the first served requests: each assembled from
    # host arrays and solved alone by nn_qp_solve in FP64, one after another
    dev = torch.device("cuda")
    fp64 = P.solve_opts(precision=P.NN_PREC_FP64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for sp in kept.values():
        s_ = P.nn_assemble(P.Problem(sp), P.assemble_opts())
        c_ = torch.zeros(sp.n_nodes, dtype=torch.float64, device=dev)
        P.nn_qp_solve(s_, c_, fp64)
        c_.cpu()
        del s_
    seq_s = time.perf_counter() - t1
    sequential = {"value": len(kept) / seq_s if kept else None, "unit": "solves/s", "requests": len(kept),
                  "mean_nodes": float(np.mean([sp.n_nodes for sp in kept.values()])) if kept else None,
                  "served_mean_nodes": float(np.mean([nn for _, _, nn in ids])) if ids else None,
                  "how": "the first %d served requests, copied from host, assembled and solved alone in FP64 one "
                         "after another (nn_assemble + nn_qp_solve)" % len(kept)}
    return dict(stats=st, wall=wall, window=window, offered=len(arrivals), submitted=len(ids), refused=refused,
                fallbacks=fallbacks, kkt_max=kkt_max,
                late=late, ok=ok, failed=len(failed), sequential=sequential, gen_mean_s=float(np.mean(gen_s)) if gen_s else 0.0,
                first_failure=failed[0] if failed else None, launches=launches,
                config={"workload": "serve_poisson%g_for%gs" % (rate, duration), "requests": "request r seeded (2015, r)",
                        "max_inflight": args.inflight, "queue_capacity": args.queue, "budget_gb": args.budget_gb,
                        "precision": args.cur_precision, "client_workers": workers})


def serving_object(r, args):
    st = r["stats"]
    return {"metric": "serving p50/p99 latency (submit -> result)", "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_ms": st["mean_ms"], "solves_per_s": st["solves_per_s"], "offered": r["offered"],
            "offered_per_s": args.rate, "duration_s": args.duration, "submitted": r["submitted"],
            "refused_at_arrival": r["refused"], "refused_at_submit": r["late"], "completed": st["completed"],
            "ok": r["ok"], "failed": st["failed"], "first_failure": r["first_failure"], "window_s": r["window"],
            "max_kkt_rel": r["kkt_max"], "fp64_fallbacks": r["fallbacks"],
            "wall_s": r["wall"], "saturated": r["refused"] > 0 or st["solves_per_s"] < 0.95 * args.rate,
            "client_generation_mean_s": r["gen_mean_s"], "bytes_peak_measured": st["bytes_peak"],
            "bytes_reserved_peak": st["bytes_reserved_peak"], "estimate_overruns": st["estimate_overruns"],
            "estimate_max_ratio": st["estimate_max_ratio"], "inflight_peak": st["inflight_peak"],
            "dtype": {"mixed": "f32+f64", "auto": "f32+f64 where the FP32 operator exceeds 48 MB, else f64"}.get(
                args.cur_precision, "f64"), "gpu_launches": r["launches"],
            "sequential_fp64": r["sequential"],
            "vs_sequential_fp64": (st["solves_per_s"] / r["sequential"]["value"]) if r["sequential"]["value"] else None,
            "config": r["config"]}


def resolve_precision(args):
    """--precision default: both precisions for the 150^3 workload (the FP64
    line with the mixed run as a sub-object), the serving precision for the
    serving workload, FP64 otherwise; "both" only where the workload has the
    sub-object and the preconditioner is Jacobi (SSOR runs in FP64)."""
    if args.workload == "serve" and args.precision == "default":
        args.precision = args.serve_precision
    if args.workload == "steady3d" and args.precision == "default":
        args.precision = "both"
    elif args.precision == "default":
        args.precision = "fp64"
    if args.precision == "both" and (args.workload != "steady3d" or getattr(args, "precond", "jacobi") == "ssor"):
        args.precision = "fp64"
    return args


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="steady3d",
                    choices=["transient3d", "steady3d", "steady2d", "batch", "serve", "cube_hole"])
    ap.add_argument("--precision", default="default", choices=["default", "auto", "fp64", "mixed", "both"],
                    help="default: both for steady3d (FP64 line + mixed object), the serving precision for serve, "
                         "fp64 otherwise; auto: the library's NN_PREC_AUTO")
    ap.add_argument("--mass", default="consistent", choices=["consistent", "lumped"],
                    help="capacity matrix of the transient workload")
    ap.add_argument("--solver", default="gpcg", choices=["gpcg", "lbfgs", "tron"])
    ap.add_argument("--ksp-rtol", type=float, default=1e-1, help="TRON: subspace tolerance relative to the face gradient at the Cauchy point")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "ssor"],
                    help="preconditioner of the CG iterations (ssor: multicolour SSOR, FP64 only)")
    ap.add_argument("--omega", type=float, default=1.0, help="SSOR relaxation factor")
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--m", type=int, default=16, help="cube with a hole: n = 9m hexahedra per side")
    ap.add_argument("--mesh", default="mirrored", choices=["kuhn", "mirrored"], help="cube with a hole: mesh type")
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--serve-precision", default="auto", choices=["fp64", "mixed", "auto"],
                    help="precision of the serving run attached to the default line")
    ap.add_argument("--no-serving", action="store_true", help="default workload: skip the serving run")
    ap.add_argument("--inflight", type=int, default=8)
    ap.add_argument("--queue", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--e2e-steps", type=int, default=5, help="end-to-end repeats (host buffers, copies timed)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "bench_out"))
    args = ap.parse_args()
    os.makedirs(args.out_dir, exist_ok=True)
    dist, rank, ws = dist_init()
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else FALLBACK_HBM
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback"

    resolve_precision(args)

    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    import paper_1506_08435_gb300 as P
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    P.lib()
    barrier(dist)
    if args.workload == "serve":
        return serve_line(P, torch, args, rank, ws)
    precisions = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    lines = []
    for prec in precisions:
        args.cur_precision = prec
        if args.workload == "transient3d":
            r = run_transient(P, torch, args, rank)
        elif args.workload in ("steady3d", "cube_hole"):
            r = run_steady(P, torch, args, rank, 3)
        elif args.workload == "steady2d":
            r = run_steady(P, torch, args, rank, 2)
        else:
            r = run_batch(P, torch, args, rank)
        barrier(dist)
        lines.append(result_line(r, args, prec, dist, ws, hbm_peak, peak_src))
    line = lines[0]
    if len(lines) > 1:
        m = lines[1]
        sub = {k: m[k] for k in ("value", "unit", "ms_per_step", "dtype", "roofline", "alu", "e2e", "max_kkt_rel",
                                 "statuses_ok", "spmv_per_step", "spmv64_per_step", "refinements_per_step",
                                 "fp64_fallbacks", "gpu_launches", "clocks") if k in m}
        line["mixed"] = sub
        line["vs_plain_fp64"] = m["value"] / line["value"]
        line["precision_note"] = "the line is the plain FP64 solve; \"mixed\" is the same workload in mixed precision"
    if args.workload == "steady3d" and not args.no_serving and not args.n:
        # the serving stream (Poisson arrivals) on the same GPU, reported beside the line
        args.cur_precision = args.serve_precision
        line["serving"] = serving_object(run_serve(P, torch, args, rank), args)
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample(args.workload, n=args.n or None, lumped=args.mass == "lumped")
        if v is not None:
            line["cpu_baseline"] = {"value": v, "unit": line["unit"], "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def workload_config(args):
    """config object of a line (both arms print the same one)."""
    if args.workload == "transient3d":
        return transient_config(I.config2_transient_3d(), args)
    if args.workload == "steady3d":
        n = args.n or 150
        spec = I.config3_steady_3d(n=n)
        return steady3d_config(spec, n, args)
    return {"workload": args.workload}


def steady3d_config(spec, n, args):
    return {"workload": "steady3d_n%d" % n, "nodes": int(spec.n_nodes), "tets": 6 * n ** 3,
            "free": int((np.asarray(spec.dmask) == 0).sum()), "rtol": args.rtol,
            "solver": args.solver + ("(ksp %g)" % args.ksp_rtol if args.solver == "tron" else ""),
            "precision": args.precision, "precond": precond_name(args),
            "l2": "inputs far larger than L2, flushed between steps (256 MB write)"}


def reference_arm(args, rank):
    """The oracle as it stands on the host cores, on this arm's config,
    metric and unit; each step a bounded sample of the workload."""
    if rank != 0:
        return 0
    t0 = time.perf_counter()
    cores = os.cpu_count() or 1
    if args.workload == "steady3d":
        orc = Steady3dOracle(args.n or 150, cores)
        for _ in range(args.warmup):
            orc.iterations(2)
        k = 20
        vals = [orc.value(orc.iterations(k)) for _ in range(args.steps)]
        desc = orc.describe(k) + "; one step = one batch"
    else:
        vals = []
        for _ in range(args.warmup):
            oracle_sample(args.workload, budget_s=1.0, lumped=args.mass == "lumped")
        for _ in range(args.steps):
            v, cores, desc = oracle_sample(args.workload, budget_s=8.0, lumped=args.mass == "lumped")
            vals.append(v)
    v = float(np.median(vals)) if all(x is not None for x in vals) else None
    print(json.dumps({"impl": "reference", "metric": "QP solves/s", "value": v, "unit": "QP solves/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": workload_config(args),
                      "cpu_baseline": {"value": v, "unit": "QP solves/s", "cores": cores, "kind": "oracle",
                                       "sample": desc},
                      "e2e": {"value": v, "unit": "QP solves/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0},
                      "wall_s": time.perf_counter() - t0}))
    return 0


def result_line(r, args, prec, dist, ws, hbm_peak, peak_src):
    """The contract's JSON line of one timed run r."""
    total_ms = max_over_ranks(dist, sum(r["times"]))
    units = r["units_per_step"] * args.steps * ws
    value = units / (total_ms / 1e3)
    kern_ms = float(np.mean(r["kern_ms"]))
    kern_bytes = float(np.mean(r["kern_bytes"]))
    achieved = kern_bytes / (kern_ms / 1e3) / 1e9
    # DRAM bytes per launch of the dominant kernel from the committed ncu
    # summary of this workload and precision (a line "dram_bytes_per_launch:
    # N"), used only while that summary's "source_digest:" line matches the
    # kernel sources as they are now (counters of an older kernel are void)
    infos = r["infos"]
    spl = sum(i["spmv"] for i in infos) / args.steps
    # (a solver other than GPCG, or the SSOR preconditioner, runs other code:
    # its summary carries the solver and preconditioner in the name)
    tag = prec + ("" if getattr(args, "solver", "gpcg") == "gpcg" else "_" + args.solver) + \
        ("_ssor" if getattr(args, "precond", "jacobi") == "ssor" else "")
    traffic, traffic_src = profile_traffic(os.path.join(ROOT, "profiles"), r.get("kernel_name", "k_solve_grid"),
                                           r["config"]["workload"], tag, source_digest(),
                                           r.get("profile_scale_from"), spl, r.get("nnz_free"), kern_bytes)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": traffic, "traffic_source": traffic_src,
            "kernel": "solve kernel (persistent, one launch per step)", "kernel_ms": kern_ms,
            "algo_bytes_per_launch": kern_bytes, "peak_source": peak_src,
            "achieved_is": "algorithmic bytes (products at the MatMult model + every vector stream) / launch time"}
    if traffic:
        roof["dram_gbs"] = traffic / (kern_ms / 1e3) / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / hbm_peak
    line = {"metric": r["metric"], "value": value, "unit": r["unit"], "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic", "config": r["config"],
            "roofline": roof, "gpu_launches": r["launches"], "clocks": r["clocks"],
            "max_kkt_rel": float(max(i["kkt_rel"] for i in infos)),
            "statuses_ok": all(i["status"] == 0 for i in infos),
            "spmv_per_step": sum(i["spmv"] for i in infos) / args.steps,
            "spmv64_per_step": sum(i["spmv64"] for i in infos) / args.steps,
            "cg_iters_per_step": sum(i["cg_iters"] for i in infos) / args.steps,
            "phases_per_step": sum(i["iterations"] for i in infos) / args.steps,
            "refinements_per_step": sum(i["refinements"] for i in infos) / args.steps,
            "fp64_fallbacks": int(sum(i["fp64_fallback"] for i in infos))}
    pcs = sum(i.get("pc_applies", 0) for i in infos)
    if pcs:
        line["pc_applies_per_step"] = pcs / args.steps
    # the FP64 pipe as the second roof: algorithmic FP64 operations of the
    # launch / its time, against 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
    fl64 = sum(i.get("flops64_algo", 0.0) for i in infos) / args.steps
    fl_all = sum(i.get("flops_algo", 0.0) for i in infos) / args.steps
    if fl64 > 0 and fl64 >= 0.5 * fl_all:   # the FP64 pipe is a roof only where FP64 work dominates
        ach = fl64 / (kern_ms / 1e3) / 1e9
        line["alu"] = {"bound": "alu", "pipe": "fp64", "achieved": ach, "peak": FP64_PIPE_PEAK_GFLOPS,
                       "unit": "GFLOP/s", "frac": ach / FP64_PIPE_PEAK_GFLOPS, "flops_per_launch": fl64,
                       "peak_source": "152 SMs x 2 DFMA/clk (ncu unit count) x 2 flop x 2.07 GHz"}
        hbm_frac = roof.get("dram_frac") or roof["frac"]
        if line["alu"]["frac"] > max(roof["frac"], roof.get("dram_frac") or 0.0):
            roof["bound"] = "alu"
            roof["bound_note"] = "the FP64 pipe fraction (alu) exceeds the HBM fraction"
        elif line["alu"]["frac"] >= 0.8 * hbm_frac:
            roof["bound_note"] = ("co-bound: the FP64 pipe fraction (alu %.2f, algorithmic FP64 operations) is close "
                                  "to the HBM fraction (%.2f, %s)"
                                  % (line["alu"]["frac"], hbm_frac, "DRAM" if roof.get("dram_frac") else "algorithmic"))
    for key in ("graph", "dmp", "sequential_fp64"):
        if r.get(key):
            line["galerkin_dmp" if key == "dmp" else key] = r[key]
    if r["e2e"]:
        e2e_ms = max_over_ranks(dist, sum(r["e2e"]))
        line["e2e"] = {"value": r["units_per_step"] * len(r["e2e"]) * ws / (e2e_ms / 1e3), "unit": r["unit"],
                       "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"], "steps": len(r["e2e"])}
    else:
        line["e2e"] = None
    return line


def serve_line(P, torch, args, rank, ws):
    args.cur_precision = args.precision
    r = run_serve(P, torch, args, rank)
    if rank == 0:
        obj = serving_object(r, args)
        line = {"metric": "serving p50/p99 latency", "value": obj["p50_ms"], "unit": "ms", "higher_is_better": False,
                "n_gpus": ws, "data": "synthetic"}
        line.update(obj)
        if not args.no_cpu_baseline:
            v, cores, desc = oracle_sample("serve")
            line["cpu_baseline"] = {"value": v, "unit": "QP solves/s (throughput)", "cores": cores, "kind": "oracle",
                                    "sample": desc}
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
