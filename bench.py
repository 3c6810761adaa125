"""Benchmark of the non-negative diffusion QP path on GB300.

Default workload (no flags, N = 1): the 3D transient problem -- unit cube,
40^3 hexahedra x 6 tetrahedra (68,921 nodes), dispersion tensor from the
vortex velocity field (alpha_L = 1, alpha_T = 1e-3, D_M = 1e-9), c = 1 on
the x = 0 patch and c = 0 on x = 1, 0 <= c <= 1, backward Euler dt = 0.01
over 50 steps, one warm-started QP per step, FP64.  One benchmark step is
the whole path on one synthetic input: device assembly (pattern, element
matrices, elimination, SELL build) + the 50-step transient run in one
persistent launch (every QP to KKT <= 1e-10 relative, tighter than the
1e-8 acceptance).  metric: QP solves per second (50 per step).  The inputs
(about 12 MB) fit in L2, so L2 is flushed between timed steps (256 MB write).

Options of the default workload: --precision fp64|mixed, --solver
gpcg|lbfgs|tron (--ksp-rtol: TRON's subspace tolerance), --mass
consistent|lumped (capacity matrix).

Other workloads (--workload), each printing its own line:
  steady3d   config 3 (150^3 x 6 tets; --n to shrink), --precision fp64|mixed,
             --solver gpcg|lbfgs|tron; a step = assembly + one solve
  steady2d   config 1 (50 x 50, 2D); a step = assembly + one solve
  batch      config 4 (512 2D instances, one persistent launch); a step =
             one batched solve of all instances, --precision fp64|mixed; also
             reports the single-system FP64 solver on the same instances
  cube_hole  the cube with a cubic hole (Sec. 5.1 analogue; --m, --mesh
             kuhn|mirrored); a step = assembly + one solve; also reports the
             Galerkin solution's departure from [0, 1] (an unbounded solve)
  serve      config 5 (Poisson arrivals); reports p50/p99 latency
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

def oracle_sample(workload, budget_s=20.0, n=None, lumped=False):
    """The FP64 oracle as it stands, on a bounded sample of the workload;
    returns (units per second, cores used, description)."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
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

def profile_traffic(pdir, kname, workload, precision, digest, scale_from=None, products=None, nnz_free=None):
    """DRAM bytes per launch of kernel kname on this workload from the committed
    ncu summary <kname>_<workload>_<precision>.md in pdir (its line
    "dram_bytes_per_launch: N"), used only while its "source_digest:" line
    equals digest.  Without a summary for the workload itself, the summary of
    the smaller case scale_from is scaled by products x nnz_free (its
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
        if key in ("dram_bytes_per_launch", "source_digest", "products_per_launch", "nnz_free"):
            v = line.split(":", 1)[1].strip()
            fields[key] = v.split()[0] if v else ""
    if fields.get("source_digest") != digest:
        return None, "kernel changed since the ncu capture in %s" % name
    try:
        traffic = float(fields["dram_bytes_per_launch"])
        if not scaled:
            return traffic, "ncu capture, %s" % name
        traffic *= products / float(fields["products_per_launch"]) * nnz_free / float(fields["nnz_free"])
        return traffic, "ncu capture of a smaller case (%s), scaled by products x nnz_free" % name
    except (KeyError, ValueError, TypeError, ZeroDivisionError):
        return None, "incomplete ncu summary %s" % name


def solver_code(P, args):
    return {"gpcg": P.NN_SOLVER_GPCG, "lbfgs": P.NN_SOLVER_LBFGS, "tron": P.NN_SOLVER_TRON}[args.solver]


def transient_config(spec, args):
    """config of the default workload (both arms print the same one)."""
    return {"workload": "transient3d_n40_dt0.01_50steps", "nodes": spec.n_nodes, "tets": spec.n_elems,
            "qp_per_step": spec.nsteps, "rtol": args.rtol, "l2": "flushed between steps (256 MB write)",
            "solver": args.solver + ("(ksp %g)" % args.ksp_rtol if args.solver == "tron" else ""),
            "precision": args.precision, "mass": args.mass,
            "first_iterate": "projected 3c^n - 3c^(n-1) + c^(n-2)"}


def run_transient(P, torch, args, rank):
    spec = I.config2_transient_3d()
    dev = torch.device("cuda")
    nsteps = spec.nsteps
    prob = P.Problem(spec, device=dev)
    mixed = args.precision == "mixed"
    opts = P.solve_opts(rtol=args.rtol, solver=solver_code(P, args), ksp_rtol=args.ksp_rtol,
                        precision=P.NN_PREC_MIXED if mixed else P.NN_PREC_FP64)
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
    for _ in range(args.steps):
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
    prec = P.NN_PREC_MIXED if args.precision == "mixed" else P.NN_PREC_FP64
    opts = P.solve_opts(rtol=args.rtol, precision=prec, max_iter=args.max_iter,
                        solver=solver_code(P, args), ksp_rtol=args.ksp_rtol)
    aopts = P.assemble_opts(build_mixed=1 if prec == P.NN_PREC_MIXED else 0)
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
    for _ in range(args.steps):
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
    scale_from = "steady3d_n104" if dim == 3 else None
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
                config={"workload": name, "nodes": spec.n_nodes, "free": desc.get("n_free"),
                        "nnz_free": desc.get("nnz_free"), "rtol": args.rtol,
                        "solver": args.solver + ("(ksp %g)" % args.ksp_rtol if args.solver == "tron" else ""),
                        "precision": args.precision, "l2": "flushed between steps (256 MB write)"},
                dtype="f64" if prec == P.NN_PREC_FP64 else "f32+f64", unit="QP solves/s", metric="QP solves/s")


def run_batch(P, torch, args, rank):
    count = args.count
    insts = I.config4_batch(count)
    dev = torch.device("cuda")
    prec = P.NN_PREC_MIXED if args.precision == "mixed" else P.NN_PREC_FP64
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
    for _ in range(args.steps):
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
                        "precision": args.precision, "rtol": args.rtol, "l2": "flushed between steps"},
                dtype="f64" if prec == P.NN_PREC_FP64 else "f32+f64", unit="QP solves/s", metric="QP solves/s")


def run_serve(P, torch, args, rank):
    rate, duration = args.rate, args.duration
    arrivals = I.serve_arrivals(rate, duration)
    pool = [I.serve_request(r) for r in range(args.pool)]
    probs = [P.Problem(sp) for sp in pool]
    budget = int(args.budget_gb * (1 << 30))
    sopts = P.solve_opts(precision=P.NN_PREC_MIXED if args.precision == "mixed" else P.NN_PREC_FP64)
    sv = P.nn_serve_create(budget, P.serve_opts(max_inflight=args.inflight, queue_capacity=args.queue, solve=sopts))
    # warm-up: one request of each kind
    for k in range(min(2, len(probs))):
        rid = P.nn_serve_submit(sv, probs[k])
        P.nn_serve_drain(sv)
        P.nn_serve_poll(sv, rid, np.zeros(pool[k].n_nodes))
    P.nn_serve_destroy(sv)
    # a bounded queue: past saturation, arrivals are refused (counted) instead
    # of piling up, so the drain after the arrival window stays short
    sv = P.nn_serve_create(budget, P.serve_opts(max_inflight=args.inflight, queue_capacity=args.queue, solve=sopts))
    l0 = P.kernel_launches()
    ids = []
    t0 = time.perf_counter()
    for k, ta in enumerate(arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        try:
            ids.append((P.nn_serve_submit(sv, probs[k % len(probs)]), k % len(probs)))
        except P.NnError:
            pass
    P.nn_serve_drain(sv)
    wall = time.perf_counter() - t0
    st = P.nn_serve_stats(sv)
    ok, failed = 0, []
    for rid, k in ids:
        try:
            info = P.nn_serve_poll(sv, rid, np.zeros(pool[k].n_nodes))
        except P.NnError as e:
            failed.append(str(e))
            continue
        ok += info is not None and info["status"] == 0
    P.nn_serve_destroy(sv)
    launches = P.kernel_launches() - l0
    # the plain path for comparison: the first requests of the pool, each
    # assembled and solved alone in FP64 (nn_assemble + nn_qp_solve), one after another
    dev = torch.device("cuda")
    seq_n = min(args.pool, 32)
    fp64 = P.solve_opts(precision=P.NN_PREC_FP64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for sp in pool[:seq_n]:
        s_ = P.nn_assemble(P.Problem(sp, device=dev))
        c_ = torch.zeros(sp.n_nodes, dtype=torch.float64, device=dev)
        P.nn_qp_solve(s_, c_, fp64)
        c_.cpu()
        del s_
    seq_s = time.perf_counter() - t1
    served_work = sum(pool[k].n_nodes for _, k in ids) / max(len(ids), 1)
    sequential = {"value": seq_n / seq_s, "unit": "solves/s", "requests": seq_n,
                  "mean_nodes": float(np.mean([sp.n_nodes for sp in pool[:seq_n]])),
                  "served_mean_nodes": served_work,
                  "how": "first %d requests of the payload pool, copied from host, assembled and solved alone in "
                         "FP64 one after another" % seq_n}
    return dict(stats=st, wall=wall, offered=len(arrivals), ok=ok, failed=len(failed), sequential=sequential,
                first_failure=failed[0] if failed else None, launches=launches,
                config={"workload": "serve_poisson%g_for%gs" % (rate, duration), "payload_pool": args.pool,
                        "max_inflight": args.inflight, "queue_capacity": args.queue, "budget_gb": args.budget_gb,
                        "precision": args.precision})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="transient3d",
                    choices=["transient3d", "steady3d", "steady2d", "batch", "serve", "cube_hole"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--mass", default="consistent", choices=["consistent", "lumped"],
                    help="capacity matrix of the transient workload")
    ap.add_argument("--solver", default="gpcg", choices=["gpcg", "lbfgs", "tron"])
    ap.add_argument("--ksp-rtol", type=float, default=1e-1, help="TRON: subspace tolerance relative to the face gradient at the Cauchy point")
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--m", type=int, default=16, help="cube with a hole: n = 9m hexahedra per side")
    ap.add_argument("--mesh", default="mirrored", choices=["kuhn", "mirrored"], help="cube with a hole: mesh type")
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--inflight", type=int, default=8)
    ap.add_argument("--queue", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "bench_out"))
    args = ap.parse_args()
    os.makedirs(args.out_dir, exist_ok=True)
    dist, rank, ws = dist_init()
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else FALLBACK_HBM
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback"

    if args.impl == "reference":
        if rank != 0:
            return 0
        vals, cores, desc = [], os.cpu_count() or 1, ""
        t0 = time.perf_counter()
        for _ in range(args.warmup):
            oracle_sample(args.workload, budget_s=1.0, lumped=args.mass == "lumped")
        for _ in range(args.steps):
            v, cores, desc = oracle_sample(args.workload, budget_s=8.0, lumped=args.mass == "lumped")
            vals.append(v)
        v = float(np.median(vals))
        print(json.dumps({"impl": "reference", "metric": "QP solves/s", "value": v, "unit": "QP solves/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic",
                          "config": (transient_config(I.config2_transient_3d(), args) if args.workload == "transient3d"
                                     else {"workload": args.workload}),
                          "cpu_baseline": {"value": v, "unit": "QP solves/s", "cores": cores, "kind": "oracle",
                                           "sample": desc},
                          "e2e": {"value": v, "unit": "QP solves/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0},
                          "wall_s": time.perf_counter() - t0}))
        return 0

    import torch
    import paper_1506_08435_gb300 as P
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    P.lib()
    barrier(dist)
    if args.workload == "serve":
        r = run_serve(P, torch, args, rank)
        st = r["stats"]
        if rank == 0:
            print(json.dumps({"metric": "serving p50/p99 latency", "value": st["p50_ms"], "unit": "ms",
                              "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "solves_per_s": st["solves_per_s"],
                              "offered": r["offered"], "offered_per_s": args.rate, "completed": st["completed"],
                              "ok": r["ok"], "failed": st["failed"], "first_failure": r["first_failure"],
                              "rejected": st["rejected"],
                              "wall_s": r["wall"], "saturated": st["rejected"] > 0 or st["solves_per_s"] < 0.95 * args.rate,
                              "bytes_peak": st["bytes_peak"], "inflight_peak": st["inflight_peak"],
                              "higher_is_better": False, "n_gpus": ws,
                              "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
                              "gpu_launches": r["launches"], "sequential_fp64": r["sequential"],
                              "config": r["config"]}))
        return 0
    if args.workload == "transient3d":
        r = run_transient(P, torch, args, rank)
    elif args.workload == "steady3d":
        r = run_steady(P, torch, args, rank, 3)
    elif args.workload == "steady2d":
        r = run_steady(P, torch, args, rank, 2)
    elif args.workload == "cube_hole":
        r = run_steady(P, torch, args, rank, 3)
    else:
        r = run_batch(P, torch, args, rank)
    barrier(dist)
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
    spl = sum(i["spmv"] for i in r["infos"]) / args.steps
    traffic, traffic_src = profile_traffic(os.path.join(ROOT, "profiles"), r.get("kernel_name", "k_solve_grid"),
                                           r["config"]["workload"], args.precision, source_digest(),
                                           r.get("profile_scale_from"), spl, r.get("nnz_free"))
    infos = r["infos"]
    line = {"metric": r["metric"], "value": value, "unit": r["unit"], "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic", "config": r["config"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic, "traffic_source": traffic_src,
                         "kernel": "solve kernel (persistent, one launch per step)",
                         "kernel_ms": kern_ms, "algo_bytes_per_launch": kern_bytes, "peak_source": peak_src},
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "max_kkt_rel": float(max(i["kkt_rel"] for i in infos)),
            "statuses_ok": all(i["status"] == 0 for i in infos),
            "spmv_per_step": sum(i["spmv"] for i in infos) / args.steps,
            "cg_iters_per_step": sum(i["cg_iters"] for i in infos) / args.steps,
            "phases_per_step": sum(i["iterations"] for i in infos) / args.steps}
    # the FP64 pipe as a second bound: algorithmic FP64 operations of the dominant
    # kernel per launch / its time, against 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
    fl64 = sum(i.get("flops64_algo", 0.0) for i in infos) / args.steps
    if fl64 > 0:
        ach = fl64 / (kern_ms / 1e3) / 1e9
        line["fp64_pipe"] = {"achieved": ach, "peak": FP64_PIPE_PEAK_GFLOPS, "unit": "GFLOP/s",
                             "frac": ach / FP64_PIPE_PEAK_GFLOPS, "flops_per_launch": fl64}
    if r.get("graph"):
        line["graph"] = r["graph"]
    if r.get("dmp"):
        line["galerkin_dmp"] = r["dmp"]
    if r.get("sequential_fp64"):
        line["sequential_fp64"] = r["sequential_fp64"]
    if r["e2e"] is not None:
        e2e_ms = max_over_ranks(dist, sum(r["e2e"]))
        line["e2e"] = {"value": r["units_per_step"] * len(r["e2e"]) * ws / (e2e_ms / 1e3), "unit": r["unit"],
                       "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]}
    else:
        line["e2e"] = None
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample(args.workload, lumped=args.mass == "lumped")
        if v is not None:
            line["cpu_baseline"] = {"value": v, "unit": r["unit"], "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
