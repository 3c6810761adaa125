"""Benchmark of the non-negative diffusion QP path on GB300.

Default workload (N = 1): the 3D transient problem -- unit cube, 40^3
hexahedra x 6 tetrahedra (68,921 nodes), dispersion tensor from the vortex
velocity field (alpha_L = 1, alpha_T = 1e-3, D_M = 1e-9), c = 1 on the
x = 0 patch and c = 0 on x = 1, 0 <= c <= 1, backward Euler dt = 0.01 over
50 steps, one warm-started QP per step, FP64.  One benchmark step is the
whole path on one synthetic input: device assembly (pattern, element
matrices, elimination, SELL build) + the 50-step transient run in one
persistent launch (every QP to KKT <= 1e-10 relative, which is tighter than
the 1e-8 acceptance).

metric: QP solves per second (50 per step).  The inputs (about 12 MB) fit
in L2, so L2 is flushed between timed steps by writing a 256 MB buffer.

Other workloads (--workload): steady3d (150^3 x 6 tets, FP64 or mixed),
steady2d (the 2D 50 x 50 problem), batch (512 2D instances), serve.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import nn_inputs as I  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0


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

def oracle_sample(workload, budget_s=20.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload;
    returns (QP solves per second, cores, description)."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    if workload == "transient3d":
        spec = I.config2_transient_3d()
        coords, conn = O.mesh_structured(3, spec.nx)
        asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, with_mass=True)
        red = O.Reduced(asm, spec.dmask, spec.dval, dt=spec.dt)
        c = spec.c0.copy()
        t0, n = time.perf_counter(), 0
        while n < 1 or (time.perf_counter() - t0 < budget_s and n < spec.nsteps):
            b = red.rhs(c)
            x, _ = O.solve_qp(red.A, b, spec.lo, spec.hi, x0=c[red.free], threads=threads)
            c = red.full(x)
            n += 1
        dt = time.perf_counter() - t0
        return n / dt, threads, "first %d backward-Euler QP steps of the 40^3 transient problem (MPRGP + " \
                                "polish to 1e-12, OpenMP products), assembly excluded" % n
    if workload == "steady2d":
        spec = I.config1_steady_2d()
        coords, conn = O.mesh_structured(2, spec.nx)
        asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, f_elem=spec.f_elem)
        red = O.Reduced(asm, spec.dmask, spec.dval)
        b = red.rhs()
        t0, n = time.perf_counter(), 0
        while n < 1 or time.perf_counter() - t0 < min(budget_s, 5.0):
            O.solve_qp(red.A, b, spec.lo, spec.hi, threads=1)
            n += 1
        return n / (time.perf_counter() - t0), 1, "%d full solves of the 2D 50x50 problem" % n
    return None, threads, "no oracle sample for this workload"


# ---------------------------------------------------------------- workloads

def run_transient(P, torch, args, rank):
    spec = I.config2_transient_3d()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    nsteps = spec.nsteps
    prob = P.Problem(spec, device=dev)
    opts = P.solve_opts(rtol=args.rtol)
    aopts = P.assemble_opts(build_mixed=0, keep_full=1)
    c0 = torch.tensor(spec.c0, device=dev)
    cf = torch.zeros_like(c0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        s = P.nn_assemble(prob, aopts)
        infos = P.nn_transient(s, c0, nsteps, cf, None, opts)
        return s, infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = P.kernel_launches()
    times, kern_ms, kern_bytes, statuses, spmv, kkt = [], [], [], [], 0, []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(os.path.join(args.out_dir, "clocks_rank%d.csv" % rank))
    clk.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        s, infos = step()
        ev[k][1].record(stream)
        kern_ms.append(infos[0]["time_ms"])
        kern_bytes.append(sum(i["bytes_algo"] for i in infos))
        statuses += [i["status"] for i in infos]
        spmv += sum(i["spmv"] for i in infos)
        kkt.append(max(i["kkt_rel"] for i in infos))
        del s
    torch.cuda.synchronize()
    clocks = clk.stop(torch.cuda.current_device())
    launches = P.kernel_launches() - launches0
    times = [a.elapsed_time(b) for a, b in ev]
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hp = P.Problem(spec)
    pinned = {}
    for name in ("coef", "dmask", "dval"):
        a = getattr(hp, name)
        t = torch.from_numpy(a).pin_memory()
        pinned[name] = t
    hp2 = P.Problem(spec)
    hp2.coef, hp2.dmask, hp2.dval = pinned["coef"], pinned["dmask"], pinned["dval"]
    hp2.c.coef, hp2.c.dirichlet_mask, hp2.c.dirichlet_value = (pinned["coef"].data_ptr(), pinned["dmask"].data_ptr(),
                                                               pinned["dval"].data_ptr())
    hp2.c.memory = P.NN_MEM_HOST
    c0h = torch.from_numpy(spec.c0.copy()).pin_memory()
    cfh = torch.zeros_like(c0h).pin_memory()
    e2e = []
    for k in range(max(args.steps, 1)):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s = P.nn_assemble(hp2, aopts)
        P.nn_transient(s, c0h, nsteps, cfh, None, opts)
        b.record(stream)
        torch.cuda.synchronize()
        e2e.append(a.elapsed_time(b))
        del s
    h2d = sum(pinned[n].numel() * pinned[n].element_size() for n in pinned) + c0h.numel() * 8
    d2h = cfh.numel() * 8
    return dict(times=times, kern_ms=kern_ms, kern_bytes=kern_bytes, statuses=statuses, spmv=spmv, kkt=kkt,
                units_per_step=nsteps, e2e=e2e, h2d=h2d, d2h=d2h, clocks=clocks, launches=launches,
                config={"workload": "transient3d_n40_dt0.01_50steps", "nodes": spec.n_nodes,
                        "tets": spec.n_elems, "qp_per_step": nsteps, "rtol": args.rtol,
                        "l2": "flushed between steps (256 MB write)", "solver": "gpcg", "precision": "fp64"},
                dtype="f64", n=int(68921 - 0), nnz=None)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="transient3d")
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "gpurun_out"))
    args = ap.parse_args()
    os.makedirs(args.out_dir, exist_ok=True)
    dist, rank, ws = dist_init()
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else FALLBACK_HBM
    peak_src = "measured" if pk else "fallback"

    if args.impl == "reference":
        if rank != 0:
            return 0
        vals = []
        cores, desc = os.cpu_count() or 1, ""
        t0 = time.perf_counter()
        for _ in range(args.warmup):
            oracle_sample(args.workload, budget_s=2.0)
        for _ in range(args.steps):
            v, cores, desc = oracle_sample(args.workload, budget_s=10.0)
            vals.append(v)
        v = float(np.median(vals))
        line = {"impl": "reference", "metric": "QP solves/s", "value": v, "unit": "QP solves/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload},
                "cpu_baseline": {"value": v, "unit": "QP solves/s", "cores": cores, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": v, "unit": "QP solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": time.perf_counter() - t0}
        print(json.dumps(line))
        return 0

    import torch
    import paper_1506_08435_gb300 as P
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    P.lib()
    barrier(dist)
    if args.workload != "transient3d":
        raise SystemExit("workload %s is run by bench_extra" % args.workload)
    r = run_transient(P, torch, args, rank)
    barrier(dist)
    total_ms = max_over_ranks(dist, sum(r["times"]))
    units = r["units_per_step"] * args.steps * ws
    value = units / (total_ms / 1e3)
    e2e_ms = max_over_ranks(dist, sum(r["e2e"]))
    e2e_val = r["units_per_step"] * len(r["e2e"]) * ws / (e2e_ms / 1e3)
    kern_ms = float(np.mean(r["kern_ms"]))
    kern_bytes = float(np.mean(r["kern_bytes"]))
    achieved = kern_bytes / (kern_ms / 1e3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "transient3d_traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    line = {"metric": "QP solves/s", "value": value, "unit": "QP solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic", "config": r["config"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic,
                         "kernel": "k_solve_grid (persistent GPCG, 50 steps per launch)",
                         "kernel_ms": kern_ms, "algo_bytes_per_launch": kern_bytes, "peak_source": peak_src},
            "e2e": {"value": e2e_val, "unit": "QP solves/s", "h2d_bytes_per_step": r["h2d"],
                    "d2h_bytes_per_step": r["d2h"]},
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "max_kkt_rel": float(max(r["kkt"])),
            "statuses_ok": all(s == 0 for s in r["statuses"]),
            "spmv_per_step": r["spmv"] / args.steps}
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample("transient3d")
        line["cpu_baseline"] = {"value": v, "unit": "QP solves/s", "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
