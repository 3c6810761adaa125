"""Host-side logic that needs no GPU: the compact L-BFGS algebra used by the
device solver, the seeded input generator, and the multi-process replica
path of the benchmark (gloo, world size 2)."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import nn_inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1506_08435_gb300", "csrc")


@pytest.fixture(scope="module")
def lbfgs_lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("lb")
    src = d / "lb.cpp"
    src.write_text('#include "lbfgs_small.h"\n'
                   'extern "C" int coef(int k, const double* SY, const double* YY, const double* u,'
                   ' const double* v, double gamma, double* cs, double* cy) {'
                   ' return nnqp::lbfgs_coefficients(k, SY, YY, u, v, gamma, cs, cy) ? 1 : 0; }\n')
    so = d / "lb.so"
    subprocess.check_call(["g++", "-O2", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)])
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.coef.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_double, dp, dp]
    return L


def two_loop(S, Y, g, gamma):
    """Textbook L-BFGS two-loop recursion H g (pairs oldest first)."""
    q = g.copy()
    k = S.shape[1]
    alpha = np.zeros(k)
    for i in range(k - 1, -1, -1):
        rho = 1.0 / (S[:, i] @ Y[:, i])
        alpha[i] = rho * (S[:, i] @ q)
        q -= alpha[i] * Y[:, i]
    r = gamma * q
    for i in range(k):
        rho = 1.0 / (S[:, i] @ Y[:, i])
        beta = rho * (Y[:, i] @ r)
        r += S[:, i] * (alpha[i] - beta)
    return r


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_compact_lbfgs_equals_two_loop(lbfgs_lib, k):
    rng = np.random.default_rng(k)
    n = 30
    B = rng.normal(size=(n, n))
    A = B @ B.T + n * np.eye(n)          # SPD: y = A s gives s'y > 0
    S = rng.normal(size=(n, k))
    Y = A @ S
    g = rng.normal(size=n)
    gamma = (S[:, -1] @ Y[:, -1]) / (Y[:, -1] @ Y[:, -1])
    SY = np.zeros((16, 16))
    YY = np.zeros((16, 16))
    SY[:k, :k] = S.T @ Y
    YY[:k, :k] = Y.T @ Y
    u, v = S.T @ g, Y.T @ g
    cs, cy = np.zeros(16), np.zeros(16)
    p = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    SYc, YYc, uc, vc = [np.ascontiguousarray(a, np.float64) for a in (SY, YY, u, v)]
    assert lbfgs_lib.coef(k, p(SYc), p(YYc), p(uc), p(vc), gamma, cs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          cy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 1
    hg = gamma * g + S @ cs[:k] + Y @ cy[:k]
    ref = two_loop(S, Y, g, gamma)
    assert np.allclose(hg, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_splitmix64_published_vector():
    """SplitMix64 from state 0 (Steele, Lea & Flood 2014): the first outputs
    are 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f."""
    r = I.SplitMix64(0, 0)
    assert [r.u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_inputs_are_deterministic_and_shaped_like_the_workloads():
    a, b = I.config4_instance(17), I.config4_instance(17)
    assert a.nx == b.nx and np.array_equal(a.coef, b.coef) and np.array_equal(a.f_elem, b.f_elem)
    sizes = [I.config4_instance(i).nx for i in range(200)]
    assert min(sizes) >= 20 and max(sizes) <= 200 and len(set(sizes)) > 50
    s = I.config2_transient_3d(n=6)
    assert s.coef.shape == (6 * 6 ** 3, 3) and np.all(np.linalg.norm(s.coef, axis=1) >= 0.1 - 1e-15)
    t = I.serve_arrivals(200.0, 10.0)
    assert 1800 < len(t) < 2200 and all(np.diff(t) > 0)


def test_cube_with_hole_inputs():
    """Node and element counts of the explicit mesh, the Dirichlet sets (outer
    faces 0, hole faces 1) and the mirror x -> 1 - x of the second mesh type."""
    for m in (1, 2, 3):
        n = 9 * m
        k = I.cube_with_hole(m, "kuhn")
        assert k.n_nodes == (n + 1) ** 3 - (m - 1) ** 3
        assert k.n_elems == 6 * (n ** 3 - m ** 3)
        assert k.conn.min() == 0 and k.conn.max() == k.n_nodes - 1
        hole_nodes = (m + 1) ** 3 - (m - 1) ** 3
        outer_nodes = (n + 1) ** 3 - (n - 1) ** 3
        assert int(k.dmask.sum()) == hole_nodes + outer_nodes
        assert int((k.dval == 1.0).sum()) == hole_nodes
        r = I.cube_with_hole(m, "mirrored")
        assert np.array_equal(r.conn, k.conn) and np.array_equal(r.dmask, k.dmask)
        i = np.rint(k.coords[:, 0] * n)
        assert np.array_equal(r.coords[:, 0], (n - i) / n)     # the lattice point, rounded once
        assert np.array_equal(r.coords[:, 1:], k.coords[:, 1:])
    with pytest.raises(ValueError):
        I.cube_with_hole(1, "other")


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the oracle (CPU, no GPU needed) on the
    default workload and prints one JSON line with the contract's keys and
    the same config as the GPU arm."""
    import json
    sys.path.insert(0, ROOT)
    import bench

    def run(*extra):
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                              "--warmup", "0", *extra], capture_output=True, text=True, timeout=600,
                             env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
        assert out.returncode == 0, out.stderr[-800:]
        return json.loads(out.stdout.strip().splitlines()[-1])

    # the default workload's family (steady 3D, rotated dispersion), shrunk
    # to 40^3 so that the oracle's own assembly fits a CPU test
    line = run("--workload", "steady3d", "--n", "40")
    assert line["impl"] == "reference" and line["metric"] == "QP solves/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "MPRGP" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "steady3d_n40" and line["config"]["free"] == 66799
    args = bench.argparse.Namespace(n=40, rtol=1e-10, solver="gpcg", ksp_rtol=0.1, precision="both")
    assert line["config"] == bench.steady3d_config(I.config3_steady_3d(n=40), 40, args)
    line = run("--workload", "transient3d")
    assert line["config"]["workload"] == "transient3d_n40_dt0.01_50steps"
    assert line["config"]["mass"] == "consistent" and line["config"]["solver"] == "gpcg"


def test_profile_traffic_lookup(tmp_path):
    """The bench takes DRAM traffic from a committed ncu summary only while its
    source digest matches, scales a smaller capture by algorithmic bytes (or,
    without them, by products x nnz_free), and otherwise reports null with
    the reason."""
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "k_w_fp64.md").write_text("source_digest: abc\ndram_bytes_per_launch: 1000\n")
    (tmp_path / "k_small_fp64.md").write_text("source_digest: abc\nproducts_per_launch: 10\nnnz_free: 50\n"
                                              "dram_bytes_per_launch: 2000\n")
    assert bench.profile_traffic(str(tmp_path), "k", "w", "fp64", "abc")[0] == 1000.0
    t, why = bench.profile_traffic(str(tmp_path), "k", "w", "fp64", "xyz")
    assert t is None and "changed" in why
    t, why = bench.profile_traffic(str(tmp_path), "k", "big", "fp64", "abc", "small", 30, 100)
    assert t == 2000.0 * 3 * 2 and "scaled" in why
    assert bench.profile_traffic(str(tmp_path), "k", "other", "fp64", "abc")[0] is None
    # a summary with its algorithmic bytes scales by the full launch's algorithmic bytes
    (tmp_path / "k_cap_fp64.md").write_text("source_digest: abc\nproducts_per_launch: 10\nnnz_free: 50\n"
                                            "algo_bytes_per_launch: 4000\ndram_bytes_per_launch: 2000\n")
    t, why = bench.profile_traffic(str(tmp_path), "k", "full", "fp64", "abc", "cap", 30, 100, 20000)
    assert t == 2000.0 * 5 and "algorithmic" in why
    t, why = bench.profile_traffic(str(tmp_path), "k", "full", "fp64", "abc", "cap", 30, 100)
    assert t == 2000.0 * 3 * 2 and "products" in why
    (tmp_path / "k_bad_fp64.md").write_text("source_digest: abc\n")
    assert "incomplete" in bench.profile_traffic(str(tmp_path), "k", "bad", "fp64", "abc")[1]


WORKER = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
d, rank, ws = bench.dist_init()
assert ws == 2
bench.barrier(d)
m = bench.max_over_ranks(d, 10.0 + rank)
# shard independent units across ranks (no data-path collective)
import nn_inputs as I
mine = [I.config4_instance(i, nmin=8, nmax=10).nx for i in range(rank, 6, ws)]
print(json.dumps({"rank": rank, "max": m, "units": len(mine)}))
d.destroy_process_group()
'''


def test_replica_timing_path_world_size_2(tmp_path):
    w = tmp_path / "w.py"
    w.write_text(WORKER)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT="29531", CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(w), ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    import json
    res = [json.loads(o[0].strip().splitlines()[-1]) for o in outs]
    assert all(p.returncode == 0 for p in procs), [o[1][-500:] for o in outs]
    assert all(r["max"] == 11.0 for r in res)
    assert sum(r["units"] for r in res) == 6


def test_oracle_iteration_count_record_or_power_law(tmp_path):
    """The oracle sample of the benchmark scales a timed batch of MPRGP
    iterations by the iteration count of a recorded full oracle run; without
    a record for the grid it extrapolates the records of smaller grids by a
    power law and says so."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    for n, it in ((40, 20000), (80, 40000)):
        (tmp_path / ("steady3d_n%d.json" % n)).write_text(json.dumps({"mprgp_iters": it, "kkt_rel": 1e-14}))
    rec, note = bench.oracle_iterations(40, str(tmp_path))
    assert rec["mprgp_iters"] == 20000 and note is None
    rec, note = bench.oracle_iterations(160, str(tmp_path))
    assert rec["mprgp_iters"] == 80000 and "extrapolated" in note and "n = 40, 80" in note
    rec, note = bench.oracle_iterations(30, str(tmp_path))
    assert rec is None


def test_result_line_carries_the_contract_keys_and_names_the_bound():
    """The JSON line built from one timed run: the contract's keys, the
    roofline with algorithmic and DRAM figures, the FP64 pipe as a second
    roof, and the e2e object."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    infos = [dict(spmv=100, spmv64=100, cg_iters=90, iterations=3, refinements=0, fp64_fallback=0, kkt_rel=1e-11,
                  status=0, flops64_algo=8.0e11, flops_algo=8.0e11)]
    r = dict(times=[1000.0], infos=infos, kern_ms=[990.0], kern_bytes=[5.0e12], units_per_step=1, e2e=[1010.0],
             h2d=123, d2h=45, clocks={"sm_mhz": 2070.0}, launches=3, nnz_free=None, config={"workload": "w"},
             dtype="f64", unit="QP solves/s", metric="QP solves/s")
    args = argparse.Namespace(steps=1, warmup=3)
    line = bench.result_line(r, args, "fp64", None, 1, 6795.5, "measured")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks", "e2e"):
        assert k in line, k
    assert abs(line["value"] - 1.0) < 1e-12 and line["e2e"]["h2d_bytes_per_step"] == 123
    roof = line["roofline"]
    assert roof["unit"] == "GB/s" and abs(roof["achieved"] - 5.0e12 / 0.99 / 1e9) < 1e-6
    assert roof["traffic"] is None and "no ncu summary" in roof["traffic_source"]
    assert line["alu"]["bound"] == "alu" and 0.6 < line["alu"]["frac"] < 0.7
    assert roof["bound"] == "hbm" and "co-bound" in roof["bound_note"]


def test_precision_resolution_of_the_bench():
    sys.path.insert(0, ROOT)
    import argparse
    import bench

    def res(**kw):
        a = dict(workload="steady3d", precision="default", precond="jacobi", serve_precision="auto")
        a.update(kw)
        return bench.resolve_precision(argparse.Namespace(**a)).precision

    assert res() == "both"
    assert res(precond="ssor") == "fp64"
    assert res(workload="transient3d") == "fp64"
    assert res(workload="serve") == "auto"
    assert res(workload="batch", precision="both") == "fp64"
    assert res(precision="mixed") == "mixed"
    assert res(precision="auto", workload="steady2d") == "auto"
