"""Parity of the projected L-BFGS solver, the batched persistent solve and
the serving loop with the FP64 oracle; alone-vs-in-the-mix equality."""
import math
import os
import time

import numpy as np
import pytest

import nn_inputs as I
from oracle import oracle as O
from tests.gpu_common import compare_solution, oracle_reduced, oracle_solution

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1506_08435_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.lib()


def gpu_system(spec, **kw):
    return P.nn_assemble(P.Problem(spec, device=DEV), P.assemble_opts(**kw))


# ------------------------------------------------------------------ projected L-BFGS

@pytest.mark.parametrize("m", [1, 3, 5])
def test_lbfgs_steady_matches_oracle(m):
    spec = I.config1_steady_2d(n=30)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, P.solve_opts(solver=P.NN_SOLVER_LBFGS, lbfgs_m=m, rtol=1e-11))
    assert info["status"] == 0, info
    red, b, x_ref, _ = oracle_solution(spec)
    compare_solution(c.cpu().numpy()[red.free], x_ref, red.A, b, spec.lo, spec.hi)


@pytest.mark.parametrize("case", ["2d_n4_box", "3d_n3_lower"])
def test_lbfgs_matches_bruteforce(case):
    if case == "2d_n4_box":
        spec = I.tiny_2d(4, 4, hi=1.5e-5)
    else:
        Q = I.quaternion_rotation(I.SplitMix64(2, 0))
        Dm = Q @ np.diag([1000.0, 1.0, 1.0]) @ Q.T
        spec = I.tiny_3d(3, [Dm[0, 0], Dm[0, 1], Dm[0, 2], Dm[1, 1], Dm[1, 2], Dm[2, 2]])
    asm, red = oracle_reduced(spec)
    b = red.rhs()
    (xb, assign), = O.brute_force(red.A, b, spec.lo, spec.hi)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, P.solve_opts(solver=P.NN_SOLVER_LBFGS, rtol=1e-12))
    x = c.cpu().numpy()[red.free]
    assert info["status"] == 0
    active = np.where(x == spec.lo, 1, np.where(x == spec.hi, 2, 0))
    assert np.array_equal(active, assign)
    assert np.abs(x - xb).max() <= 1e-9 * np.abs(xb).max()


def test_lbfgs_transient_matches_gpcg():
    spec = I.config2_transient_3d(n=10, nsteps=4)
    s = gpu_system(spec)
    outs = {}
    for solver in (P.NN_SOLVER_GPCG, P.NN_SOLVER_LBFGS):
        c0 = torch.tensor(spec.c0, device=DEV)
        cf = torch.zeros_like(c0)
        hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
        infos = P.nn_transient(s, c0, spec.nsteps, cf, hist, P.solve_opts(solver=solver, rtol=1e-11))
        assert all(i["status"] == 0 for i in infos)
        outs[solver] = hist.cpu().numpy().reshape(spec.nsteps, -1)
    asm, red = oracle_reduced(spec)
    ref = O.transient(red, spec.c0, spec.lo, spec.hi, spec.nsteps)
    for n in range(spec.nsteps):
        b = red.rhs(ref[n - 1] if n else spec.c0)
        for solver in outs:
            compare_solution(outs[solver][n][red.free], ref[n][red.free], red.A, b, spec.lo, spec.hi)


# ------------------------------------------------------------------ TRON

TRON_SPECS = {
    "steady2d_n30": lambda: I.config1_steady_2d(n=30),
    "steady3d_rot_n12": lambda: I.config3_steady_3d(n=12, seed=5),
    "cube_hole_mirrored_m2": lambda: I.cube_with_hole(2),
}


@pytest.mark.parametrize("ksp", [1e-1, 1e-3])
@pytest.mark.parametrize("name", list(TRON_SPECS))
def test_tron_steady_matches_oracle(name, ksp):
    """TRON with the paper's loosest and tightest subspace tolerances reaches
    the oracle's minimiser (the tolerance changes the path, not the result)."""
    spec = TRON_SPECS[name]()
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, P.solve_opts(solver=P.NN_SOLVER_TRON, ksp_rtol=ksp, rtol=1e-11))
    assert info["status"] == 0, info
    assert info["iterations"] >= 1 and info["cg_iters"] >= 1
    red, b, x_ref, _ = oracle_solution(spec)
    compare_solution(c.cpu().numpy()[red.free], x_ref, red.A, b, spec.lo, spec.hi)


@pytest.mark.parametrize("case", ["2d_n4_box", "3d_n3_lower"])
def test_tron_matches_bruteforce(case):
    if case == "2d_n4_box":
        spec = I.tiny_2d(4, 4, hi=1.5e-5)
    else:
        Q = I.quaternion_rotation(I.SplitMix64(2, 0))
        Dm = Q @ np.diag([1000.0, 1.0, 1.0]) @ Q.T
        spec = I.tiny_3d(3, [Dm[0, 0], Dm[0, 1], Dm[0, 2], Dm[1, 1], Dm[1, 2], Dm[2, 2]])
    asm, red = oracle_reduced(spec)
    b = red.rhs()
    (xb, assign), = O.brute_force(red.A, b, spec.lo, spec.hi)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, P.solve_opts(solver=P.NN_SOLVER_TRON, rtol=1e-12))
    x = c.cpu().numpy()[red.free]
    assert info["status"] == 0
    active = np.where(x == spec.lo, 1, np.where(x == spec.hi, 2, 0))
    assert np.array_equal(active, assign)
    assert np.abs(x - xb).max() <= 1e-9 * np.abs(xb).max()


def test_tron_transient_matches_oracle():
    spec = I.config2_transient_3d(n=10, nsteps=5)
    s = gpu_system(spec)
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    infos = P.nn_transient(s, c0, spec.nsteps, cf, hist, P.solve_opts(solver=P.NN_SOLVER_TRON, rtol=1e-11))
    assert all(i["status"] == 0 for i in infos)
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    asm, red = oracle_reduced(spec)
    ref = O.transient(red, spec.c0, spec.lo, spec.hi, spec.nsteps)
    for n in range(spec.nsteps):
        b = red.rhs(ref[n - 1] if n else spec.c0)
        compare_solution(H[n][red.free], ref[n][red.free], red.A, b, spec.lo, spec.hi)


def test_tron_rejects_unsupported_options():
    spec = I.config1_steady_2d(n=10)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    for kw in (dict(precision=P.NN_PREC_MIXED), dict(format=P.NN_FMT_CSR), dict(ksp_rtol=0.0),
               dict(ksp_rtol=1.0)):
        with pytest.raises(P.NnError) as e:
            P.nn_qp_solve(s, c, P.solve_opts(solver=P.NN_SOLVER_TRON, **kw))
        assert e.value.status == P.NN_ERR_INVALID_ARG
    with pytest.raises(P.NnError) as e:
        P.nn_batch_solve([s], [c], P.solve_opts(solver=P.NN_SOLVER_TRON))
    assert e.value.status == P.NN_ERR_INVALID_ARG


# ------------------------------------------------------------------ batched persistent solve

def _batch(count=24, nmin=12, nmax=40):
    insts = [I.config4_instance(i, nmin=nmin, nmax=nmax) for i in range(count)]
    systems = [gpu_system(sp) for sp in insts]
    return insts, systems


@pytest.mark.parametrize("prec", [P.NN_PREC_FP64, P.NN_PREC_MIXED])
def test_batch_matches_oracle_per_instance(prec):
    insts, systems = _batch()
    cs = [torch.zeros(sp.n_nodes, dtype=torch.float64, device=DEV) for sp in insts]
    infos = P.nn_batch_solve(systems, cs, P.solve_opts(precision=prec, rtol=1e-10))
    assert all(i["status"] == 0 for i in infos), [i["status"] for i in infos]
    for sp, c, inf in zip(insts, cs, infos):
        red, b, x_ref, _ = oracle_solution(sp)
        x = c.cpu().numpy()
        compare_solution(x[red.free], x_ref, red.A, b, sp.lo, sp.hi)
        assert np.array_equal(x[sp.dmask == 1], sp.dval[sp.dmask == 1])
        assert inf["kkt_rel"] <= 1e-10


def test_batch_equals_single_block_solve_alone():
    """An instance gives the same result inside the batch as in a batch of
    one (the same one-block solver, deterministic reductions)."""
    insts, systems = _batch(count=16)
    cs = [torch.zeros(sp.n_nodes, dtype=torch.float64, device=DEV) for sp in insts]
    P.nn_batch_solve(systems, cs)
    for k in (0, 5, 11):
        alone = torch.zeros_like(cs[k])
        P.nn_batch_solve([systems[k]], [alone])
        assert torch.equal(alone, cs[k])


@pytest.mark.parametrize("shape,variant", [("256x4", 0), ("256x8", 0), ("256x16", 0), ("256x8", 1), ("256x8", 2),
                                           ("256x1", 2)])
def test_batch_cluster_shapes_match_oracle(shape, variant, monkeypatch):
    """One thread-block cluster per instance (hardware cluster barrier,
    reductions through distributed shared memory) gives oracle parity, with
    each CG form of the face phase."""
    monkeypatch.setenv("NNQP_BATCH_SHAPE", shape)
    monkeypatch.setenv("NNQP_BATCH_CG_VARIANT", str(variant))
    insts, systems = _batch(count=12, nmin=16, nmax=48)
    cs = [torch.zeros(sp.n_nodes, dtype=torch.float64, device=DEV) for sp in insts]
    for prec in (P.NN_PREC_FP64, P.NN_PREC_MIXED):
        for c in cs:
            c.zero_()
        infos = P.nn_batch_solve(systems, cs, P.solve_opts(precision=prec, rtol=1e-10))
        assert all(i["status"] == 0 for i in infos)
        for sp, c in list(zip(insts, cs))[:4]:
            red, b, x_ref, _ = oracle_solution(sp)
            compare_solution(c.cpu().numpy()[red.free], x_ref, red.A, b, sp.lo, sp.hi)


def test_batch_autotune_picks_a_shape_and_results_hold():
    insts, systems = _batch(count=20)
    best = P.nn_batch_autotune(systems)
    assert best // 100 in (128, 256, 512) and best % 100 in (1, 4, 8, 16)
    cs = [torch.zeros(sp.n_nodes, dtype=torch.float64, device=DEV) for sp in insts]
    infos = P.nn_batch_solve(systems, cs, P.solve_opts(precision=P.NN_PREC_MIXED))
    assert all(i["status"] == 0 for i in infos)
    sp, c = insts[3], cs[3]
    red, b, x_ref, _ = oracle_solution(sp)
    compare_solution(c.cpu().numpy()[red.free], x_ref, red.A, b, sp.lo, sp.hi)


# ------------------------------------------------------------------ serving

def _serve_specs(count=10):
    out = []
    r = 0
    while len(out) < count:
        sp = I.serve_request(r)
        r += 1
        if sp.n_nodes <= 30000:
            out.append(sp)
    return out


def _serve(specs, max_inflight, share=16, budget=8 << 30):
    sv = P.nn_serve_create(budget, P.serve_opts(max_inflight=max_inflight, sm_share_blocks=share))
    ids = [P.nn_serve_submit(sv, P.Problem(sp)) for sp in specs]
    P.nn_serve_drain(sv)
    res = []
    for rid, sp in zip(ids, specs):
        c = np.zeros(sp.n_nodes)
        info = P.nn_serve_poll(sv, rid, c)
        res.append((c, info))
    st = P.nn_serve_stats(sv)
    P.nn_serve_destroy(sv)
    return res, st


def test_serving_results_alone_and_in_the_mix_are_identical_and_correct():
    specs = _serve_specs(10)
    alone, st1 = _serve(specs, max_inflight=1)
    mixed, st8 = _serve(specs, max_inflight=8)
    assert st1["completed"] == st8["completed"] == len(specs)
    assert st8["inflight_peak"] > 1, "requests must overlap on the device"
    assert st1["inflight_peak"] == 1
    for (c1, i1), (c2, i2), sp in zip(alone, mixed, specs):
        assert i1["status"] == 0 and i2["status"] == 0
        assert np.array_equal(c1, c2)          # same grid share, deterministic reductions
    for (c, _), sp in list(zip(mixed, specs))[:4]:
        red, b, x_ref, _ = oracle_solution(sp)
        compare_solution(c[red.free], x_ref, red.A, b, sp.lo, sp.hi)
    assert st8["p50_ms"] > 0 and st8["p99_ms"] >= st8["p50_ms"]


def test_serving_whole_grid_share_concurrent_sizes_all_succeed():
    """Default share (each request may take the whole co-resident grid) with
    several requests of different sizes in flight: the shared-memory operator
    kernel is chosen per request with a different dynamic size on each worker
    thread, and every request must still launch and converge."""
    specs = _serve_specs(12)
    sv = P.nn_serve_create(8 << 30, P.serve_opts(max_inflight=4))
    ids = [P.nn_serve_submit(sv, P.Problem(sp)) for sp in specs]
    P.nn_serve_drain(sv)
    out = []
    for rid, sp in zip(ids, specs):
        c = np.zeros(sp.n_nodes)
        assert P.nn_serve_poll(sv, rid, c)["status"] == 0
        out.append(c)
    st = P.nn_serve_stats(sv)
    P.nn_serve_destroy(sv)
    assert st["completed"] == len(specs) and st["failed"] == 0
    for c, sp in list(zip(out, specs))[:2]:
        red, b, x_ref, _ = oracle_solution(sp)
        compare_solution(c[red.free], x_ref, red.A, b, sp.lo, sp.hi)


def test_serving_budget_admission_and_rejection():
    specs = _serve_specs(6)
    sizes = sorted(sp.n_nodes for sp in specs)
    # a budget that fits one request at a time: admission must serialise them
    sv = P.nn_serve_create(400 << 20, P.serve_opts(max_inflight=8, sm_share_blocks=8))
    ids = [P.nn_serve_submit(sv, P.Problem(sp)) for sp in specs]
    P.nn_serve_drain(sv)
    st = P.nn_serve_stats(sv)
    assert st["completed"] == len(specs)
    assert st["bytes_reserved_peak"] <= st["budget"]
    # measured bytes: never above the estimates admission charged
    assert st["estimate_overruns"] == 0 and 0.0 < st["estimate_max_ratio"] <= 1.0, st
    assert st["bytes_peak"] <= st["bytes_reserved_peak"] <= st["budget"]
    for rid, sp in zip(ids, specs):
        assert P.nn_serve_poll(sv, rid, np.zeros(sp.n_nodes))["status"] == 0
    # a request larger than the whole budget is refused at submit
    big = I.config3_steady_3d(n=60, seed=1)
    with pytest.raises(P.NnError) as e:
        P.nn_serve_submit(sv, P.Problem(big))
    assert e.value.status == P.NN_ERR_INVALID_ARG
    # invalid problems are refused at submit
    bad = I.serve_request(0)
    bad.lo, bad.hi = 1.0, 0.0
    with pytest.raises(P.NnError):
        P.nn_serve_submit(sv, P.Problem(bad))
    P.nn_serve_destroy(sv)


# ------------------------------------------------------------------ reusable plans

def test_plan_launches_equal_single_solves_and_replay_in_a_cuda_graph():
    """A plan's launches (back to back, no allocation, no host sync) and
    their replay from a captured CUDA graph give the same bits as
    nn_qp_solve; a transient plan matches nn_transient."""
    spec = I.config1_steady_2d()
    s = gpu_system(spec)
    ref = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, ref, P.solve_opts())
    assert info["status"] == 0
    plan = P.Plan(s, P.solve_opts())
    zero = torch.zeros_like(ref)
    outs = [torch.empty_like(ref) for _ in range(3)]
    for o in outs:
        plan.launch(zero, o)
    pinfo = plan.result()[0]
    assert pinfo["status"] == 0 and pinfo["spmv"] == info["spmv"]
    for o in outs:
        assert torch.equal(o, ref)
    # capture two launches into a CUDA graph and replay it
    side = torch.cuda.Stream()
    g_out = torch.empty_like(ref)
    side.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        plan.launch(zero, g_out, stream=side)
    for _ in range(3):
        g_out.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(g_out, ref)
    assert plan.result()[0]["status"] == 0
    plan.close()
    # transient
    spec = I.config2_transient_3d(n=10, nsteps=4)
    st = gpu_system(spec)
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    P.nn_transient(st, c0, spec.nsteps, cf, hist)
    tplan = P.Plan(st, P.solve_opts(), nsteps=spec.nsteps)
    cf2 = torch.zeros_like(c0)
    hist2 = torch.zeros_like(hist)
    tplan.launch(c0, cf2, hist2)
    infos = tplan.result()
    assert all(i["status"] == 0 for i in infos) and len(infos) == spec.nsteps
    assert torch.equal(cf2, cf) and torch.equal(hist2, hist)
    tplan.close()


def test_plan_rejects_bad_arguments():
    spec = I.config1_steady_2d(n=10)
    s = gpu_system(spec)
    with pytest.raises(P.NnError):
        P.Plan(s, P.solve_opts(), nsteps=3)   # steady systems take nsteps = 1
    plan = P.Plan(s)
    with pytest.raises(P.NnError):
        plan.launch(None, None)
    plan.close()


def test_serving_mid_size_requests_are_not_co_scheduled_beyond_the_sms():
    """Requests of ~36k nodes get one 512-thread block per SM on 128 SMs:
    two of them do not fit the 152 SMs together, so admission runs them one
    after the other (each grid must be wholly resident to pass its barriers),
    while small requests still run beside each other."""
    mids = [I.config3_steady_3d(n=32, seed=s) for s in (11, 12, 13)]
    sv = P.nn_serve_create(16 << 30, P.serve_opts(max_inflight=4))
    ids = [P.nn_serve_submit(sv, P.Problem(sp)) for sp in mids]
    P.nn_serve_drain(sv)
    st = P.nn_serve_stats(sv)
    outs = []
    for rid, sp in zip(ids, mids):
        c = np.zeros(sp.n_nodes)
        assert P.nn_serve_poll(sv, rid, c)["status"] == 0
        outs.append(c)
    P.nn_serve_destroy(sv)
    assert st["completed"] == 3 and st["failed"] == 0
    assert st["inflight_peak"] == 1, st
    red, b, x_ref, _ = oracle_solution(mids[0], threads=os.cpu_count() or 1)
    compare_solution(outs[0][red.free], x_ref, red.A, b, mids[0].lo, mids[0].hi)
    smalls = [sp for sp in _serve_specs(8) if sp.n_nodes < 15000][:4]
    sv = P.nn_serve_create(16 << 30, P.serve_opts(max_inflight=4))
    ids = [P.nn_serve_submit(sv, P.Problem(sp)) for sp in smalls]
    P.nn_serve_drain(sv)
    st = P.nn_serve_stats(sv)
    P.nn_serve_destroy(sv)
    assert st["completed"] == len(smalls) and st["inflight_peak"] > 1, st


def test_serving_per_request_options_and_measured_bytes_within_the_estimate():
    """Each request carries its own solver options (FP64 or mixed precision,
    tolerance); every result meets the oracle's KKT test, mixed requests
    refine in FP64, and the device bytes each request really held (assembly
    with temporaries, or system + solution + scratch) stay within the
    estimate admission charged for it, over 2D and 3D requests up to ~0.5M
    nodes."""
    specs = [I.serve_request(r) for r in range(40)]
    specs = sorted([sp for sp in specs if sp.n_nodes <= 500_000], key=lambda sp: sp.n_nodes)
    pick = specs[::max(1, len(specs) // 8)][:8] + [specs[-1]]
    sv = P.nn_serve_create(32 << 30, P.serve_opts(max_inflight=4))
    opts = [P.solve_opts(precision=P.NN_PREC_MIXED if k % 2 else P.NN_PREC_FP64, rtol=1e-10) for k in range(len(pick))]
    ids = [P.nn_serve_submit(sv, P.Problem(sp), o) for sp, o in zip(pick, opts)]
    P.nn_serve_drain(sv)
    infos, outs = [], []
    for rid, sp in zip(ids, pick):
        c = np.zeros(sp.n_nodes)
        infos.append(P.nn_serve_poll(sv, rid, c))
        outs.append(c)
    st = P.nn_serve_stats(sv)
    P.nn_serve_destroy(sv)
    assert st["completed"] == len(pick) and st["failed"] == 0
    assert st["estimate_overruns"] == 0 and 0.0 < st["estimate_max_ratio"] <= 1.0, st
    for k, (sp, c, info) in enumerate(zip(pick, outs, infos)):
        assert info["status"] == 0
        assert (info["refinements"] > 0) == (k % 2 == 1), (k, info)
        _, red = oracle_reduced(sp)
        kk = O.kkt(red.A, red.rhs(), sp.lo, sp.hi, c[red.free])
        assert kk["bounds_ok"] and kk["kkt_rel"] <= 1e-8, (k, kk)
    # options are checked at submit
    sv = P.nn_serve_create(1 << 30)
    with pytest.raises(P.NnError) as e:
        P.nn_serve_submit(sv, P.Problem(pick[0]), P.solve_opts(solver=P.NN_SOLVER_LBFGS))
    assert e.value.status == P.NN_ERR_INVALID_ARG
    P.nn_serve_destroy(sv)


def test_auto_precision_picks_fp32_only_for_streaming_operators():
    """NN_PREC_AUTO solves a system whose FP32 operator exceeds the 48 MB
    streaming threshold in mixed precision (refinements in FP64) and a
    smaller one in plain FP64; both meet the oracle's KKT test."""
    for n, mixed in ((20, False), (76, True)):
        spec = I.config3_steady_3d(n=n, seed=3)
        s = gpu_system(spec, build_mixed=1)
        d = s.describe()
        assert (d["nnz_free"] * 8 > 48 * 2 ** 20) == mixed
        c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
        info = P.nn_qp_solve(s, c, P.solve_opts(precision=P.NN_PREC_AUTO))
        assert info["status"] == 0, info
        assert (info["refinements"] > 0) == mixed, (n, info)
        _, red = oracle_reduced(spec)
        x = c.cpu().numpy()[red.free]
        kk = O.kkt(red.A, red.rhs(), spec.lo, spec.hi, x)
        assert kk["bounds_ok"] and kk["kkt_rel"] <= 1e-8, kk
