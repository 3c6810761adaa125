"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bit-exact: mesh coordinates/connectivity, CSR patterns, free numbering,
active sets on nondegenerate entries.  Floating point: assembled values to
1e-13 relative to the row's absolute sum; QP solutions to 1e-6 relative in
the max norm with the oracle's KKT residual of the GPU vector <= 1e-8 and
bounds exact (the acceptance of the method's QP, Sec. 2.1.3).
"""
import math
import os

import numpy as np
import scipy.sparse as sps
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


def copy(sys_, what, n, dtype):
    a = np.zeros(n, dtype)
    return P.nn_system_copy_out(sys_, what, a)


def solve_gpu(spec, **opts):
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, P.solve_opts(**opts))
    return s, c.cpu().numpy(), info


# ------------------------------------------------------------------ mesh and pattern

@pytest.mark.parametrize("dim,nx,ny,nz", [(2, 7, 5, 0), (2, 50, 50, 0), (3, 4, 3, 5), (3, 17, 17, 17)])
def test_mesh_bit_exact(dim, nx, ny, nz):
    N, E = P.nn_mesh_counts(dim, nx, ny, nz)
    coords = torch.zeros(N * dim, dtype=torch.float64, device=DEV)
    conn = torch.zeros(E * (dim + 1), dtype=torch.int32, device=DEV)
    P.nn_mesh_structured(dim, nx, ny, nz, coords, conn)
    torch.cuda.synchronize()
    oc, on = O.mesh_structured(dim, nx, ny, nz if dim == 3 else None)
    assert np.array_equal(coords.cpu().numpy(), oc.ravel())
    assert np.array_equal(conn.cpu().numpy(), on.ravel())


SPECS = {
    "steady2d_n50": lambda: I.config1_steady_2d(),
    "steady2d_n23": lambda: I.config1_steady_2d(n=23),
    "transient3d_n9": lambda: I.config2_transient_3d(n=9),
    "steady3d_rot_n12": lambda: I.config3_steady_3d(n=12, seed=5),
    "batch_inst": lambda: I.config4_instance(7, nmin=30, nmax=60),
    "serve2d": lambda: I.serve_request(3),
    "cube_hole_mirrored_m2": lambda: I.cube_with_hole(2),
}


@pytest.mark.parametrize("name", list(SPECS))
def test_assembly_pattern_bit_exact_values_close(name):
    spec = SPECS[name]()
    if spec.n_nodes > 200000:
        pytest.skip("large")
    s = gpu_system(spec)
    d = s.describe()
    asm, red = oracle_reduced(spec, with_mass=True)
    N, nnz = spec.n_nodes, int(asm.rowptr[-1])
    assert d["n_nodes"] == N and d["nnz_full"] == nnz
    assert np.array_equal(copy(s, "K_rowptr", N + 1, np.int64), asm.rowptr)
    assert np.array_equal(copy(s, "K_col", nnz, np.int32), asm.col)
    rabs = np.repeat(np.add.reduceat(np.abs(asm.Kval), asm.rowptr[:-1]), np.diff(asm.rowptr))
    K = copy(s, "K_val", nnz, np.float64)
    assert np.all(np.abs(K - asm.Kval) <= 1e-13 * rabs + 1e-300)
    M = copy(s, "M_val", nnz, np.float64)
    assert np.all(np.abs(M - asm.Mval) <= 1e-14 * np.abs(asm.Mval))
    F = copy(s, "F", N, np.float64)
    assert np.all(np.abs(F - asm.F) <= 1e-14 * max(np.abs(asm.F).max(), 1e-300))
    NF = red.nF
    assert d["n_free"] == NF
    assert np.array_equal(copy(s, "free_node", NF, np.int32), red.free.astype(np.int32))
    A = red.A
    assert d["nnz_free"] == A.nnz
    assert np.array_equal(copy(s, "A_rowptr", NF + 1, np.int64), A.indptr.astype(np.int64))
    assert np.array_equal(copy(s, "A_col", A.nnz, np.int32), A.indices.astype(np.int32))
    Av = copy(s, "A_val", A.nnz, np.float64)
    arabs = np.repeat(np.add.reduceat(np.abs(A.data), A.indptr[:-1]), np.diff(A.indptr))
    assert np.all(np.abs(Av - A.data) <= 1e-13 * arabs)
    b0 = copy(s, "b0", NF, np.float64)
    # transient: b0 = F_F - K_FD c_D is the step right-hand side for a state that
    # is 0 at the free nodes (the M_FD c_D / dt terms cancel), i.e. red.rhs(c_D)
    b_ref = red.rhs(red.full(np.zeros(NF))) if spec.dt > 0 else red.rhs()
    assert np.abs(b0 - b_ref).max() <= 1e-13 * max(np.abs(b_ref).max(), 1e-300) + 1e-300


# ------------------------------------------------------------------ SpMV

@pytest.mark.parametrize("name", ["steady2d_n50", "transient3d_n9", "steady3d_rot_n12"])
def test_spmv_formats_and_precisions(name):
    spec = SPECS[name]()
    s = gpu_system(spec)
    asm, red = oracle_reduced(spec)
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, red.nF)
    y_ref = red.A @ x
    scale = np.abs(red.A) @ np.abs(x)
    xt = torch.tensor(x, device=DEV)
    for fmt in (P.NN_FMT_SELL, P.NN_FMT_CSR):
        y = torch.zeros_like(xt)
        P.nn_spmv(s, xt, y, fmt, P.NN_PREC_FP64)
        torch.cuda.synchronize()
        assert np.all(np.abs(y.cpu().numpy() - y_ref) <= 1e-13 * scale)
    y = torch.zeros_like(xt)
    P.nn_spmv(s, xt, y, P.NN_FMT_SELL, P.NN_PREC_MIXED)
    torch.cuda.synchronize()
    # FP32 values and arithmetic: a few units of 2^-24 of |A||x| per entry
    assert np.all(np.abs(y.cpu().numpy() - y_ref) <= 2e-6 * scale)


# ------------------------------------------------------------------ steady QP

def test_qp_steady_2d_config():
    spec = I.config1_steady_2d()
    s, c, info = solve_gpu(spec, rtol=1e-10)
    assert info["status"] == 0
    red, b, x_ref, _ = oracle_solution(spec)
    k, err, degenerate = compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)
    assert np.array_equal(c[spec.dmask == 1], spec.dval[spec.dmask == 1])
    assert info["active_lo"] == int((c[red.free] == 0.0).sum()) > 0
    k2 = P.nn_kkt_residual(s, torch.tensor(c, device=DEV))
    # two FP64 evaluations of a residual near 1e-11 differ in the cancellation of Ax - b
    assert k2["kkt_rel"] == pytest.approx(k["kkt_rel"], rel=1e-3, abs=1e-15) and k2["bounds_ok"]
    assert info["kkt_rel"] <= 1e-10


@pytest.mark.parametrize("opts", [dict(format=P.NN_FMT_CSR), dict(precision=P.NN_PREC_MIXED),
                                  dict(grid_blocks=3), dict(grid_blocks=1)])
def test_qp_steady_2d_variants(opts):
    spec = I.config1_steady_2d(n=40)
    s, c, info = solve_gpu(spec, rtol=1e-10, **opts)
    assert info["status"] == 0, info
    red, b, x_ref, _ = oracle_solution(spec)
    compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)
    if opts.get("precision") == P.NN_PREC_MIXED:
        assert info["refinements"] >= 1 and info["spmv"] > info["spmv64"]


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("prec", [P.NN_PREC_FP64, P.NN_PREC_MIXED])
def test_cg_variants_reach_the_oracle_solution(variant, prec, monkeypatch):
    """Every CG form of the face phase (textbook, Chronopoulos-Gear,
    pipelined) gives the oracle's solution, steady and transient."""
    monkeypatch.setenv("NNQP_CG_VARIANT", str(variant))
    spec = I.config1_steady_2d(n=40)
    s, c, info = solve_gpu(spec, rtol=1e-10, precision=prec)
    assert info["status"] == 0, info
    red, b, x_ref, _ = oracle_solution(spec)
    compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)
    spec = I.config2_transient_3d(n=8, nsteps=3)
    st = gpu_system(spec)
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    infos = P.nn_transient(st, c0, spec.nsteps, cf, hist, P.solve_opts(rtol=1e-11, precision=prec))
    assert all(i["status"] == 0 for i in infos)
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    asm, red = oracle_reduced(spec)
    ref = O.transient(red, spec.c0, spec.lo, spec.hi, spec.nsteps)
    for n in range(spec.nsteps):
        b = red.rhs(ref[n - 1] if n else spec.c0)
        compare_solution(H[n][red.free], ref[n][red.free], red.A, b, spec.lo, spec.hi)


@pytest.mark.parametrize("case", ["2d_n4_lower", "2d_n4_box", "3d_n3_lower", "2d_4x5_lower"])
@pytest.mark.parametrize("prec", [P.NN_PREC_FP64, P.NN_PREC_MIXED])
def test_qp_matches_bruteforce(case, prec):
    if case == "2d_n4_lower":
        spec = I.tiny_2d(4, 4)
    elif case == "2d_n4_box":
        spec = I.tiny_2d(4, 4, hi=1.5e-5)
    elif case == "3d_n3_lower":
        Q = I.quaternion_rotation(I.SplitMix64(2, 0))
        Dm = Q @ np.diag([1000.0, 1.0, 1.0]) @ Q.T
        spec = I.tiny_3d(3, [Dm[0, 0], Dm[0, 1], Dm[0, 2], Dm[1, 1], Dm[1, 2], Dm[2, 2]])
    else:
        spec = I.tiny_2d(4, 5, theta=0.3, source_cell=(1, 2))
    asm, red = oracle_reduced(spec)
    b = red.rhs()
    sols = O.brute_force(red.A, b, spec.lo, spec.hi)
    assert len(sols) == 1
    xb, assign = sols[0]
    s, c, info = solve_gpu(spec, rtol=1e-12, precision=prec)
    x = c[red.free]
    assert info["status"] == 0
    active = np.where(x == spec.lo, 1, np.where(x == spec.hi, 2, 0))
    assert np.array_equal(active, assign)
    assert np.abs(x - xb).max() <= 1e-9 * np.abs(xb).max()


def test_qp_3d_rotated_dispersion():
    spec = I.config3_steady_3d(n=16, seed=9)
    for prec in (P.NN_PREC_FP64, P.NN_PREC_MIXED):
        s, c, info = solve_gpu(spec, rtol=1e-10, precision=prec)
        assert info["status"] == 0, info
        if prec == P.NN_PREC_FP64:
            red, b, x_ref, _ = oracle_solution(spec)
        compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)
        assert c.max() <= 1.0 and c.min() >= 0.0


def test_qp_is_deterministic_and_warm_start_is_cheap():
    spec = I.config1_steady_2d(n=30)
    s = gpu_system(spec)
    c1 = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    c2 = torch.zeros_like(c1)
    i1 = P.nn_qp_solve(s, c1)
    i2 = P.nn_qp_solve(s, c2)
    assert torch.equal(c1, c2) and i1["spmv"] == i2["spmv"]
    i3 = P.nn_qp_solve(s, c1)          # warm start at the solution
    assert i3["spmv"] <= 3 and torch.equal(c1, c2)


def test_host_memory_round_trip():
    spec = I.config1_steady_2d(n=20)
    s = P.nn_assemble(P.Problem(spec))             # host arrays
    c = np.zeros(spec.n_nodes)
    info = P.nn_qp_solve(s, c)
    red, b, x_ref, _ = oracle_solution(spec)
    compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)
    k = P.nn_kkt_residual(s, c)
    assert k["kkt_rel"] <= 1e-10 and k["bounds_ok"]


def test_not_converged_returns_feasible_iterate():
    spec = I.config1_steady_2d(n=30)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, P.solve_opts(max_iter=4))
    assert info["status"] == P.NN_ERR_NOT_CONVERGED
    assert float(c.min()) >= 0.0


# ------------------------------------------------------------------ transient

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shared_memory_operator_gives_identical_steps(prec, monkeypatch):
    """Mid-size solves keep each block's operator slices in shared memory; the
    products do the same arithmetic in the same order as from global memory,
    so every step is bit-identical, and each meets the oracle's KKT test."""
    spec = I.config2_transient_3d(n=30, nsteps=5)
    s = gpu_system(spec)
    p = P.NN_PREC_MIXED if prec == "mixed" else P.NN_PREC_FP64
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("NNQP_SMEM_OP", flag)
        c0 = torch.tensor(spec.c0, device=DEV)
        cf = torch.zeros_like(c0)
        hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
        infos = P.nn_transient(s, c0, spec.nsteps, cf, hist, P.solve_opts(precision=p))
        assert all(i["status"] == 0 for i in infos)
        out[flag] = hist.cpu().numpy().reshape(spec.nsteps, -1)
    assert np.array_equal(out["1"], out["0"])
    asm, red = oracle_reduced(spec)
    prev = spec.c0
    for n in range(spec.nsteps):
        k = O.kkt(red.A, red.rhs(prev), spec.lo, spec.hi, out["1"][n][red.free])
        assert k["bounds_ok"] and k["kkt_rel"] <= 1e-8
        prev = out["1"][n]


@pytest.mark.parametrize("extrapolate,prec", [(0, "fp64"), (1, "fp64"), (2, "fp64"), (1, "mixed")])
def test_transient_small_matches_oracle_trajectory(extrapolate, prec):
    """Either first iterate (c^(n), or the projected extrapolation
    2 c^(n) - c^(n-1)) and either precision (FP64, or FP32 inner solves
    refined in FP64) reach the oracle's step solution."""
    spec = I.config2_transient_3d(n=10, nsteps=8)
    s = gpu_system(spec)
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    p = P.NN_PREC_MIXED if prec == "mixed" else P.NN_PREC_FP64
    infos = P.nn_transient(s, c0, spec.nsteps, cf, hist,
                           P.solve_opts(rtol=1e-11, extrapolate=extrapolate, precision=p))
    assert all(i["status"] == 0 for i in infos)
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    assert np.array_equal(H[-1], cf.cpu().numpy())
    asm, red = oracle_reduced(spec)
    ref = O.transient(red, spec.c0, spec.lo, spec.hi, spec.nsteps)
    prev = spec.c0
    for n in range(spec.nsteps):
        b = red.rhs(ref[n - 1] if n else spec.c0)
        compare_solution(H[n][red.free], ref[n][red.free], red.A, b, spec.lo, spec.hi)
        # the GPU step is also the KKT point of its own step problem (any size property)
        k = P.nn_kkt_residual(s, torch.tensor(H[n], device=DEV), torch.tensor(prev, device=DEV))
        assert k["kkt_rel"] <= 1e-10 and k["bounds_ok"]
        prev = H[n]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_transient_lumped_mass_matches_oracle(prec):
    """Row-sum lumped capacity matrix: the assembled M (diagonal, zero
    off-diagonal entries kept on the pattern), the reduced operator and the
    transient trajectory agree with the oracle's lumped variant."""
    spec = I.config2_transient_3d(n=10, nsteps=6)
    s = gpu_system(spec, lumped_mass=1)
    coords, conn = O.mesh_structured(3, spec.nx, spec.ny, spec.nz)
    asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, spec.f_elem,
                     with_mass=True, lumped=True)
    red = O.Reduced(asm, spec.dmask, spec.dval, dt=spec.dt)
    nnz = int(asm.rowptr[-1])
    M = copy(s, "M_val", nnz, np.float64)
    assert np.all(np.abs(M - asm.Mval) <= 1e-14 * np.abs(asm.Mval))
    assert np.count_nonzero(M) == spec.n_nodes
    # the device keeps the structural pattern; the oracle's sparse sum K + M_L/dt
    # drops entries that are exactly zero, so compare the operators, not arrays
    d = s.describe()
    NF, nnzF = d["n_free"], d["nnz_free"]
    Ag = sps.csr_matrix((copy(s, "A_val", nnzF, np.float64), copy(s, "A_col", nnzF, np.int32),
                         copy(s, "A_rowptr", NF + 1, np.int64)), shape=(NF, NF))
    rs = np.abs(red.A).sum(axis=1).A1
    diff = abs(Ag - red.A).max(axis=1).toarray().ravel()
    assert np.all(diff <= 1e-13 * rs)
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    p = P.NN_PREC_MIXED if prec == "mixed" else P.NN_PREC_FP64
    infos = P.nn_transient(s, c0, spec.nsteps, cf, hist, P.solve_opts(rtol=1e-11, precision=p))
    assert all(i["status"] == 0 for i in infos)
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    ref = O.transient(red, spec.c0, spec.lo, spec.hi, spec.nsteps)
    for n in range(spec.nsteps):
        b = red.rhs(ref[n - 1] if n else spec.c0)
        compare_solution(H[n][red.free], ref[n][red.free], red.A, b, spec.lo, spec.hi)
    # the consistent and lumped trajectories differ (the flag reached the kernel)
    sc = gpu_system(spec)
    cc = torch.zeros_like(c0)
    P.nn_transient(sc, c0, spec.nsteps, cc, None, P.solve_opts(rtol=1e-11))
    assert np.abs(cc.cpu().numpy() - H[-1]).max() > 1e-4


def test_assembly_rejects_unknown_mass_flag():
    with pytest.raises(P.NnError) as e:
        gpu_system(I.config2_transient_3d(n=4, nsteps=1), lumped_mass=2)
    assert e.value.status == P.NN_ERR_INVALID_ARG


@pytest.mark.parametrize("mesh", ["kuhn", "mirrored"])
def test_cube_hole_qp_and_galerkin_match_oracle(mesh):
    """Cube with a hole on an explicit mesh: the device QP solution matches
    the oracle's, and the same system solved without bounds (lo = -inf,
    hi = +inf: GPCG reduces to preconditioned CG) is the Galerkin solution,
    which leaves [0, 1] on the mirrored mesh only."""
    import dataclasses
    spec = I.cube_with_hole(2, mesh)
    s, c, info = solve_gpu(spec)
    assert info["status"] == 0
    red, b, x_ref, _ = oracle_solution(spec)
    compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)
    free_spec = dataclasses.replace(spec, lo=-math.inf, hi=math.inf)
    _, cg, ginfo = solve_gpu(free_spec)
    assert ginfo["status"] == 0
    xg = O.galerkin(red.A, b)
    assert np.abs(cg[red.free] - xg).max() <= 1e-8 * np.abs(xg).max()
    if mesh == "mirrored":
        assert cg.min() < -0.01
    else:
        assert cg.min() >= -1e-12


def test_sell_padding_equals_the_pattern_count_on_the_cube_with_a_hole():
    """The library's SELL-32 storage of A holds the off-diagonals plus the
    padding of 32-row slices with even widths, computed here from the
    oracle's matrix: the small padding that leaves no room for sigma-sorting
    on these meshes (rows near the hole are shorter)."""
    spec = I.cube_with_hole(4)
    s = gpu_system(spec)
    d = s.describe()
    _, red = oracle_reduced(spec)
    off = np.diff(red.A.indptr) - 1
    w = np.zeros(((len(off) + 31) // 32) * 32, np.int64)
    w[:len(off)] = off
    w = w.reshape(-1, 32).max(axis=1)
    assert d["sell_stored"] == 32 * int((w + (w & 1)).sum())
    assert d["sell_stored"] <= 1.03 * (d["nnz_free"] - d["n_free"])


def test_transient_step_api_equals_batched_steps():
    spec = I.config2_transient_3d(n=8, nsteps=3)
    s = gpu_system(spec)
    c = torch.tensor(spec.c0, device=DEV)
    outs = []
    for _ in range(3):
        nxt = torch.zeros_like(c)
        P.nn_step(s, c, nxt)
        outs.append(nxt)
        c = nxt
    cf = torch.zeros_like(c)
    hist = torch.zeros(3 * spec.n_nodes, dtype=torch.float64, device=DEV)
    # nn_step starts each QP from c^(n); so does nn_transient without extrapolation
    P.nn_transient(s, torch.tensor(spec.c0, device=DEV), 3, cf, hist, P.solve_opts(extrapolate=0))
    H = hist.view(3, -1)
    for n in range(3):
        assert torch.equal(H[n], outs[n])


def test_transient_full_config_first_steps_and_kkt_every_step():
    spec = I.config2_transient_3d()
    s = gpu_system(spec)
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    infos = P.nn_transient(s, c0, spec.nsteps, cf, hist)
    assert all(i["status"] == 0 for i in infos)
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    assert H.min() >= 0.0 and H.max() <= 1.0
    asm, red = oracle_reduced(spec)
    nthreads = os.cpu_count() or 1
    c = spec.c0
    for n in range(2):
        b = red.rhs(c)
        x, _ = O.solve_qp(red.A, b, spec.lo, spec.hi, x0=c[red.free], threads=nthreads)
        compare_solution(H[n][red.free], x, red.A, b, spec.lo, spec.hi)
        c = red.full(x)
    prev = spec.c0
    for n in range(spec.nsteps):
        k = P.nn_kkt_residual(s, torch.tensor(H[n], device=DEV), torch.tensor(prev, device=DEV))
        assert k["kkt_rel"] <= 1e-8 and k["bounds_ok"]
        prev = H[n]


# ------------------------------------------------------------------ invalid input and bounded waits

def test_invalid_inputs_are_rejected_and_library_stays_usable():
    base = I.config1_steady_2d(n=6)
    bad = I.config1_steady_2d(n=6)
    bad.lo, bad.hi = 1.0, 0.0
    with pytest.raises(P.NnError) as e:
        gpu_system(bad)
    assert e.value.status == P.NN_ERR_INFEASIBLE
    bad = I.config1_steady_2d(n=6)
    bad.hi = 1.0
    bad.dval = bad.dval + 2.0
    with pytest.raises(P.NnError) as e:
        gpu_system(bad)
    assert e.value.status == P.NN_ERR_INFEASIBLE
    bad = I.config1_steady_2d(n=6)
    bad.coef = bad.coef.copy()
    bad.coef[5] = [1.0, 2.0, 1.0]
    with pytest.raises(P.NnError) as e:
        gpu_system(bad)
    assert e.value.status == P.NN_ERR_NOT_SPD
    bad = I.config1_steady_2d(n=6)
    bad.coef = bad.coef.copy()
    bad.coef[3, 1] = math.nan
    with pytest.raises(P.NnError) as e:
        gpu_system(bad)
    assert e.value.status == P.NN_ERR_NUMERIC
    # explicit meshes: out-of-range connectivity, zero-measure element
    coords, conn = O.mesh_structured(2, 3)
    spec = I.tiny_2d(3, 3)
    spec.coords, spec.conn = coords, conn.copy()
    spec.conn[2, 1] = 10_000
    with pytest.raises(P.NnError) as e:
        gpu_system(spec)
    assert e.value.status == P.NN_ERR_INVALID_ARG
    spec.conn = conn.copy()
    spec.conn[4] = [0, 1, 2]          # three collinear nodes on the bottom edge
    with pytest.raises(P.NnError) as e:
        gpu_system(spec)
    assert e.value.status == P.NN_ERR_DEGENERATE
    # an explicit mesh equal to the structured one gives the same solution
    spec.conn = conn
    s1, c1, _ = solve_gpu(spec)
    spec2 = I.tiny_2d(3, 3)
    s2, c2, _ = solve_gpu(spec2)
    assert np.array_equal(c1, c2)
    s, c, info = solve_gpu(base)
    assert info["status"] == 0
    # every node a Dirichlet node: no unknowns, refused (the solution is the data)
    empty = I.config1_steady_2d(n=1)
    assert (empty.dmask == 1).all()
    with pytest.raises(P.NnError) as e:
        gpu_system(empty)
    assert e.value.status == P.NN_ERR_INVALID_ARG
    s, c, info = solve_gpu(base)
    assert info["status"] == 0


def test_bounded_wait_times_out_with_status(monkeypatch):
    spec = I.config1_steady_2d(n=20)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    monkeypatch.setenv("NNQP_TEST_STALL_BARRIER", "1")
    with pytest.raises(P.NnError) as e:
        P.nn_qp_solve(s, c, P.solve_opts(wait_timeout_s=0.2))
    assert e.value.status == P.NN_ERR_TIMEOUT
    monkeypatch.delenv("NNQP_TEST_STALL_BARRIER")
    info = P.nn_qp_solve(s, c)
    assert info["status"] == 0
