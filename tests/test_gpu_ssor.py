"""The multicolour SSOR preconditioner on the device against the FP64 oracle.

Three levels: the ordering (the colour of every free unknown, bit for bit
the oracle's DSatur colouring), the preconditioner itself (z = M_F^-1 r from
nn_precond_apply, which runs the solve kernels' sweep code, entry by entry
against the oracle's two triangular solves, with and without a face), and
the solves that use it (GPCG's CG phases and TRON's subspace steps with
SSOR: the minimiser equals the oracle's, in FP64, on the mid-size and the
large-system launch shapes and over backward-Euler steps).  The QP's
minimiser does not depend on the preconditioner (it is unique, Sec. 2.1.3),
so the solves must agree with the oracle exactly as the Jacobi ones do."""
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


def ssor(**kw):
    return P.solve_opts(precond=P.NN_PC_SSOR, **kw)


# ------------------------------------------------------------------ ordering

@pytest.mark.parametrize("spec", [I.config1_steady_2d(n=50), I.config3_steady_3d(n=20)], ids=lambda s: s.name)
def test_ordering_is_the_oracle_colouring(spec):
    s = gpu_system(spec)
    before = P.nn_system_describe(s)
    assert before["ssor_colors"] == 0
    P.nn_precond_setup(s)
    d = P.nn_system_describe(s)
    _, red = oracle_reduced(spec)
    col = np.zeros(d["n_free"], np.int32)
    P.nn_system_copy_out(s, "ssor_color", col)
    ref = O.dsatur(red.A)
    assert np.array_equal(col, ref)
    assert d["ssor_colors"] == ref.max() + 1 == (3 if spec.dim == 2 else 4)
    # lower + upper parts hold every off-diagonal once (12 bytes each) at least
    assert d["device_bytes"] - before["device_bytes"] >= 12 * (d["nnz_free"] - d["n_free"])
    P.nn_precond_setup(s)                        # built once
    assert P.nn_system_describe(s)["device_bytes"] == d["device_bytes"]


# ------------------------------------------------------------------ z = M^-1 r

@pytest.mark.parametrize("spec", [I.config3_steady_3d(n=20), I.config3_steady_3d(n=40), I.config1_steady_2d(n=50)],
                         ids=lambda s: s.name)
@pytest.mark.parametrize("omega", [1.0, 1.5])
@pytest.mark.parametrize("with_face", [False, True])
def test_preconditioner_matches_oracle_entrywise(spec, omega, with_face):
    _, red = oracle_reduced(spec)
    n = red.nF
    rng = np.random.default_rng(17)
    r = rng.normal(size=n)
    face = (rng.uniform(size=n) < 0.8).astype(np.uint8) if with_face else None
    ref = O.ssor_apply(red.A, O.dsatur(red.A), r, omega, face=face)
    s = gpu_system(spec)
    z = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
    P.nn_precond_apply(s, torch.tensor(r, device=DEV), z, P.NN_PC_SSOR, omega,
                       torch.tensor(face, device=DEV) if face is not None else None)
    zh = z.cpu().numpy()
    assert np.isfinite(zh).all()
    if face is not None:
        assert np.all(zh[face == 0] == 0.0)
    assert np.abs(zh - ref).max() <= 1e-12 * np.abs(ref).max()


def test_jacobi_preconditioner_is_the_diagonal_scaling():
    spec = I.config3_steady_3d(n=12)
    _, red = oracle_reduced(spec)
    r = np.random.default_rng(3).normal(size=red.nF)
    s = gpu_system(spec)
    z = torch.empty(red.nF, dtype=torch.float64, device=DEV)
    P.nn_precond_apply(s, torch.tensor(r, device=DEV), z, P.NN_PC_JACOBI)
    assert np.abs(z.cpu().numpy() - r / red.A.diagonal()).max() <= 1e-15 * np.abs(r / red.A.diagonal()).max()


def test_preconditioner_argument_checks():
    spec = I.config1_steady_2d(n=10)
    s = gpu_system(spec)
    n = P.nn_system_describe(s)["n_free"]
    r = torch.ones(n, dtype=torch.float64, device=DEV)
    z = torch.empty_like(r)
    for kw in (dict(omega=2.0), dict(omega=0.0), dict(precond=7)):
        with pytest.raises(P.NnError) as e:
            P.nn_precond_apply(s, r, z, **kw)
        assert e.value.status == P.NN_ERR_INVALID_ARG
    with pytest.raises(P.NnError):
        P.nn_precond_apply(s, r, r)


# ------------------------------------------------------------------ solves

@pytest.mark.parametrize("spec", [I.config1_steady_2d(n=50), I.config3_steady_3d(n=20)], ids=lambda s: s.name)
@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_gpcg_with_ssor_matches_oracle(spec, omega):
    red, b, x_ref, _ = oracle_solution(spec)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, ssor(ssor_omega=omega, rtol=1e-11))
    assert info["status"] == 0, info
    assert info["pc_applies"] >= info["cg_iters"] > 0
    k, err, _ = compare_solution(c.cpu().numpy()[red.free], x_ref, red.A, b, spec.lo, spec.hi)
    print("%s SSOR(%.1f): max error vs oracle %.3e, kkt %.3e, %d CG iterations"
          % (spec.name, omega, err, k["kkt_rel"], info["cg_iters"]))


@pytest.mark.parametrize("spec", [I.config1_steady_2d(n=50), I.config3_steady_3d(n=20)], ids=lambda s: s.name)
def test_ssor_needs_fewer_cg_iterations_than_jacobi(spec):
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    ij = P.nn_qp_solve(s, c, P.solve_opts())
    c.zero_()
    iss = P.nn_qp_solve(s, c, ssor())
    assert ij["status"] == 0 and iss["status"] == 0
    assert iss["cg_iters"] < ij["cg_iters"], (iss["cg_iters"], ij["cg_iters"])
    assert ij["pc_applies"] == 0
    print("%s CG iterations: Jacobi %d, SSOR %d" % (spec.name, ij["cg_iters"], iss["cg_iters"]))


def test_large_system_path_with_ssor_matches_oracle(monkeypatch):
    """The 768-thread large-system launch with the SSOR sweeps (forced on a
    mid-size system, as the Jacobi large path is tested)."""
    spec = I.config3_steady_3d(n=24)
    red, b, x_ref, _ = oracle_solution(spec)
    monkeypatch.setenv("NNQP_FORCE_LARGE", "1")
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, ssor())
    assert info["status"] == 0, info
    compare_solution(c.cpu().numpy()[red.free], x_ref, red.A, b, spec.lo, spec.hi)


def test_transient_steps_with_ssor_match_oracle():
    spec = I.config2_transient_3d(n=12, nsteps=3)
    _, red = oracle_reduced(spec)
    ref = O.transient(red, spec.c0, spec.lo, spec.hi, spec.nsteps)
    s = gpu_system(spec)
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    infos = P.nn_transient(s, c0, spec.nsteps, cf, hist, ssor(rtol=1e-11))
    assert all(i["status"] == 0 for i in infos), infos
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    c = spec.c0
    for n in range(spec.nsteps):
        b = red.rhs(c)
        compare_solution(H[n][red.free], ref[n][red.free], red.A, b, spec.lo, spec.hi)
        c = ref[n]


def test_tron_with_ssor_matches_oracle():
    spec = I.config3_steady_3d(n=16)
    red, b, x_ref, _ = oracle_solution(spec)
    s = gpu_system(spec)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, ssor(solver=P.NN_SOLVER_TRON, rtol=1e-11))
    assert info["status"] == 0, info
    assert info["pc_applies"] > 0
    compare_solution(c.cpu().numpy()[red.free], x_ref, red.A, b, spec.lo, spec.hi)


def test_ssor_plan_launches_are_deterministic():
    spec = I.config3_steady_3d(n=16)
    s = gpu_system(spec)
    plan = P.Plan(s, ssor())
    c_in = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    outs = []
    for _ in range(2):
        c = torch.empty_like(c_in)
        plan.launch(c_in, c)
        info = plan.result()
        assert info[0]["status"] == 0
        outs.append(c.clone())
    assert torch.equal(outs[0], outs[1])


def test_ssor_option_combinations():
    spec = I.config3_steady_3d(n=10)
    s = gpu_system(spec, build_mixed=1, build_csr=1)
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    for kw in (dict(precision=P.NN_PREC_MIXED), dict(format=P.NN_FMT_CSR), dict(solver=P.NN_SOLVER_LBFGS),
               dict(ssor_omega=2.0), dict(ssor_omega=-1.0)):
        with pytest.raises(P.NnError) as e:
            P.nn_qp_solve(s, c, ssor(**kw))
        assert e.value.status == P.NN_ERR_INVALID_ARG, kw
    info = P.nn_qp_solve(s, c, ssor(precision=P.NN_PREC_AUTO))   # AUTO is taken as FP64
    assert info["status"] == 0 and info["refinements"] == 0 and info["pc_applies"] > 0
    with pytest.raises(P.NnError) as e:
        P.nn_batch_solve([s], [c], ssor())
    assert e.value.status == P.NN_ERR_INVALID_ARG
    srv = P.nn_serve_create(1 << 30)
    with pytest.raises(P.NnError) as e:
        P.nn_serve_submit(srv, P.Problem(spec), ssor())
    assert e.value.status == P.NN_ERR_INVALID_ARG
    P.nn_serve_destroy(srv)
