"""Element-wise parity of the large-system solve path with the FP64 oracle.

Systems above about 32 slices of 32 rows per SM (the 150^3 steady problem
has 106,704 slices) run differently from mid-size ones: one 768-thread block
per SM, the textbook CG form with packed update passes, the FP64 operator
streaming through L2 with evict-first loads and slice prefetches, and the
FP32 operator of mixed inner solves streaming through shared memory by bulk
asynchronous copies.  At full size that path can be checked only through the oracle's KKT
test (the oracle needs hours for a 3.4M-unknown QP).  NNQP_FORCE_LARGE=1
runs a system of any size through exactly that path, so here it is compared
entry by entry with the oracle's minimiser at sizes the oracle solves in
seconds: solution within 1e-6 relative in the max norm, the oracle's KKT
residual of the GPU vector <= 1e-8, bounds exact, active sets equal where
the oracle's solution is strictly complementary (the QP's minimiser is
unique: A is positive definite, Sec. 2.1.3).  Also the projected L-BFGS and
TRON solvers at the 40^3 transient size (its first two backward-Euler
steps), and the mixed-precision path's FP64 fallback."""
import os

import numpy as np
import pytest

import nn_inputs as I
from oracle import oracle as O
from tests.gpu_common import compare_solution, oracle_reduced

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1506_08435_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.lib()


@pytest.fixture(scope="module")
def steady28():
    """The 150^3 problem's field (dispersion rotated per 10^3 block, patch
    Dirichlet data, 0 <= c <= 1) on a 28^3 grid: 24,389 nodes, several
    active bounds at both ends."""
    spec = I.config3_steady_3d(n=28)
    asm, red = oracle_reduced(spec)
    b = red.rhs()
    x, info = O.solve_qp(red.A, b, spec.lo, spec.hi, threads=THREADS)
    assert info["polished"]
    return spec, red, b, x


def solve(spec, **opts):
    s = P.nn_assemble(P.Problem(spec, device=DEV), P.assemble_opts(build_mixed=1))
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    info = P.nn_qp_solve(s, c, P.solve_opts(**opts))
    return c.cpu().numpy(), info


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_large_system_path_matches_oracle_entrywise(prec, steady28, monkeypatch):
    spec, red, b, x_ref = steady28
    monkeypatch.setenv("NNQP_FORCE_LARGE", "1")
    p = P.NN_PREC_MIXED if prec == "mixed" else P.NN_PREC_FP64
    c, info = solve(spec, precision=p)
    assert info["status"] == 0, info
    k, err, degenerate = compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)
    assert info["active_lo"] > 0 and info["active_hi"] > 0
    assert np.array_equal(c[spec.dmask == 1], spec.dval[spec.dmask == 1])
    if prec == "mixed":
        assert info["refinements"] >= 1 and info["fp64_fallback"] == 0, info
    print("large path %s: max error vs oracle %.3e, kkt %.3e, degenerate entries %d"
          % (prec, err, k["kkt_rel"], degenerate))


def test_large_and_default_paths_agree(steady28, monkeypatch):
    """The forced large path and the size-chosen path (here the mid-size one)
    solve the same QP: both within the acceptance of the oracle and of each
    other."""
    spec, red, b, x_ref = steady28
    c_mid, i_mid = solve(spec)
    monkeypatch.setenv("NNQP_FORCE_LARGE", "1")
    c_big, i_big = solve(spec)
    assert i_mid["status"] == 0 and i_big["status"] == 0
    scale = np.abs(x_ref).max()
    assert np.abs(c_mid - c_big).max() <= 2e-6 * scale


def test_mixed_fallback_branch_matches_oracle(steady28, monkeypatch):
    """Inner FP32 solves capped at 30 products cannot contract the FP64
    residual four-fold: the refinement falls back to FP64 GPCG from its
    current iterate, and the result must still be the oracle's minimiser."""
    spec, red, b, x_ref = steady28
    monkeypatch.setenv("NNQP_FORCE_LARGE", "1")
    monkeypatch.setenv("NNQP_INNER_CAP", "30")
    c, info = solve(spec, precision=P.NN_PREC_MIXED)
    assert info["status"] == 0, info
    assert info["fp64_fallback"] == 1, info
    compare_solution(c[red.free], x_ref, red.A, b, spec.lo, spec.hi)


@pytest.mark.parametrize("solver", ["lbfgs", "tron"])
def test_lbfgs_and_tron_at_40_cubed_transient_first_steps(solver):
    """The projected L-BFGS and TRON solvers on the 40^3 transient problem
    (68,921 nodes, one launch for two backward-Euler steps): each step equals
    the oracle's minimiser of that step's QP."""
    spec = I.config2_transient_3d(nsteps=2)
    s = P.nn_assemble(P.Problem(spec, device=DEV))
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    code = P.NN_SOLVER_LBFGS if solver == "lbfgs" else P.NN_SOLVER_TRON
    infos = P.nn_transient(s, c0, spec.nsteps, cf, hist, P.solve_opts(solver=code, rtol=1e-11))
    assert all(i["status"] == 0 for i in infos), infos
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    asm, red = oracle_reduced(spec)
    c = spec.c0
    for n in range(spec.nsteps):
        b = red.rhs(c)
        x, _ = O.solve_qp(red.A, b, spec.lo, spec.hi, x0=c[red.free], threads=THREADS)
        k, err, _ = compare_solution(H[n][red.free], x, red.A, b, spec.lo, spec.hi)
        print("%s step %d: max error vs oracle %.3e kkt %.3e" % (solver, n, err, k["kkt_rel"]))
        c = red.full(x)
