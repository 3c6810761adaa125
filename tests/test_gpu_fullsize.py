"""Full-size workloads in the launch configuration the benchmark times,
checked by the oracle: the oracle assembles each system itself (its own
element loop and elimination) and evaluates the FP64 KKT residual of the
GPU's vector, so nothing of the CUDA path enters the check.  A QP solution
is unique (A is positive definite, Sec. 2.1.3), so KKT <= 1e-8 with exact
bounds pins it at any size; a sample of instances is also compared with the
oracle's own solution."""
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
def steady150():
    spec = I.config3_steady_3d(n=150)
    asm, red = oracle_reduced(spec)
    return spec, red, red.rhs()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_ssor"])
def test_steady_3d_150_kkt_by_oracle(prec, steady150):
    """150^3 x 6 tets (3,442,951 nodes): the GPU solution meets the oracle's
    KKT test and the bounds exactly (plain FP64, mixed precision, and FP64
    with the multicolour SSOR preconditioner)."""
    spec, red, b = steady150
    s = P.nn_assemble(P.Problem(spec, device=DEV))
    c = torch.zeros(spec.n_nodes, dtype=torch.float64, device=DEV)
    p = P.NN_PREC_MIXED if prec == "mixed" else P.NN_PREC_FP64
    pc = P.NN_PC_SSOR if prec.endswith("ssor") else P.NN_PC_JACOBI
    info = P.nn_qp_solve(s, c, P.solve_opts(precision=p, precond=pc))
    assert info["status"] == 0, info
    x = c.cpu().numpy()
    del s
    k = O.kkt(red.A, b, spec.lo, spec.hi, x[red.free])
    assert k["bounds_ok"]
    assert k["kkt_rel"] <= 1e-8, k
    assert np.array_equal(x[spec.dmask == 1], spec.dval[spec.dmask == 1])
    assert x.min() >= 0.0 and x.max() <= 1.0


def test_transient_40_every_step_kkt_by_oracle():
    """The 50-step transient run as benchmarked (one launch, projected
    extrapolation as first iterate): every step meets the oracle's KKT test
    for its own right-hand side b = F + M c^(n)/dt - Kt_FD c_D."""
    spec = I.config2_transient_3d()
    s = P.nn_assemble(P.Problem(spec, device=DEV))
    c0 = torch.tensor(spec.c0, device=DEV)
    cf = torch.zeros_like(c0)
    hist = torch.zeros(spec.nsteps * spec.n_nodes, dtype=torch.float64, device=DEV)
    infos = P.nn_transient(s, c0, spec.nsteps, cf, hist)
    assert all(i["status"] == 0 for i in infos)
    H = hist.cpu().numpy().reshape(spec.nsteps, -1)
    asm, red = oracle_reduced(spec)
    prev = spec.c0
    for n in range(spec.nsteps):
        k = O.kkt(red.A, red.rhs(prev), spec.lo, spec.hi, H[n][red.free])
        assert k["bounds_ok"] and k["kkt_rel"] <= 1e-8, (n, k)
        prev = H[n]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_512_kkt_by_oracle_and_sampled_solutions(prec):
    """All 512 instances of the batch in one launch with the autotuned shape:
    every instance meets the oracle's KKT test; 6 of them (the largest, the
    smallest and 4 more) equal the oracle's solution."""
    insts = I.config4_batch(512)
    systems = [P.nn_assemble(P.Problem(sp, device=DEV)) for sp in insts]
    p = P.NN_PREC_MIXED if prec == "mixed" else P.NN_PREC_FP64
    opts = P.solve_opts(precision=p)
    P.nn_batch_autotune(systems, opts)
    cs = [torch.zeros(sp.n_nodes, dtype=torch.float64, device=DEV) for sp in insts]
    infos = P.nn_batch_solve(systems, cs, opts)
    assert all(i["status"] == 0 for i in infos)
    sizes = np.array([sp.n_nodes for sp in insts])
    sample = {int(np.argmax(sizes)), int(np.argmin(sizes)), 7, 100, 301, 499}
    for k, (sp, c) in enumerate(zip(insts, cs)):
        x = c.cpu().numpy()
        asm, red = oracle_reduced(sp)
        b = red.rhs()
        kk = O.kkt(red.A, b, sp.lo, sp.hi, x[red.free])
        assert kk["bounds_ok"] and kk["kkt_rel"] <= 1e-8, (k, kk)
        if k in sample:
            x_ref, _ = O.solve_qp(red.A, b, sp.lo, sp.hi, threads=THREADS)
            compare_solution(x[red.free], x_ref, red.A, b, sp.lo, sp.hi)
