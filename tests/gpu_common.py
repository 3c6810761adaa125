"""Shared helpers of the GPU tests: the same seeded spec goes to the FP64
oracle (CPU) and through the C ABI to the CUDA path."""
import numpy as np

import nn_inputs as I
from oracle import oracle as O


def oracle_reduced(spec, with_mass=None):
    """(assembled, reduced) oracle system of a spec."""
    if spec.coords is not None:
        coords, conn = spec.coords, spec.conn
    else:
        coords, conn = O.mesh_structured(spec.dim, spec.nx, spec.ny, spec.nz)
    wm = spec.dt > 0 if with_mass is None else with_mass
    asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, spec.f_elem,
                     with_mass=wm)
    red = O.Reduced(asm, spec.dmask, spec.dval, dt=spec.dt)
    return asm, red


def oracle_solution(spec, threads=1):
    asm, red = oracle_reduced(spec)
    b = red.rhs()
    x, info = O.solve_qp(red.A, b, spec.lo, spec.hi, threads=threads)
    return red, b, x, info


def active_margin_ok(x, g, lo, hi, bscale, rel=1e-6):
    """Strict complementarity margins of a reference solution: entries off the
    bounds by more than rel*|x|_inf, active gradients above rel*|b|_inf."""
    xs = max(np.abs(x).max(), 1e-300)
    at = (x <= lo) | (x >= hi)
    gap = np.minimum(np.abs(x - lo), np.abs(x - hi))
    return (gap[~at] > rel * xs), (np.abs(g[at]) > rel * bscale)


def compare_solution(x_gpu, x_ref, A, b, lo, hi, tol_sol=1e-6, tol_kkt=1e-8):
    """Acceptance: bounds exact, oracle KKT of the GPU vector <= tol_kkt,
    max-norm error <= tol_sol relative, active sets equal where the
    reference is strictly complementary."""
    k = O.kkt(A, b, lo, hi, x_gpu)
    assert k["bounds_ok"], "an entry left the box"
    assert k["kkt_rel"] <= tol_kkt, k
    err = np.abs(x_gpu - x_ref).max() / max(np.abs(x_ref).max(), 1e-300)
    assert err <= tol_sol, err
    g = A @ x_ref - b
    xs = np.abs(x_ref).max()
    at_ref = (x_ref <= lo) | (x_ref >= hi)
    gap = np.minimum(np.abs(x_ref - lo), np.abs(x_ref - hi))
    clear = np.where(at_ref, np.abs(g) > 1e-6 * np.abs(b).max(), gap > 1e-6 * xs)
    at_gpu = (x_gpu <= lo) | (x_gpu >= hi)
    assert np.array_equal(at_gpu[clear], at_ref[clear]), "active sets differ on nondegenerate entries"
    # entries that are active are exactly at the bound
    assert np.all((x_gpu[at_gpu] == lo) | (x_gpu[at_gpu] == hi))
    return k, err, int((~clear).sum())
