"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook
element matrices, hand-derived stencils, closed forms, invariants of the
continuous and discrete problems, exact brute force on tiny meshes, and a
second, independent solver.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import nn_inputs as I
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_matrices(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        r, c = int(tok[1]), int(tok[2])
        out[tok[0]] = np.array([float(t) for t in tok[3:]]).reshape(r, c)
    return out


def load_scalars(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


def build(spec, with_mass=False):
    coords, conn = O.mesh_structured(spec.dim, spec.nx, spec.ny, spec.nz)
    asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, spec.f_elem,
                     with_mass=with_mass)
    return coords, conn, asm


# ------------------------------------------------------------------ mesh

@pytest.mark.parametrize("n", [1, 2, 5, 13])
def test_mesh_counts_and_pattern_size_2d(n):
    coords, conn = O.mesh_structured(2, n)
    assert coords.shape == ((n + 1) ** 2, 2) and conn.shape == (2 * n * n, 3)
    rowptr, col = O.pattern(len(coords), conn)
    edges = 2 * n * (n + 1) + n * n
    assert rowptr[-1] == (n + 1) ** 2 + 2 * edges


@pytest.mark.parametrize("n", [1, 2, 4, 7])
def test_mesh_counts_and_pattern_size_3d(n):
    coords, conn = O.mesh_structured(3, n)
    assert coords.shape == ((n + 1) ** 3, 3) and conn.shape == (6 * n ** 3, 4)
    rowptr, col = O.pattern(len(coords), conn)
    edges = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    assert rowptr[-1] == (n + 1) ** 3 + 2 * edges
    lens = np.diff(rowptr)
    if n >= 3:
        assert lens.max() == 15          # interior rows of the Kuhn split


def test_mesh_elements_tile_the_domain():
    """Every element has positive measure, measures sum to 1 and every
    centroid lies in its own lattice cell (no element outside the box)."""
    for dim, n in [(2, 7), (3, 5)]:
        coords, conn = O.mesh_structured(dim, n)
        X = coords[conn]                                # [E, d+1, d]
        J = X[:, 1:, :] - X[:, :1, :]
        vol = np.abs(np.linalg.det(J)) / math.factorial(dim)
        assert (vol > 0).all()
        assert abs(vol.sum() - 1.0) < 1e-13
        assert np.allclose(vol, 1.0 / (math.factorial(dim) * n ** dim))
        cen = X.mean(axis=1)
        assert (cen > 0).all() and (cen < 1).all()


def test_mesh_lattice_numbering():
    coords, conn = O.mesh_structured(3, 4, 5, 6)
    i, j, k = 3, 2, 5
    v = i + 5 * (j + 6 * k)
    assert np.array_equal(coords[v], [i / 4, j / 5, k / 6])
    hex_id = 1 + 4 * (2 + 5 * 3)
    t = conn[6 * hex_id + 3]                            # permutation (y, z, x)
    v0 = 1 + 5 * (2 + 6 * 3)
    assert list(t) == [v0, v0 + 5, v0 + 5 + 30, v0 + 5 + 30 + 1]


# ------------------------------------------------------------------ element matrices

def single_element(dim):
    if dim == 2:
        coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
        conn = np.array([[0, 1, 2]], np.int32)
        coef = np.array([[1.0, 0.0, 1.0]])
    else:
        coords = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
        conn = np.array([[0, 1, 2, 3]], np.int32)
        coef = np.array([[1.0, 0, 0, 1, 0, 1]])
    return O.assemble(coords, conn, I.KIND_TENSOR, coef, f_elem=np.ones(1), with_mass=True)


@pytest.mark.parametrize("dim,tag", [(2, "tri"), (3, "tet")])
def test_reference_element_matrices(dim, tag):
    g = load_matrices("p1_reference_elements.txt")
    asm = single_element(dim)
    assert np.allclose(asm.K.toarray(), g["K_" + tag], rtol=0, atol=1e-15)
    assert np.allclose(asm.M.toarray(), g["M_" + tag], rtol=0, atol=1e-16)
    assert np.allclose(asm.F, g["F_" + tag].ravel(), rtol=0, atol=1e-16)


def test_element_matrices_affine_covariance():
    """Mapping the reference triangle by x -> Bx + t with D = B B^T gives
    the reference D = I stiffness scaled by |det B| (change of variables)."""
    B = np.array([[2.0, 0.5], [0.3, 1.5]])
    ref = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    coords = ref @ B.T + np.array([0.7, -0.2])
    Dm = B @ B.T
    coef = np.array([[Dm[0, 0], Dm[0, 1], Dm[1, 1]]])
    asm = O.assemble(coords, np.array([[0, 1, 2]], np.int32), I.KIND_TENSOR, coef, with_mass=True)
    g = load_matrices("p1_reference_elements.txt")
    det = abs(np.linalg.det(B))
    assert np.allclose(asm.K.toarray(), det * g["K_tri"], atol=1e-13)
    assert np.allclose(asm.M.toarray(), det * g["M_tri"], atol=1e-15)


def test_dispersion_law():
    """D = (aT|v| + DM) I + (aL - aT) v v^T / |v| (Sec. 5): on one element
    the velocity form must equal the tensor form with that D."""
    v = np.array([0.3, -0.4, 1.2])
    aL, aT, DM = 1.0, 1e-3, 1e-9
    vn = np.linalg.norm(v)
    Dm = (aT * vn + DM) * np.eye(3) + (aL - aT) * np.outer(v, v) / vn
    coords = np.array([[0.0, 0, 0], [0.9, 0.1, 0], [0.2, 1.1, 0.1], [0.1, 0.2, 0.8]])
    conn = np.array([[0, 1, 2, 3]], np.int32)
    a1 = O.assemble(coords, conn, I.KIND_VELOCITY, v[None], aL, aT, DM)
    a2 = O.assemble(coords, conn, I.KIND_TENSOR,
                    np.array([[Dm[0, 0], Dm[0, 1], Dm[0, 2], Dm[1, 1], Dm[1, 2], Dm[2, 2]]]))
    assert np.allclose(a1.K.toarray(), a2.K.toarray(), rtol=1e-14, atol=0)
    # eigen-structure: v is an eigenvector with eigenvalue aL|v| + DM
    assert np.allclose(Dm @ v, (aL * vn + DM) * v)


# ------------------------------------------------------------------ P1: symmetry, zero row sums

@pytest.mark.parametrize("which", ["2d", "3d"])
def test_symmetric_zero_row_sum_and_mass(which):
    if which == "2d":
        spec = I.config1_steady_2d(n=12)
    else:
        spec = I.config3_steady_3d(n=10, seed=7)
    _, _, asm = build(spec, with_mass=True)
    K, M = asm.K, asm.M
    assert abs(K - K.T).max() <= 1e-13 * abs(K).max()
    rs = np.asarray(K.sum(axis=1)).ravel()
    ra = np.asarray(abs(K).sum(axis=1)).ravel()
    assert (np.abs(rs) <= 1e-13 * ra).all()
    assert abs(M - M.T).max() == 0.0
    assert (M.data > 0).all()
    assert abs(M.sum() - 1.0) < 1e-13


# ------------------------------------------------------------------ P2 / P3: closed-form stencils

def test_stencil_2d_rotated_tensor_closed_form():
    g = load_scalars("stencil_2d_rotated.txt")
    n = 9
    spec = I.config1_steady_2d(n=n)
    _, _, asm = build(spec)
    K = asm.K.toarray()
    for (i, j) in [(3, 4), (1, 1), (7, 7)]:
        p = i + (n + 1) * j
        nb = lambda di, dj: p + di + (n + 1) * dj
        assert K[p, nb(1, 0)] == pytest.approx(g["east_west"], rel=1e-12)
        assert K[p, nb(-1, 0)] == pytest.approx(g["east_west"], rel=1e-12)
        assert K[p, nb(0, 1)] == pytest.approx(g["north_south"], rel=1e-12)
        assert K[p, nb(0, -1)] == pytest.approx(g["north_south"], rel=1e-12)
        assert K[p, nb(1, 1)] == pytest.approx(g["diag_ne_sw"], rel=1e-12)
        assert K[p, nb(-1, -1)] == pytest.approx(g["diag_ne_sw"], rel=1e-12)
        assert K[p, p] == pytest.approx(g["center"], rel=1e-12)
        row = asm.col[asm.rowptr[p]:asm.rowptr[p + 1]]
        assert nb(1, -1) not in row and nb(-1, 1) not in row and len(row) == 7
    # D = I: the 5-point Laplacian
    E = 2 * n * n
    asm = O.assemble(*O.mesh_structured(2, n), I.KIND_TENSOR, np.tile([1.0, 0.0, 1.0], (E, 1)))
    K = asm.K.toarray()
    p = 4 + (n + 1) * 4
    assert K[p, p] == pytest.approx(4.0, abs=1e-14)
    for q in (p + 1, p - 1, p + n + 1, p - n - 1):
        assert K[p, q] == pytest.approx(-1.0, abs=1e-14)
    assert abs(K[p, p + n + 2]) < 1e-14


def test_stencil_3d_kuhn_laplacian_closed_form():
    """Kuhn split with D = I: interior row = h * (7-point Laplacian), and the
    8 other structural neighbours carry exactly 0 (to roundoff)."""
    n = 6
    h = 1.0 / n
    E = 6 * n ** 3
    asm = O.assemble(*O.mesh_structured(3, n), I.KIND_TENSOR, np.tile([1.0, 0, 0, 1, 0, 1], (E, 1)))
    for (i, j, k) in [(2, 3, 3), (1, 1, 1), (4, 2, 5)]:
        p = i + (n + 1) * (j + (n + 1) * k)
        cols = asm.col[asm.rowptr[p]:asm.rowptr[p + 1]]
        vals = asm.Kval[asm.rowptr[p]:asm.rowptr[p + 1]]
        assert len(cols) == 15
        axis = {p + 1, p - 1, p + n + 1, p - n - 1, p + (n + 1) ** 2, p - (n + 1) ** 2}
        for c, v in zip(cols, vals):
            if c == p:
                assert v == pytest.approx(6 * h, rel=1e-13)
            elif c in axis:
                assert v == pytest.approx(-h, rel=1e-13)
            else:
                assert abs(v) < 1e-15


# ------------------------------------------------------------------ P4: loads

def test_load_sum_equals_source_integral():
    spec = I.config1_steady_2d(n=50)
    _, _, asm = build(spec)
    ntri = spec.f_elem.sum()
    assert asm.F.sum() == pytest.approx(ntri * (1.0 / 50) ** 2 / 2, rel=1e-13)
    # the box [3/8, 5/8]^2 holds 12.5 x 12.5 squares: 2 * 12 * 12 + edge rows
    assert ntri > 0 and ntri < 2 * 13 * 13


# ------------------------------------------------------------------ patch test (assembly + lifting + solver)

@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_linear_solution_is_exact(dim):
    """With constant D and f = 0, the P1 Galerkin solution equals a linear
    field prescribed on the whole boundary (the FE patch test).  The field is
    positive, so the bound c >= 0 is inactive and the QP returns it too."""
    n = 7 if dim == 2 else 5
    if dim == 2:
        coef = I.rotated_tensor(0.4, 50.0, 1.0)
        mask = I.boundary_mask_2d(n, n)
    else:
        Q = I.quaternion_rotation(I.SplitMix64(3, 1))
        Dm = Q @ np.diag([40.0, 2.0, 1.0]) @ Q.T
        coef = np.array([Dm[0, 0], Dm[0, 1], Dm[0, 2], Dm[1, 1], Dm[1, 2], Dm[2, 2]])
        mask = I.boundary_mask_3d(n, n, n)
    coords, conn = O.mesh_structured(dim, n)
    asm = O.assemble(coords, conn, I.KIND_TENSOR, np.tile(coef, (len(conn), 1)))
    a = np.array([0.3, -0.2, 0.45][:dim])
    lin = 1.0 + coords @ a
    red = O.Reduced(asm, mask, lin)
    b = red.rhs()
    xg = O.galerkin(red.A, b)
    assert np.allclose(xg, lin[red.free], rtol=0, atol=1e-13)
    x, info = O.solve_qp(red.A, b, 0.0, math.inf)
    assert info["polished"]
    assert np.allclose(x, lin[red.free], rtol=0, atol=1e-13)


# ------------------------------------------------------------------ P5: DMP holds -> QP = Galerkin

def test_qp_equals_galerkin_when_dmp_holds():
    """D = I on the '/' grid gives an M-matrix; with f >= 0 and c^p >= 0 the
    Galerkin solution is already non-negative (Sec. 2.1.1 maximum principle),
    so the QP minimiser must coincide with it."""
    n = 24
    E = 2 * n * n
    coords, conn = O.mesh_structured(2, n)
    asm = O.assemble(coords, conn, I.KIND_TENSOR, np.tile([1.0, 0.0, 1.0], (E, 1)),
                     f_elem=I.square_box_source(n, n, 0.2, 0.5, 0.3, 0.9))
    mask = I.boundary_mask_2d(n, n)
    red = O.Reduced(asm, mask, np.zeros(len(mask)))
    b = red.rhs()
    xg = O.galerkin(red.A, b)
    assert xg.min() >= 0.0
    x, info = O.solve_qp(red.A, b, 0.0, math.inf)
    assert np.allclose(x, xg, rtol=0, atol=1e-12 * xg.max())
    # 3D Kuhn, D = I, patch boundary data in [0, 1], f = 0: 0 <= c <= 1 holds
    n = 8
    coords, conn = O.mesh_structured(3, n)
    asm = O.assemble(coords, conn, I.KIND_TENSOR, np.tile([1.0, 0, 0, 1, 0, 1], (len(conn), 1)))
    mask, val = I.patch_dirichlet_3d(n, n, n)
    red = O.Reduced(asm, mask, val)
    b = red.rhs()
    xg = O.galerkin(red.A, b)
    assert xg.min() >= -1e-15 and xg.max() <= 1.0 + 1e-15
    x, _ = O.solve_qp(red.A, b, 0.0, 1.0)
    assert np.allclose(x, np.clip(xg, 0, 1), rtol=0, atol=1e-12)


# ------------------------------------------------------------------ P6: brute force

def _reduced(spec):
    _, _, asm = build(spec)
    red = O.Reduced(asm, spec.dmask, spec.dval)
    return red, red.rhs()


@pytest.mark.parametrize("case", ["2d_n4_lower", "2d_n4_box", "3d_n3_lower", "2d_4x5_lower"])
def test_bruteforce_unique_kkt_point_matches_oracle(case):
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
    red, b = _reduced(spec)
    assert red.nF <= 12
    sols = O.brute_force(red.A, b, spec.lo, spec.hi)
    assert len(sols) == 1, "a strictly convex QP has exactly one KKT point"
    xb, assign = sols[0]
    x, info = O.solve_qp(red.A, b, spec.lo, spec.hi)
    assert np.allclose(x, xb, rtol=0, atol=1e-13 * max(1.0, np.abs(xb).max()))
    active = np.where(x == spec.lo, 1, np.where(x == spec.hi, 2, 0))
    assert np.array_equal(active, assign)
    assert (assign != 0).any(), "the case must have active bounds"
    # strict complementarity: free entries off the bounds, active multipliers nonzero
    g = red.A @ xb - b
    bound_gap = np.minimum(np.abs(xb - spec.lo), np.abs(xb - spec.hi))
    assert bound_gap[assign == 0].min() > 1e-6 * np.abs(xb).max()
    assert np.abs(g[assign != 0]).min() > 1e-6 * np.abs(b).max()
    if case == "2d_n4_box":
        assert (assign == 2).any() and (assign == 1).any()


# ------------------------------------------------------------------ P7: two independent solvers agree

@pytest.mark.parametrize("which", ["config1_n20", "batch_instance"])
def test_pgs_and_mprgp_agree(which):
    if which == "config1_n20":
        spec = I.config1_steady_2d(n=20)
    else:
        spec = I.config4_instance(3, nmin=16, nmax=24)
    red, b = _reduced(spec)
    x1, _ = O.solve_qp(red.A, b, spec.lo, spec.hi)
    x2, sweeps = O.pgs(red.A, b, spec.lo, spec.hi, tol=1e-16, maxsweep=400000)
    k2 = O.kkt(red.A, b, spec.lo, spec.hi, x2)
    assert k2["kkt_rel"] < 1e-9
    scale = np.abs(x1).max()
    assert np.abs(x1 - x2).max() <= 1e-8 * scale
    k1 = O.kkt(red.A, b, spec.lo, spec.hi, x1)
    assert k1["kkt_rel"] < 1e-12 and k1["bounds_ok"]


def test_pgs_and_mprgp_agree_on_the_mirrored_cube_with_a_hole():
    """Explicit mesh with a hole and active bounds: the two independent
    solvers reach the same minimiser, with lower bounds active."""
    sp, asm, red = _cube_hole(1, "mirrored")
    b = red.rhs()
    x1, _ = O.solve_qp(red.A, b, 0.0, 1.0)
    x2, _ = O.pgs(red.A, b, 0.0, 1.0, tol=1e-16, maxsweep=400000)
    assert O.kkt(red.A, b, 0.0, 1.0, x2)["kkt_rel"] < 1e-9
    assert np.abs(x1 - x2).max() <= 1e-8 * np.abs(x1).max()
    assert (x1 == 0.0).sum() > 0


# ------------------------------------------------------------------ closed-form QPs

def test_diagonal_qp_closed_form():
    """A diagonal: the minimiser is clamp(b/d, lo, hi) componentwise."""
    import scipy.sparse as sp
    rng = np.random.default_rng(5)
    d = rng.uniform(0.5, 3.0, 40)
    b = rng.normal(size=40)
    A = sp.diags(d).tocsr()
    for lo, hi in [(0.0, math.inf), (-0.2, 0.3), (-math.inf, 0.1)]:
        x, _ = O.solve_qp(A, b, lo, hi)
        assert np.array_equal(x, np.clip(b / d, lo, hi)) or np.allclose(x, np.clip(b / d, lo, hi), atol=1e-15)
        assert O.kkt(A, b, lo, hi, x)["kkt_rel"] < 1e-15


def test_two_variable_qp_by_hand():
    """A = [[2,-1],[-1,2]], b = (1,-2), x >= 0.  Unconstrained (0,-1) is
    infeasible; with x2 = 0 active: 2 x1 = 1 -> x1 = 1/2, and
    g2 = -x1 - b2 = -1/2 + 2 = 3/2 >= 0, so (1/2, 0) is the KKT point."""
    import scipy.sparse as sp
    A = sp.csr_matrix(np.array([[2.0, -1.0], [-1.0, 2.0]]))
    b = np.array([1.0, -2.0])
    x, _ = O.solve_qp(A, b, 0.0, math.inf)
    assert np.allclose(x, [0.5, 0.0], atol=1e-15) and x[1] == 0.0
    k = O.kkt(A, b, 0.0, math.inf, x)
    assert k["kkt_rel"] < 1e-15 and k["obj"] == pytest.approx(-0.25)


def test_kkt_measure_by_hand():
    import scipy.sparse as sp
    A = sp.identity(3, format="csr")
    b = np.array([1.0, -1.0, 2.0])
    x = np.array([0.0, 0.0, 3.0])        # g = x - b = (-1, 1, 1), box [0, 3]
    k = O.kkt(A, b, 0.0, 3.0, x)
    # x1 at lo with g < 0 -> -1 ; x2 at lo with g > 0 -> 0 ; x3 at hi with g > 0 -> 1
    assert k["gp2"] == pytest.approx(math.sqrt(2.0))
    assert k["kkt_rel"] == pytest.approx(math.sqrt(2.0) / math.sqrt(6.0))
    assert k["kkt_inf"] == pytest.approx(1.0 / 2.0)
    assert k["bounds_ok"]
    assert not O.kkt(A, b, 0.0, 3.0, np.array([0.0, -1e-300, 1.0]))["bounds_ok"]


# ------------------------------------------------------------------ transient pins

def _transient_setup(n=6, dt=0.01, hi=1.0):
    spec = I.config2_transient_3d(n=n, dt=dt, nsteps=3)
    _, _, asm = build(spec, with_mass=True)
    return spec, asm


def test_transient_constant_states_are_fixed_points():
    """K 1 = 0 (zero row sums), so with c^p = 1, c^(0) = 1 and f = 0 the
    backward-Euler QP returns c = 1 at every step, with the upper bound
    active; c = 0 everywhere is a fixed point likewise."""
    spec, asm = _transient_setup()
    for val in (1.0, 0.0):
        dval = np.full(spec.n_nodes, val)
        red = O.Reduced(asm, spec.dmask, dval, dt=spec.dt)
        states = O.transient(red, np.full(spec.n_nodes, val), 0.0, 1.0, 3)
        for c in states:
            assert np.abs(c - val).max() <= 1e-13


def test_transient_single_mode_decay():
    """Without bounds, f = 0 and c^p = 0, a generalized eigenvector
    K_FF v = lam M_FF v decays by exactly 1/(1 + lam dt) per backward-Euler
    step: pins the right-hand side M c^(n)/dt (not c^(n+1))."""
    spec, asm = _transient_setup(n=5, dt=0.05)
    mask = I.boundary_mask_3d(5, 5, 5)
    red = O.Reduced(asm, mask, np.zeros(spec.n_nodes), dt=spec.dt)
    Kf = asm.K[red.free][:, red.free].toarray()
    Mf = asm.M[red.free][:, red.free].toarray()
    lam, V = sla.eigh(Kf, Mf)
    for k in (0, 7):
        c0 = red.full(V[:, k] / np.abs(V[:, k]).max())
        states = O.transient(red, c0, -math.inf, math.inf, 2)
        fac = 1.0 / (1.0 + lam[k] * spec.dt)
        assert np.allclose(states[0], c0 * fac, atol=1e-12)
        assert np.allclose(states[1], c0 * fac ** 2, atol=1e-12)


def test_transient_steps_stay_in_bounds_and_match_dmp():
    """The transient QP keeps 0 <= c <= 1 exactly while the unconstrained
    backward-Euler step leaves the box for this anisotropic field."""
    spec = I.config2_transient_3d(n=8, nsteps=2)
    _, _, asm = build(spec, with_mass=True)
    red = O.Reduced(asm, spec.dmask, spec.dval, dt=spec.dt)
    b = red.rhs(spec.c0)
    xg = O.galerkin(red.A, b)
    assert xg.min() < 0.0
    states = O.transient(red, spec.c0, 0.0, 1.0, 2)
    for c in states:
        assert c.min() == 0.0 and c.max() <= 1.0


# ------------------------------------------------------------------ lumped capacity matrix

def _simplex_measures(coords, conn):
    """|e| of every simplex from its vertex coordinates: |det J| / d!."""
    d = coords.shape[1]
    J = coords[conn[:, 1:]] - coords[conn[:, :1]]
    return np.abs(np.linalg.det(J)) / math.factorial(d)


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 3)])
def test_lumped_mass_is_the_nodal_share_of_element_measures(dim, n):
    """Row-sum lumping of the consistent P1 mass gives the diagonal matrix
    M_ii = sum over elements e containing node i of |e| / (d+1), computed here
    by brute force from the vertex coordinates; off-diagonal entries are 0,
    the entries sum to the domain volume 1, and K does not change."""
    coords, conn = O.mesh_structured(dim, n)
    coef = np.tile([1.0, 0.2, 2.0] if dim == 2 else [1.0, 0.1, 0, 2.0, 0.3, 1.5], (len(conn), 1))
    cons = O.assemble(coords, conn, I.KIND_TENSOR, coef, with_mass=True)
    lump = O.assemble(coords, conn, I.KIND_TENSOR, coef, with_mass=True, lumped=True)
    assert np.array_equal(cons.Kval, lump.Kval)
    vol = _simplex_measures(coords, conn)
    want = np.zeros(len(coords))
    for e, verts in enumerate(conn):
        for v in verts:
            want[v] += vol[e] / (dim + 1)
    ML = lump.M.toarray()
    assert np.allclose(np.diag(ML), want, rtol=1e-14, atol=0)
    assert np.count_nonzero(ML - np.diag(np.diag(ML))) == 0
    assert ML.sum() == pytest.approx(1.0, rel=1e-14)
    # consistent mass: positive off-diagonal entries, same row sums
    Mc = cons.M.toarray()
    assert (Mc[~np.eye(len(Mc), dtype=bool) & (Mc != 0)] > 0).all()
    assert np.allclose(Mc.sum(axis=1), want, rtol=1e-14, atol=0)


def test_lumped_backward_euler_keeps_the_maximum_principle():
    """D = I on Kuhn tetrahedra: K has non-positive off-diagonal entries, so
    K + M_L/dt is an M-matrix and a backward-Euler step from data in [0, 1]
    stays in [0, 1] without constraints: the QP step equals the Galerkin step.
    With the consistent M the same step undershoots (its positive
    off-diagonal entries M_ij/dt break the M-matrix property), which is what
    makes the bounds necessary there."""
    n = 6
    coords, conn = O.mesh_structured(3, n)
    coef = np.tile([1.0, 0, 0, 1, 0, 1], (len(conn), 1))
    mask, val = I.patch_dirichlet_3d(n, n, n)
    c0 = np.where(mask == 1, val, 0.0)
    for dt in (1e-2, 1e-3):
        lump = O.assemble(coords, conn, I.KIND_TENSOR, coef, with_mass=True, lumped=True)
        red = O.Reduced(lump, mask, val, dt=dt)
        A = red.A.tocoo()
        assert A.data[A.row != A.col].max() <= 0.0
        xg = O.galerkin(red.A, red.rhs(c0))
        assert xg.min() >= 0.0 and xg.max() <= 1.0
        states = O.transient(red, c0, 0.0, 1.0, 2)
        assert np.allclose(states[0][red.free], xg, rtol=0, atol=1e-12)
        cons = O.assemble(coords, conn, I.KIND_TENSOR, coef, with_mass=True)
        redc = O.Reduced(cons, mask, val, dt=dt)
        assert O.galerkin(redc.A, redc.rhs(c0)).min() < -1e-3


# ------------------------------------------------------------------ cube with a hole (Sec. 5.1 analogue)

def _cube_hole(m, mesh):
    sp = I.cube_with_hole(m, mesh)
    asm = O.assemble(sp.coords, sp.conn, sp.coef_kind, sp.coef, sp.aL, sp.aT, sp.DM, with_mass=True)
    return sp, asm, O.Reduced(asm, sp.dmask, sp.dval)


def test_cube_hole_mesh_and_volume():
    """The explicit mesh generator with an empty hole reproduces the oracle's
    structured Kuhn mesh; with the hole, the element measures sum to the
    domain volume 1 - (1/9)^3, the capacity matrix too, and every row of K
    sums to zero (constants are in the kernel of the Neumann operator)."""
    c, e, _ = I.kuhn_mesh_without_box(5, 0, 0)
    oc, oe = O.mesh_structured(3, 5)
    assert np.array_equal(c, oc) and np.array_equal(e, oe)
    for mesh in ("kuhn", "mirrored"):
        sp, asm, _ = _cube_hole(2, mesh)
        assert sp.n_nodes == 19 ** 3 - 1                 # one lattice node strictly inside the hole
        assert sp.n_elems == 6 * (18 ** 3 - 2 ** 3)
        assert _simplex_measures(sp.coords, sp.conn).sum() == pytest.approx(1 - 1 / 729, rel=1e-13)
        assert asm.M.sum() == pytest.approx(1 - 1 / 729, rel=1e-13)
        rs = np.abs(asm.K.sum(axis=1)).max()
        assert rs <= 1e-13 * np.abs(asm.K).sum(axis=1).max()


def test_cube_hole_aligned_mesh_keeps_dmp_mirrored_mesh_violates_it():
    """v = (1,1,1) along the Kuhn diagonals: K_FF has no positive
    off-diagonal entry (an M-matrix), the Galerkin solution stays in [0, 1]
    and the QP returns it.  On the mirrored mesh the same physical problem
    gives a Galerkin solution with negative values at a sizable share of the
    nodes (the paper's Table of DMP violations reports 26-54% on its
    unstructured meshes), while the QP keeps 0 <= c <= 1 exactly."""
    sp, asm, red = _cube_hole(2, "kuhn")
    A = red.A.tocoo()
    assert A.data[A.row != A.col].max() <= 1e-15 * np.abs(A.data).max()
    b = red.rhs()
    xg = O.galerkin(red.A, b)
    assert xg.min() >= -1e-14 and xg.max() <= 1.0
    x, _ = O.solve_qp(red.A, b, 0.0, 1.0)
    assert np.allclose(x, np.clip(xg, 0.0, 1.0), rtol=0, atol=1e-12)
    sp, asm, red = _cube_hole(2, "mirrored")
    A = red.A.tocoo()
    assert A.data[A.row != A.col].max() > 0.0
    b = red.rhs()
    xg = O.galerkin(red.A, b)
    full = red.full(xg)
    share = ((full < 0) | (full > 1)).mean()
    assert xg.min() < -0.01 and 0.2 < share < 0.4
    x, _ = O.solve_qp(red.A, b, 0.0, 1.0)
    assert x.min() == 0.0 and x.max() <= 1.0
    assert O.kkt(red.A, b, 0.0, 1.0, x)["kkt_rel"] < 1e-12


# ------------------------------------------------------------------ P9 / P10 / P11

def test_objective_order_galerkin_violation_and_exact_bounds():
    spec = I.config1_steady_2d(n=30)
    red, b = _reduced(spec)
    x, info = O.solve_qp(red.A, b, spec.lo, spec.hi)
    xg = O.galerkin(red.A, b)
    assert xg.min() < 0.0                                  # Galerkin violates c >= 0
    assert x.min() == 0.0 and (x >= 0.0).all()             # QP: exact bound
    q = lambda y: O.objective(red.A, b, y)
    assert q(x) <= q(np.clip(xg, 0, None))
    rng = np.random.default_rng(0)
    for _ in range(5):
        y = np.abs(x + 1e-4 * x.max() * rng.normal(size=len(x)))
        assert q(x) <= q(y)
    assert O.kkt(red.A, b, spec.lo, spec.hi, x)["kkt_rel"] < 1e-12


# ------------------------------------------------------------------ invalid input

def test_assembly_rejects_bad_input():
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    conn = np.array([[0, 1, 2]], np.int32)
    with pytest.raises(ValueError, match="degenerate"):
        O.assemble(coords, conn, I.KIND_TENSOR, np.array([[1.0, 0.0, 1.0]]))
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    with pytest.raises(ValueError, match="SPD"):
        O.assemble(coords, conn, I.KIND_TENSOR, np.array([[1.0, 2.0, 1.0]]))
    with pytest.raises(ValueError, match="NaN"):
        O.assemble(coords, conn, I.KIND_TENSOR, np.array([[1.0, math.nan, 1.0]]))
