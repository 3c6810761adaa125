"""Pins of the oracle's SSOR preconditioner and of its colouring.

The oracle's ``ssor_apply`` takes two sparse triangular solves on the
colour-ordered matrix; here it is checked against routes that share none of
that code: a hand-traced example, the diagonal special case, one forward and
one backward SOR sweep from zero written as plain loops (Saad, Iterative
Methods for Sparse Linear Systems, Sec. 4.1.2: one SSOR step from x = 0 is
x = M^-1 r), the explicit product M = (D + wL) D^-1 (D + wU) / (w (2 - w)),
symmetry and positivity.  ``dsatur`` is checked on graphs whose chromatic
numbers are known and on a hand-traced run of the rule.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import nn_inputs as I
from oracle import oracle as O
from tests.gpu_common import oracle_reduced


def proper(A, c):
    A = sp.coo_matrix(A)
    off = A.row != A.col
    return not np.any(c[A.row[off]] == c[A.col[off]])


def graph(n, edges):
    r = [i for i, j in edges] + [j for i, j in edges] + list(range(n))
    c = [j for i, j in edges] + [i for i, j in edges] + list(range(n))
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))


# ------------------------------------------------------------------ DSatur

def test_dsatur_hand_traced_run():
    """Edges 0-1, 0-2, 1-2, 2-3, 3-4 (degrees 2, 2, 3, 2, 1).  Step 1: all
    saturations 0, vertex 2 has the largest degree -> colour 0.  Step 2:
    vertices 0, 1, 3 have saturation 1 and degree 2, the smallest index 0
    takes colour 1.  Step 3: vertex 1 (saturation 2) -> colour 2.  Step 4:
    vertex 3 (saturation 1) -> colour 1.  Step 5: vertex 4 -> colour 0.
    Plain greedy in index order would give (0, 1, 2, 0, 1)."""
    A = graph(5, [(0, 1), (0, 2), (1, 2), (2, 3), (3, 4)])
    assert O.dsatur(A).tolist() == [1, 2, 0, 1, 0]


@pytest.mark.parametrize("n,edges,chi", [
    (6, [(i, i + 1) for i in range(5)], 2),                    # path
    (8, [(i, (i + 1) % 8) for i in range(8)], 2),              # even cycle
    (7, [(i, (i + 1) % 7) for i in range(7)], 3),              # odd cycle
    (5, [(i, j) for i in range(5) for j in range(i + 1, 5)], 5),  # complete graph K5
    (6, [(0, 3), (0, 4), (0, 5), (1, 3), (1, 4), (1, 5), (2, 3), (2, 4), (2, 5)], 2),  # K(3,3)
])
def test_dsatur_finds_the_chromatic_number_of_small_graphs(n, edges, chi):
    A = graph(n, edges)
    c = O.dsatur(A)
    assert proper(A, c)
    assert c.max() + 1 == chi


@pytest.mark.parametrize("dim,k,chi", [(2, 7, 3), (3, 5, 4)])
def test_dsatur_on_the_structured_meshes_is_proper_and_optimal(dim, k, chi):
    """The "/" triangles contain 3-cliques and the Kuhn tetrahedra 4-cliques,
    so 3 (2D) and 4 (3D) colours are the least possible."""
    coords, conn = O.mesh_structured(dim, *([k] * dim))
    rp, col = O.pattern(len(coords), conn)
    A = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(len(coords), len(coords)))
    c = O.dsatur(A)
    assert proper(A, c)
    assert c.max() + 1 == chi


def test_dsatur_on_free_patterns_is_proper():
    for spec in (I.config1_steady_2d(n=12), I.config3_steady_3d(n=8)):
        _, red = oracle_reduced(spec)
        assert proper(red.A, O.dsatur(red.A))


# ------------------------------------------------------------------ SSOR

def sor_sweeps(A, order, r, w):
    """One forward SOR sweep along `order`, then one backward sweep, from
    x = 0: x_i <- (1 - w) x_i + w (r_i - sum_{j != i} a_ij x_j) / a_ii."""
    Ad = A.toarray()
    x = np.zeros(len(r))
    for seq in (order, order[::-1]):
        for i in seq:
            s = Ad[i] @ x - Ad[i, i] * x[i]
            x[i] = (1.0 - w) * x[i] + w * (r[i] - s) / Ad[i, i]
    return x


def small_system():
    spec = I.config3_steady_3d(n=5)
    _, red = oracle_reduced(spec)
    return red.A.tocsr()


def test_ssor_hand_traced_example():
    """A = tridiag(-1, 2, -1), n = 3, colours (0, 1, 0), w = 1, r = (1, 1, 1).
    Forward, colour 0: y0 = y2 = 1/2; colour 1: y1 = (1 + y0 + y2)/2 = 1.
    Backward, colour 1: z1 = y1 = 1 (no later colour); colour 0:
    z0 = z2 = y0 + z1/2 = 1."""
    A = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(3, 3)).tocsr()
    z = O.ssor_apply(A, np.array([0, 1, 0]), np.ones(3), 1.0)
    assert np.allclose(z, [1.0, 1.0, 1.0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("w", [0.7, 1.0, 1.5])
def test_ssor_of_a_diagonal_matrix(w):
    d = np.array([2.0, 3.0, 0.5, 7.0])
    r = np.array([1.0, -2.0, 3.0, 0.25])
    z = O.ssor_apply(sp.diags(d).tocsr(), np.zeros(4, np.int32), r, w)
    assert np.allclose(z, w * (2.0 - w) * r / d, rtol=1e-15, atol=0)


@pytest.mark.parametrize("w", [0.6, 1.0, 1.4])
def test_ssor_equals_one_symmetric_sor_step_from_zero(w):
    A = small_system()
    c = O.dsatur(A)
    n = A.shape[0]
    r = np.random.default_rng(4).normal(size=n)
    order = np.lexsort((np.arange(n), c))
    z = O.ssor_apply(A, c, r, w)
    ref = sor_sweeps(A, order, r, w)
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("w", [0.8, 1.3])
def test_ssor_inverts_the_explicit_product(w):
    A = small_system()
    c = O.dsatur(A)
    n = A.shape[0]
    r = np.random.default_rng(5).normal(size=n)
    z = O.ssor_apply(A, c, r, w)
    order = np.lexsort((np.arange(n), c))
    P = sp.csr_matrix((np.ones(n), (np.arange(n), order)), shape=(n, n))   # (P v) = v[order]
    Ap = (P @ A @ P.T).toarray()
    D = np.diag(np.diag(Ap))
    M = (D + w * np.tril(Ap, -1)) @ np.linalg.inv(D) @ (D + w * np.triu(Ap, 1)) / (w * (2.0 - w))
    res = M @ (P @ z) - P @ r
    assert np.abs(res).max() <= 1e-12 * np.abs(r).max()


def test_ssor_is_symmetric_positive_definite():
    A = small_system()
    c = O.dsatur(A)
    rng = np.random.default_rng(6)
    r1, r2 = rng.normal(size=(2, A.shape[0]))
    for w in (0.5, 1.0, 1.7):
        z1, z2 = O.ssor_apply(A, c, r1, w), O.ssor_apply(A, c, r2, w)
        assert abs(r2 @ z1 - r1 @ z2) <= 1e-12 * abs(r1 @ z1)
        assert r1 @ z1 > 0 and r2 @ z2 > 0


def test_ssor_on_a_face_is_the_ssor_of_the_face_block():
    A = small_system()
    c = O.dsatur(A)
    n = A.shape[0]
    rng = np.random.default_rng(7)
    face = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    r = rng.normal(size=n)
    z = O.ssor_apply(A, c, r, 1.2, face=face)
    F = np.flatnonzero(face)
    assert np.all(z[face == 0] == 0.0)
    AF = A[F][:, F].tocsr()
    order = np.lexsort((np.arange(len(F)), c[F]))
    ref = sor_sweeps(AF, order, r[F], 1.2)
    assert np.abs(z[F] - ref).max() <= 1e-12 * np.abs(ref).max()
