"""Host side of the SSOR preconditioner: the library's DSatur colouring
(nn_color_dsatur, the ordering nn_precond_setup builds) against the
oracle's, bit for bit, and the option checks that need no device."""
import numpy as np
import pytest
import scipy.sparse as sp

import nn_inputs as I
import paper_1506_08435_gb300 as P
from oracle import oracle as O
from tests.gpu_common import oracle_reduced


@pytest.mark.parametrize("spec", [I.config1_steady_2d(n=20), I.config3_steady_3d(n=12),
                                  I.config2_transient_3d(n=8), I.config4_instance(7)],
                         ids=lambda s: s.name)
def test_library_colouring_equals_the_oracle(spec):
    _, red = oracle_reduced(spec)
    A = red.A.tocsr()
    c, k = P.nn_color_dsatur(A.indptr, A.indices)
    ref = O.dsatur(A)
    assert np.array_equal(c, ref)
    assert k == ref.max() + 1
    assert k == (3 if spec.dim == 2 else 4)


def test_library_colouring_of_small_graphs():
    # the hand-traced run of the oracle pins
    r = [0, 1, 0, 2, 1, 2, 2, 3, 3, 4]
    c = [1, 0, 2, 0, 2, 1, 3, 2, 4, 3]
    A = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(5, 5))
    col, k = P.nn_color_dsatur(A.indptr, A.indices)
    assert col.tolist() == [1, 2, 0, 1, 0] and k == 3
    # no edges: one colour; empty graph: none
    E = sp.identity(4, format="csr")
    col, k = P.nn_color_dsatur(E.indptr, E.indices)
    assert col.tolist() == [0, 0, 0, 0] and k == 1
    col, k = P.nn_color_dsatur(np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert k == 0 and len(col) == 0


def test_library_colouring_rejects_bad_patterns():
    A = sp.identity(3, format="csr")
    bad = A.indices.copy()
    bad[1] = 3
    with pytest.raises(P.NnError):
        P.nn_color_dsatur(A.indptr, bad)
    with pytest.raises(P.NnError):
        P.nn_color_dsatur(np.array([1, 1], np.int64), np.zeros(1, np.int32))
    # a clique of 65 vertices needs 65 colours: more than the library keeps
    n = 65
    K = sp.csr_matrix(np.ones((n, n)))
    with pytest.raises(P.NnError):
        P.nn_color_dsatur(K.indptr, K.indices)


def test_solve_option_defaults():
    o = P.solve_opts()
    assert o.precond == P.NN_PC_JACOBI and o.ssor_omega == 1.0
