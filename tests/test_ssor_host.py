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


def _layout_checker(tmp_path):
    """Builds tests/ssor_layout_check.cpp against the library."""
    import os
    import subprocess
    P.lib()
    here = os.path.dirname(os.path.abspath(__file__))
    pkg = os.path.dirname(P.library_path())
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = str(tmp_path / "ssor_layout_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(pkg, "csrc"), "-I", os.path.join(cuda, "include"),
                           os.path.join(here, "ssor_layout_check.cpp"), "-o", exe, "-L", pkg, "-lnnqp",
                           "-Wl,-rpath," + pkg, "-L", os.path.join(cuda, "lib64"), "-lcudart"])
    return exe


@pytest.mark.parametrize("spec,omega,share", [(I.config3_steady_3d(n=16), 1.0, 1.0), (I.config1_steady_2d(n=40), 1.3, 0.7),
                                              (I.cube_with_hole(3), 0.8, 0.9)], ids=lambda v: getattr(v, "name", str(v)))
def test_library_ssor_layout_and_sweeps_match_the_oracle(tmp_path, spec, omega, share):
    """The host half of nn_precond_setup (A's pair-interleaved SELL-32 read
    back into rows, DSatur, the colour-ordered lower and upper parts) run on
    the CPU, followed by the two sweeps with the kernels' indexing: equal to
    the oracle's SSOR application (and no read of an unwritten entry, which
    the NaN-filled scratch would show)."""
    import subprocess
    exe = _layout_checker(tmp_path)
    _, red = oracle_reduced(spec)
    A = red.A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    rng = np.random.default_rng(9)
    r = rng.normal(size=n)
    face = (rng.uniform(size=n) < share).astype(np.uint8)
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(src, "wb") as f:
        np.array([n, A.nnz], np.int64).tofile(f)
        A.indptr.astype(np.int64).tofile(f)
        A.indices.astype(np.int32).tofile(f)
        A.data.astype(np.float64).tofile(f)
        r.tofile(f)
        face.tofile(f)
        np.array([omega]).tofile(f)
    subprocess.check_call([exe, str(src), str(dst)])
    raw = open(dst, "rb").read()
    z = np.frombuffer(raw[:8 * n], np.float64)
    col = np.frombuffer(raw[8 * n:], np.int32)
    ref_col = O.dsatur(A)
    assert np.array_equal(col, ref_col)
    ref = O.ssor_apply(A, ref_col, r, omega, face=face)
    assert np.isfinite(z).all()
    assert np.abs(z - ref).max() <= 1e-13 * np.abs(ref).max()
