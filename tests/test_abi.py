"""The C-ABI library loads and exports every entry point include/nnqp.h
declares; host-only entry points behave as documented.  No GPU needed."""
import ctypes
import os
import re

import pytest

import paper_1506_08435_gb300 as P

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nnqp.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nn_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    L = P.lib()
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(P.binding.EXPORTS)


def test_library_is_built_for_sm103a_and_in_tree():
    path = P.library_path()
    assert os.path.dirname(path).endswith("paper_1506_08435_gb300")
    from paper_1506_08435_gb300 import build as b
    assert "arch=compute_103a,code=sm_103a" in b.ARCH


def test_host_only_entry_points():
    assert "sm_103a" in P.nn_version()
    assert P.nn_mesh_counts(2, 50, 50) == (2601, 5000)
    assert P.nn_mesh_counts(3, 40, 40, 40) == (68921, 384000)
    assert P.nn_mesh_counts(3, 150, 150, 150) == (151 ** 3, 20250000)
    with pytest.raises(P.NnError) as e:
        P.nn_mesh_counts(4, 1, 1, 1)
    assert e.value.status == P.NN_ERR_INVALID_ARG
    o = P.solve_opts()
    assert o.rtol == 1e-10 and o.solver == P.NN_SOLVER_GPCG and o.lbfgs_m == 5
    so = P.serve_opts()
    assert so.max_inflight >= 1


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof of every public struct, as the C compiler lays it out from the
    header, equals the ctypes mirror used by the binding."""
    structs = ["nn_problem", "nn_assemble_opts", "nn_system_desc", "nn_solve_opts", "nn_solve_info",
               "nn_serve_opts", "nn_serve_stats_t"]
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "nnqp.h"\nint main(void){\n' +
                   "".join('printf("%%zu\\n", sizeof(%s));\n' % s for s in structs) + "return 0;}\n")
    exe = tmp_path / "sz"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    sizes = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    for s, n in zip(structs, sizes):
        assert ctypes.sizeof(getattr(P.binding, s)) == n, s


def test_assembly_host_validation_without_a_device():
    """Arguments that nn_assemble rejects on the host, before any device call:
    each returns its documented status and a message."""
    import math
    import nn_inputs as I
    spec = I.config1_steady_2d(n=4)

    def status_of(mutate=None, opts=None):
        pr = P.Problem(spec)
        if mutate:
            mutate(pr.c)
        with pytest.raises(P.NnError) as e:
            P.nn_assemble(pr, opts)
        assert "nn_assemble" in str(e.value)
        return e.value.status

    def setf(**kw):
        return lambda c: [setattr(c, k, v) for k, v in kw.items()]

    assert status_of(setf(dim=4)) == P.NN_ERR_INVALID_ARG
    assert status_of(setf(memory=7)) == P.NN_ERR_INVALID_ARG
    assert status_of(setf(lo=1.0, hi=0.0)) == P.NN_ERR_INFEASIBLE
    assert status_of(setf(lo=math.nan)) == P.NN_ERR_INFEASIBLE
    assert status_of(setf(dt=-1.0)) == P.NN_ERR_INVALID_ARG
    assert status_of(setf(dt=math.inf)) == P.NN_ERR_INVALID_ARG
    assert status_of(setf(coef_kind=9)) == P.NN_ERR_INVALID_ARG
    assert status_of(setf(coef=None)) == P.NN_ERR_INVALID_ARG
    assert status_of(setf(nx=0)) == P.NN_ERR_INVALID_ARG
    assert status_of(opts=P.assemble_opts(lumped_mass=2)) == P.NN_ERR_INVALID_ARG
    ex = I.cube_with_hole(1)
    pr = P.Problem(ex)
    pr.c.n_elems = 0
    with pytest.raises(P.NnError) as e:
        P.nn_assemble(pr)
    assert e.value.status == P.NN_ERR_INVALID_ARG
