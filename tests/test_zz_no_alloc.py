"""The no-allocation product nn_spmv_mixed_noalloc.

Some callers cannot allocate device memory once they are running (a
real-time loop where cudaMalloc/cudaFree may stall the whole device, or an
application whose device memory belongs entirely to another allocator).
nn_spmv_mixed_noalloc serves them: it computes the FP32-value product of
nn_spmv(NN_PREC_MIXED) with the library's fixed scratch array instead of a
per-call temporary.  These tests call it through the C ABI and compare it
with the allocating entry point on two calls in a row, check that repeated
calls take no device memory, and that a system above the array's limit is
refused.  This file is collected last.
"""
import numpy as np
import pytest

import nn_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1506_08435_gb300 as P  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.lib()
    return torch.device("cuda:0")


@pytest.mark.parametrize("spec_fn", [lambda: I.config3_steady_3d(n=14, seed=5), lambda: I.config1_steady_2d()])
def test_noalloc_product_matches_allocating_product_twice(dev, spec_fn):
    spec = spec_fn()
    s = P.nn_assemble(P.Problem(spec, device=dev), P.assemble_opts(build_mixed=1))
    nf = s.describe()["n_free"]
    A_rows = None
    for call in range(2):
        rng = np.random.default_rng(100 + call)
        x = torch.tensor(rng.uniform(-1.0, 1.0, nf), device=dev)
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        P.nn_spmv(s, x, y_ref, P.NN_FMT_SELL, P.NN_PREC_MIXED)
        P.nn_spmv_mixed_noalloc(s, x, y)
        torch.cuda.synchronize()
        yr, yn = y_ref.cpu().numpy(), y.cpu().numpy()
        # the tolerance of the FP32-operator tests: a few units of 2^-24 of |A||x|
        xa = np.abs(x.cpu().numpy())
        if A_rows is None:
            rp = np.zeros(nf + 1, np.int64)
            col = np.zeros(s.describe()["nnz_free"], np.int32)
            val = np.zeros(len(col))
            P.nn_system_copy_out(s, "A_rowptr", rp)
            P.nn_system_copy_out(s, "A_col", col)
            P.nn_system_copy_out(s, "A_val", val)
            A_rows = (rp, col, np.abs(val))
        rp, col, aval = A_rows
        scale = np.add.reduceat(aval * xa[col], rp[:-1])
        assert np.all(np.isfinite(yn))
        assert np.all(np.abs(yn - yr) <= 2e-6 * scale)


def test_noalloc_product_allocates_nothing_on_repeated_calls(dev):
    """After the first call (which may load the library's module and look up
    the array's address), further calls take no buffer from the library's
    memory pool and leave the device's free memory unchanged; each still
    gives the allocating product's result."""
    spec = I.config3_steady_3d(n=20, seed=7)
    s = P.nn_assemble(P.Problem(spec, device=dev), P.assemble_opts(build_mixed=1))
    nf = s.describe()["n_free"]
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.uniform(-1.0, 1.0, nf), device=dev)
    y = torch.empty_like(x)
    y_ref = torch.empty_like(x)
    P.nn_spmv(s, x, y_ref, P.NN_FMT_SELL, P.NN_PREC_MIXED)
    P.nn_spmv_mixed_noalloc(s, x, y)            # first call: set-up
    torch.cuda.synchronize()
    a0 = P.nn_device_allocations()
    free0 = torch.cuda.mem_get_info()[0]
    l0 = P.nn_kernel_launches()
    for _ in range(50):
        P.nn_spmv_mixed_noalloc(s, x, y)
    torch.cuda.synchronize()
    assert P.nn_device_allocations() == a0
    assert torch.cuda.mem_get_info()[0] == free0
    assert P.nn_kernel_launches() - l0 == 100   # two kernels per call, nothing else
    assert torch.equal(y, y_ref)                 # same kernels, same FP32 arithmetic
    # the allocating entry point does take a buffer per call (the counter sees it)
    P.nn_spmv(s, x, y_ref, P.NN_FMT_SELL, P.NN_PREC_MIXED)
    torch.cuda.synchronize()
    assert P.nn_device_allocations() == a0 + 1


def test_noalloc_product_rejects_systems_above_the_limit(dev):
    n = 2050                      # 2049^2 = 4,198,401 free unknowns > 4,194,304
    spec = I.config1_steady_2d(n=n)
    s = P.nn_assemble(P.Problem(spec, device=dev), P.assemble_opts(build_mixed=1))
    nf = s.describe()["n_free"]
    assert nf > (1 << 22)
    x = torch.zeros(nf, dtype=torch.float64, device=dev)
    y = torch.zeros_like(x)
    with pytest.raises(P.NnError) as e:
        P.nn_spmv_mixed_noalloc(s, x, y)
    assert e.value.status == P.NN_ERR_INVALID_ARG
    assert "limit" in str(e.value)
