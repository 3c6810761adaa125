"""Row sharding of one QP (nn_shard_plan / nn_shard_build / nn_shard_spmv).

The paper scales one problem by domain decomposition: each MPI rank owns
part of the unknowns, a product first scatters the ghost values its rows
need, a dot product is a local sum plus an all-reduce (Sec. 3.1; strong
scaling, Sec. 5.1.2).  The CPU tests check the plan against the global
matrix and run the exchange, the local products and the distributed dots
as two gloo ranks on the oracle's own assembly of a small 3D system: the
result equals the single-process product and dots.  The GPU test runs the
library's local product of each shard on the device."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.sparse as sps

import nn_inputs as I
import paper_1506_08435_gb300 as P
from tests.gpu_common import oracle_reduced

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def system(n=10):
    spec = I.config3_steady_3d(n=n, seed=5)
    _, red = oracle_reduced(spec)
    return spec, red.A.tocsr(), red.rhs()


@pytest.mark.parametrize("nranks", [1, 2, 3, 5])
def test_plan_covers_the_rows_once_and_renumbers_columns(nranks):
    spec, A, _ = system()
    n = A.shape[0]
    starts, ghosts_total = [], 0
    for r in range(nranks):
        sh = P.nn_shard_build(A.indptr, A.indices, nranks, r)
        r0, r1 = sh["row0"], sh["row1"]
        starts.append((r0, r1))
        nrows = r1 - r0
        # local rows: the same entries in the same order, columns renumbered
        cols = np.where(sh["local_col"] < nrows, sh["local_col"] + r0,
                        sh["halo_ids"][np.maximum(sh["local_col"] - nrows, 0)] if len(sh["halo_ids"]) else 0)
        assert np.array_equal(sh["local_rowptr"], A.indptr[r0:r1 + 1] - A.indptr[r0])
        assert np.array_equal(cols, A.indices[A.indptr[r0]:A.indptr[r1]])
        # ghosts: exactly the outside columns of the owned rows, each with its owner
        outside = np.unique(A.indices[A.indptr[r0]:A.indptr[r1]])
        outside = outside[(outside < r0) | (outside >= r1)]
        assert np.array_equal(sh["halo_ids"], outside)
        ghosts_total += len(outside)
        starts_all = [P.nn_shard_plan(A.indptr, A.indices, nranks, q) for q in range(nranks)]
        for h, o in zip(sh["halo_ids"], sh["halo_owner"]):
            assert starts_all[o]["row0"] <= h < starts_all[o]["row1"]
        # on the structured cube a rank's ghosts come from its neighbouring ranks only
        assert set(sh["halo_owner"].tolist()) <= {r - 1, r + 1}
    assert starts[0][0] == 0 and starts[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(starts, starts[1:]))
    # what every rank sends is what the others hold as ghosts
    sends = sum(P.nn_shard_plan(A.indptr, A.indices, nranks, r)["n_send"] for r in range(nranks))
    assert sends == ghosts_total
    # balanced by nonzeros
    nnz = [P.nn_shard_plan(A.indptr, A.indices, nranks, r)["nnz"] for r in range(nranks)]
    assert max(nnz) - min(nnz) <= 2 * np.diff(A.indptr).max()


def test_plan_rejects_bad_input():
    spec, A, _ = system(4)
    with pytest.raises(P.NnError):
        P.nn_shard_plan(A.indptr, A.indices, 2, 2)
    bad = A.indices.copy()
    bad[3] = A.shape[0]
    with pytest.raises(P.NnError):
        P.nn_shard_plan(A.indptr, bad, 2, 0)


WORKER = r'''
import json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, scipy.sparse as sps, torch, torch.distributed as dist
import nn_inputs as I
import paper_1506_08435_gb300 as P
from tests.gpu_common import oracle_reduced
dist.init_process_group("gloo")
rank, ws = dist.get_rank(), dist.get_world_size()
spec = I.config3_steady_3d(n=10, seed=5)
_, red = oracle_reduced(spec)
A = red.A.tocsr()
n = A.shape[0]
sh = P.nn_shard_build(A.indptr, A.indices, ws, rank)
r0, r1 = sh["row0"], sh["row1"]
nrows = r1 - r0
Aloc = sps.csr_matrix((A.data[A.indptr[r0]:A.indptr[r1]], sh["local_col"], sh["local_rowptr"]),
                      shape=(nrows, nrows + len(sh["halo_ids"])))
x = np.random.default_rng(11).uniform(-1.0, 1.0, n)      # the same vector on every rank
x_own = x[r0:r1].copy()

def exchange(v_own):
    """ghost values of this rank from their owners (gloo point to point)"""
    reqs, bufs = [], {}
    for q in range(ws):
        if q == rank:
            continue
        ids = sh["send_ids"][sh["send_rank"] == q]
        if len(ids):
            reqs.append(dist.isend(torch.from_numpy(v_own[ids - r0].copy()), q))
        k = int((sh["halo_owner"] == q).sum())
        if k:
            bufs[q] = torch.empty(k, dtype=torch.float64)
            reqs.append(dist.irecv(bufs[q], q))
    for rq in reqs:
        rq.wait()
    g = np.zeros(len(sh["halo_ids"]))
    for q, b in bufs.items():
        g[sh["halo_owner"] == q] = b.numpy()
    return g

def gdot(a, b):
    t = torch.tensor([float(a @ b)], dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())

y_loc = Aloc @ np.concatenate([x_own, exchange(x_own)])
ok_prod = bool(np.array_equal(y_loc, (A @ x)[r0:r1]))
d = gdot(x_own, y_loc)
# a few Jacobi-preconditioned CG iterations on A x = b, distributed
b = red.rhs()
dinv = 1.0 / A.diagonal()
xs = np.zeros(nrows); r = b[r0:r1].copy(); z = dinv[r0:r1] * r; p = z.copy(); rho = gdot(r, z)
for it in range(25):
    q = Aloc @ np.concatenate([p, exchange(p)])
    alpha = rho / gdot(p, q)
    xs += alpha * p; r -= alpha * q; z = dinv[r0:r1] * r
    rho_new = gdot(r, z); p = z + (rho_new / rho) * p; rho = rho_new
parts = [None] * ws
dist.all_gather_object(parts, (int(r0), xs.tolist()))
xg = np.concatenate([np.array(v) for _, v in sorted(parts)])
print(json.dumps({"rank": rank, "ok_prod": ok_prod, "dot": d, "cg": xg.tolist(), "n_halo": len(sh["halo_ids"])}))
dist.destroy_process_group()
'''


def serial_cg(A, b, iters=25):
    dinv = 1.0 / A.diagonal()
    x = np.zeros(len(b)); r = b.copy(); z = dinv * r; p = z.copy(); rho = r @ z
    for _ in range(iters):
        q = A @ p
        alpha = rho / (p @ q)
        x += alpha * p; r -= alpha * q; z = dinv * r
        rho_new = r @ z; p = z + (rho_new / rho) * p; rho = rho_new
    return x


def test_two_gloo_ranks_reproduce_the_single_process_product_dot_and_cg(tmp_path):
    w = tmp_path / "w.py"
    w.write_text(WORKER)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT="29543",
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(w), ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    assert all(p.returncode == 0 for p in procs), [o[1][-800:] for o in outs]
    res = [json.loads(o[0].strip().splitlines()[-1]) for o in outs]
    spec, A, b = system()
    x = np.random.default_rng(11).uniform(-1.0, 1.0, A.shape[0])
    assert all(r["ok_prod"] for r in res)                       # halo exchange + local rows = global product
    assert all(r["n_halo"] > 0 for r in res)
    d = x @ (A @ x)
    assert all(abs(r["dot"] - d) <= 1e-13 * abs(d) for r in res)
    xc = serial_cg(A, b)
    for r in res:
        assert np.abs(np.array(r["cg"]) - xc).max() <= 1e-10 * np.abs(xc).max()


@pytest.mark.gpu
def test_shard_products_on_the_device_equal_the_global_product():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda:0")
    spec = I.config3_steady_3d(n=24, seed=5)
    s = P.nn_assemble(P.Problem(spec, device=dev))
    d = s.describe()
    nf, nnz = d["n_free"], d["nnz_free"]
    rp = np.zeros(nf + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz)
    P.nn_system_copy_out(s, "A_rowptr", rp)
    P.nn_system_copy_out(s, "A_col", col)
    P.nn_system_copy_out(s, "A_val", val)
    x = torch.tensor(np.random.default_rng(3).uniform(-1, 1, nf), device=dev)
    y = torch.empty_like(x)
    P.nn_spmv(s, x, y, P.NN_FMT_CSR)
    xh = x.cpu().numpy()
    for nranks in (2, 3):
        for r in range(nranks):
            sh = P.nn_shard_build(rp, col, nranks, r)
            r0, r1 = sh["row0"], sh["row1"]
            x_ext = torch.tensor(np.concatenate([xh[r0:r1], xh[sh["halo_ids"]]]), device=dev)
            yl = torch.empty(r1 - r0, dtype=torch.float64, device=dev)
            P.nn_shard_spmv(r1 - r0, torch.tensor(sh["local_rowptr"], device=dev),
                            torch.tensor(sh["local_col"], device=dev),
                            torch.tensor(val[rp[r0]:rp[r1]], device=dev), x_ext, yl)
            torch.cuda.synchronize()
            assert torch.equal(yl, y[r0:r1])      # same rows, same entries, same order
