"""FP64 CPU oracle for the non-negative diffusion QP (arXiv 1506.08435).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference arm of ``bench.py``.  The product
library never imports it, and it imports nothing from the product.

What each function follows:

* ``mesh_structured``  -- P1 simplices (Sec. 2.1.3, k = 1).  Reading: the
  paper's meshes are unstructured; here each square is split along the "/"
  diagonal and each cube into 6 Kuhn tetrahedra (see ``nnqp_oracle.c``).
* ``pattern``          -- sparsity of the Galerkin matrix K (Sec. 2.1.3,
  discrete system K c = f).
* ``assemble``         -- K_e = |e| G^T D G and the consistent capacity
  matrix M_e (Sec. 3.2, pointwise Jacobian F_{1,1} = D and transient
  F_{0,0} = 1/dt), load F_e = f(x_c)|e|/(d+1) (one-point rule: reading).
  ``lumped=True`` replaces M by its row-sum lumping diag(sum_j M_ij), the
  textbook lumped capacity matrix (the paper uses the consistent one; the
  lumped variant is an extension).
* ``eliminate``        -- Dirichlet values c^p on Gamma^D (Sec. 2.1) taken
  out of the unknowns: A = Kt_FF, b = ft_F - Kt_FD c_D with
  Kt = K + M/dt, ft = f + M c^(n)/dt (Sec. 2.2.2; the printed ft uses
  c^(n+1), read as c^(n)).
* ``solve_qp``         -- the unique minimiser of 1/2 x'Ax - b'x on the box
  (Sec. 2.1.3, non-negative formulation; Sec. 2.2.2 with c_min, c_max) by
  MPRGP to a tight KKT tolerance, then an active-set polish that solves the
  face system exactly.
* ``pgs``              -- projected Gauss-Seidel, an independent solver.
* ``brute_force``      -- enumeration of all active sets (tiny problems).
* ``kkt``              -- first-order optimality measure of the box QP.
* ``transient``        -- backward Euler, one warm-started QP per step
  (Sec. 2.2.2 and Algorithm 1).
* ``dsatur``           -- the colouring that orders the unknowns of the SSOR
  preconditioner: Brelaz's saturation-degree greedy rule (Comm. ACM 22,
  1979), ties by larger degree, then smaller index.
* ``ssor_apply``       -- z = M^-1 r for the symmetric SOR matrix
  M = (D + w L) D^-1 (D + w U) / (w (2 - w)) of A_FF with the unknowns
  ordered by (colour, index) (the paper's CG uses block Jacobi/ILU(0),
  Sec. 5 and 5.1; SSOR is the multicolour triangular-sweep counterpart):
  two sparse triangular solves on the permuted matrix.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, textbook special cases, brute force or invariants.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nnqp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_c_dp = ctypes.POINTER(ctypes.c_double)
_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (plain -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_mesh_counts.argtypes = [ctypes.c_int] * 4 + [_c_i64p, _c_i64p]
        L.orc_mesh_structured.argtypes = [ctypes.c_int] * 4 + [_c_dp, _c_i32p]
        L.orc_pattern_rowptr.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _c_i32p, _c_i64p]
        L.orc_pattern_rowptr.restype = ctypes.c_int64
        L.orc_pattern_cols.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _c_i32p, _c_i64p, _c_i32p]
        L.orc_pattern_cols.restype = ctypes.c_int64
        L.orc_assemble.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _c_dp, _c_i32p,
                                   ctypes.c_int, _c_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   _c_dp, _c_i64p, _c_i32p, _c_dp, _c_dp, _c_dp]
        L.orc_assemble.restype = ctypes.c_int
        L.orc_spmv.argtypes = [ctypes.c_int64, _c_i64p, _c_i32p, _c_dp, _c_dp, _c_dp]
        L.orc_kkt.argtypes = [ctypes.c_int64, _c_i64p, _c_i32p, _c_dp, _c_dp, ctypes.c_double,
                              ctypes.c_double, _c_dp, _c_dp]
        L.orc_pgs.argtypes = [ctypes.c_int64, _c_i64p, _c_i32p, _c_dp, _c_dp, ctypes.c_double,
                              ctypes.c_double, _c_dp, ctypes.c_double, ctypes.c_int64]
        L.orc_pgs.restype = ctypes.c_int64
        L.orc_mprgp.argtypes = [ctypes.c_int64, _c_i64p, _c_i32p, _c_dp, _c_dp, ctypes.c_double,
                                ctypes.c_double, _c_dp, ctypes.c_double, ctypes.c_int64, ctypes.c_int]
        L.orc_mprgp.restype = ctypes.c_int64
        L.orc_cg_face.argtypes = [ctypes.c_int64, _c_i64p, _c_i32p, _c_dp, _c_dp, _c_u8p, _c_dp,
                                  ctypes.c_double, ctypes.c_int64]
        L.orc_cg_face.restype = ctypes.c_int64
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


ERRORS = {1: "invalid argument", 2: "degenerate element", 3: "diffusivity not SPD", 4: "NaN/Inf input"}


# --------------------------------------------------------------------------
# mesh, pattern, assembly
# --------------------------------------------------------------------------

def mesh_counts(dim, nx, ny, nz=0):
    N = ctypes.c_int64()
    E = ctypes.c_int64()
    lib().orc_mesh_counts(dim, nx, ny, nz, ctypes.byref(N), ctypes.byref(E))
    return N.value, E.value


def mesh_structured(dim, nx, ny=None, nz=None):
    """Canonical structured P1 mesh of [0,1]^dim: (coords [N,dim] f64, conn [E,dim+1] i32)."""
    ny = nx if ny is None else ny
    nz = (nx if nz is None else nz) if dim == 3 else 0
    N, E = mesh_counts(dim, nx, ny, nz)
    coords = np.zeros((N, dim), np.float64)
    conn = np.zeros((E, dim + 1), np.int32)
    lib().orc_mesh_structured(dim, nx, ny, nz, _p(coords, _c_dp), _p(conn, _c_i32p))
    return coords, conn


def pattern(N, conn):
    """CSR pattern (rowptr int64 [N+1], col int32 [nnz]) of the node graph."""
    conn = np.ascontiguousarray(conn, np.int32)
    E, nv = conn.shape
    rowptr = np.zeros(N + 1, np.int64)
    nnz = lib().orc_pattern_rowptr(N, E, nv, _p(conn, _c_i32p), _p(rowptr, _c_i64p))
    col = np.zeros(nnz, np.int32)
    lib().orc_pattern_cols(N, E, nv, _p(conn, _c_i32p), _p(rowptr, _c_i64p), _p(col, _c_i32p))
    return rowptr, col


class Assembled:
    """Full-node K, M (or None) and F with their common CSR pattern."""

    def __init__(self, rowptr, col, K, M, F):
        self.rowptr, self.col, self.Kval, self.Mval, self.F = rowptr, col, K, M, F
        N = len(rowptr) - 1
        self.N = N
        self.K = sp.csr_matrix((K, col, rowptr), shape=(N, N))
        self.M = None if M is None else sp.csr_matrix((M, col, rowptr), shape=(N, N))


def assemble(coords, conn, coef_kind, coef, aL=0.0, aT=0.0, DM=0.0, f_elem=None, with_mass=False,
             rowptr=None, col=None, lumped=False):
    """Assemble K (and M, F).  coef_kind 0: coef [E, 3|6] upper-triangle tensors;
    coef_kind 1: coef [E, dim] cell velocities (dispersion law, Sec. 5).
    lumped: M is replaced by diag(row sums of the consistent M), stored on the
    same pattern with zero off-diagonal entries."""
    coords = np.ascontiguousarray(coords, np.float64)
    conn = np.ascontiguousarray(conn, np.int32)
    coef = np.ascontiguousarray(coef, np.float64)
    N, dim = coords.shape
    E = conn.shape[0]
    if rowptr is None:
        rowptr, col = pattern(N, conn)
    nnz = int(rowptr[-1])
    K = np.zeros(nnz, np.float64)
    M = np.zeros(nnz, np.float64) if with_mass else None
    F = np.zeros(N, np.float64)
    fe = None if f_elem is None else np.ascontiguousarray(f_elem, np.float64)
    st = lib().orc_assemble(dim, N, E, _p(coords, _c_dp), _p(conn, _c_i32p), coef_kind, _p(coef, _c_dp),
                            aL, aT, DM, None if fe is None else _p(fe, _c_dp), _p(rowptr, _c_i64p),
                            _p(col, _c_i32p), _p(K, _c_dp), None if M is None else _p(M, _c_dp),
                            _p(F, _c_dp))
    if st != 0:
        raise ValueError("oracle assembly failed: " + ERRORS.get(st, str(st)))
    if lumped and M is not None:
        rows = np.repeat(np.arange(N), np.diff(rowptr))
        ML = np.zeros_like(M)
        diag = np.flatnonzero(col == rows)
        ML[diag] = np.add.reduceat(M, rowptr[:-1])[rows[diag]]
        M = ML
    return Assembled(rowptr, col, K, M, F)


# --------------------------------------------------------------------------
# Dirichlet elimination
# --------------------------------------------------------------------------

class Reduced:
    """The QP in the free unknowns: A = Kt_FF and the pieces of b."""

    def __init__(self, asm: Assembled, dmask, dval, dt=0.0):
        dmask = np.asarray(dmask).astype(bool)
        self.asm, self.dmask, self.dt = asm, dmask, dt
        self.dval = np.where(dmask, np.asarray(dval, np.float64), 0.0)
        self.free = np.flatnonzero(~dmask)            # free ids ascending by node id
        self.dirc = np.flatnonzero(dmask)
        Kt = asm.K if dt == 0.0 else (asm.K + asm.M / dt).tocsr()
        self.Kt = Kt
        Kf = Kt[self.free]
        self.A = Kf[:, self.free].tocsr()
        self.A.sort_indices()
        self.A_FD = Kf[:, self.dirc].tocsr()
        self.nF = len(self.free)

    def rhs(self, c_prev_full=None):
        """b = ft_F - Kt_FD c_D, ft = F (steady) or F + M c^(n)/dt (transient)."""
        ft = self.asm.F.copy()
        if self.dt != 0.0:
            ft = ft + (self.asm.M @ c_prev_full) / self.dt
        return ft[self.free] - self.A_FD @ self.dval[self.dirc]

    def full(self, x):
        c = self.dval.copy()
        c[self.free] = x
        return c


def csr_arrays(A):
    A = A.tocsr()
    return (np.ascontiguousarray(A.indptr, np.int64), np.ascontiguousarray(A.indices, np.int32),
            np.ascontiguousarray(A.data, np.float64))


# --------------------------------------------------------------------------
# QP solvers and KKT
# --------------------------------------------------------------------------

def kkt(A, b, lo, hi, x):
    """dict(kkt_rel, kkt_inf, bounds_ok, obj, gp2) for min 1/2x'Ax-b'x on [lo,hi]^n."""
    rp, ci, v = csr_arrays(A)
    b = np.ascontiguousarray(b, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    out = np.zeros(5)
    lib().orc_kkt(len(b), _p(rp, _c_i64p), _p(ci, _c_i32p), _p(v, _c_dp), _p(b, _c_dp), lo, hi,
                  _p(x, _c_dp), _p(out, _c_dp))
    return dict(kkt_rel=out[0], kkt_inf=out[1], bounds_ok=bool(out[2]), obj=out[3], gp2=out[4])


def pgs(A, b, lo, hi, x0=None, tol=1e-15, maxsweep=200000):
    rp, ci, v = csr_arrays(A)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(len(b)) if x0 is None else np.array(x0, np.float64)
    s = lib().orc_pgs(len(b), _p(rp, _c_i64p), _p(ci, _c_i32p), _p(v, _c_dp), _p(b, _c_dp), lo, hi,
                      _p(x, _c_dp), tol, maxsweep)
    return x, int(s)


def mprgp(A, b, lo, hi, x0=None, rtol=1e-12, maxit=10_000_000, threads=1):
    rp, ci, v = csr_arrays(A)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(len(b)) if x0 is None else np.array(x0, np.float64)
    it = lib().orc_mprgp(len(b), _p(rp, _c_i64p), _p(ci, _c_i32p), _p(v, _c_dp), _p(b, _c_dp), lo, hi,
                         _p(x, _c_dp), rtol, maxit, threads)
    return x, int(it)


def _face_solve(A, b, fixed, x, tol=1e-14):
    """Solve A_FF x_F = b_F - A_FA x_A (F = not fixed), keeping x_A."""
    y = np.array(x, np.float64)
    F = np.flatnonzero(~fixed)
    if len(F) == 0:
        return y
    if len(F) <= 2000:
        Ad = A[F].toarray()
        rhs = b[F] - Ad[:, fixed] @ y[fixed]
        y[F] = np.linalg.solve(Ad[:, F], rhs)
        return y
    rp, ci, v = csr_arrays(A)
    fx = np.ascontiguousarray(fixed, np.uint8)
    bb = np.ascontiguousarray(b, np.float64)
    lib().orc_cg_face(len(b), _p(rp, _c_i64p), _p(ci, _c_i32p), _p(v, _c_dp), _p(bb, _c_dp),
                      _p(fx, _c_u8p), _p(y, _c_dp), tol, 100 * len(b) + 1000)
    return y


def solve_qp(A, b, lo, hi, x0=None, rtol=1e-12, threads=1, maxit=10_000_000):
    """Unique minimiser of 1/2 x'Ax - b'x on [lo,hi]^n (A SPD).

    MPRGP to ||gP|| <= rtol * ||b||, then an active-set polish: entries
    exactly at a bound are held fixed and the face system is solved to
    roundoff; entries that leave the box are fixed at the bound they crossed,
    and if a fixed entry's gradient has the wrong sign MPRGP resumes from the
    polished point.  Returns (x, info)."""
    A = A.tocsr()
    b = np.asarray(b, np.float64)
    x, it = mprgp(A, b, lo, hi, x0, rtol=rtol, maxit=maxit, threads=threads)
    info = dict(mprgp_iters=it, polish_rounds=0, polished=False)
    gscale = max(np.abs(b).max() if len(b) else 0.0, 1e-300)
    for r in range(12):
        info["polish_rounds"] = r + 1
        fixed = (x <= lo) | (x >= hi)
        y = _face_solve(A, b, fixed, x)
        out = (~fixed) & ((y < lo) | (y > hi))
        if out.any():
            x = np.clip(y, lo, hi)
            continue
        g = A @ y - b
        wrong = (fixed & (y <= lo) & (g < -1e-11 * gscale)) | (fixed & (y >= hi) & (g > 1e-11 * gscale))
        if wrong.any():
            x, it2 = mprgp(A, b, lo, hi, y, rtol=rtol * 1e-2, maxit=maxit, threads=threads)
            info["mprgp_iters"] += abs(it2)
            continue
        x = y
        info["polished"] = True
        break
    return x, info


def galerkin(A, b):
    """Unconstrained Galerkin solve A x = b (Sec. 2.1.3, K c = f)."""
    A = A.tocsr()
    if A.shape[0] <= 4000:
        return np.linalg.solve(A.toarray(), b)
    import scipy.sparse.linalg as spl
    return spl.spsolve(A.tocsc(), b)


def brute_force(A, b, lo, hi, tol=1e-9):
    """All KKT points found by enumerating every assignment of each unknown
    to {free, at lo} (one-sided, hi = inf) or {free, at lo, at hi}: the face
    system is solved densely and kept when it is feasible and the multipliers
    have the right sign.  For an SPD A exactly one survives.  Tiny n only."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    n = len(b)
    states = [0, 1] if not np.isfinite(hi) else [0, 1, 2]
    if not np.isfinite(lo):
        states = [0, 2] if np.isfinite(hi) else [0]
    sols = []
    bs = max(np.abs(b).max(), 1.0)
    for assign in itertools.product(states, repeat=n):
        a = np.array(assign)
        x = np.zeros(n)
        x[a == 1] = lo
        x[a == 2] = hi
        F = np.flatnonzero(a == 0)
        if len(F):
            rhs = b[F] - Ad[np.ix_(F, np.flatnonzero(a != 0))] @ x[a != 0]
            x[F] = np.linalg.solve(Ad[np.ix_(F, F)], rhs)
        if (x[F] < lo - tol).any() or (x[F] > hi + tol).any():
            continue
        g = Ad @ x - b
        if (g[a == 1] < -tol * bs).any() or (g[a == 2] > tol * bs).any():
            continue
        sols.append((x, a))
    return sols


def transient(red: Reduced, c0_full, lo, hi, nsteps, rtol=1e-12, threads=1):
    """Backward Euler (Sec. 2.2.2): per step b = ft_F - Kt_FD c_D with
    ft = F + M c^(n)/dt, QP warm-started from c^(n).  Returns the list of
    full-node states c^(1..nsteps)."""
    c = np.array(c0_full, np.float64)
    out = []
    for _ in range(nsteps):
        b = red.rhs(c)
        x, _info = solve_qp(red.A, b, lo, hi, x0=c[red.free], rtol=rtol, threads=threads)
        c = red.full(x)
        out.append(c)
    return out


def objective(A, b, x):
    return 0.5 * x @ (A @ x) - b @ x


# --------------------------------------------------------------------------
# SSOR preconditioner
# --------------------------------------------------------------------------

def dsatur(A):
    """Colour of each vertex of the graph of A's pattern (diagonal ignored):
    repeatedly the uncoloured vertex with the most distinct colours among its
    neighbours takes the smallest colour none of them has; ties go to the
    vertex with more neighbours, then to the smaller index."""
    import heapq
    A = sp.csr_matrix(A)
    n = A.shape[0]
    nbrs = [[int(j) for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i] for i in range(n)]
    color = [-1] * n
    sat = [set() for _ in range(n)]
    heap = [(0, -len(nbrs[i]), i) for i in range(n)]
    heapq.heapify(heap)
    while heap:
        s_neg, d_neg, v = heapq.heappop(heap)
        if color[v] >= 0 or -s_neg != len(sat[v]):
            continue                      # coloured, or an older entry of v
        c = 0
        while c in sat[v]:
            c += 1
        color[v] = c
        for j in nbrs[v]:
            if color[j] < 0 and c not in sat[j]:
                sat[j].add(c)
                heapq.heappush(heap, (-len(sat[j]), -len(nbrs[j]), j))
    return np.array(color, np.int32)


def ssor_apply(A, color, r, omega=1.0, face=None):
    """z = M_F^-1 r_F on the face F (all unknowns if face is None; z = 0
    outside F), M the SSOR matrix of A_FF with the unknowns of F ordered by
    (colour, index): y = (D + w L)^-1 r, then z = w (2 - w) (D + w U)^-1 D y."""
    import scipy.sparse.linalg as spl
    A = sp.csr_matrix(A)
    n = A.shape[0]
    F = np.arange(n) if face is None else np.flatnonzero(np.asarray(face) != 0)
    z = np.zeros(n)
    if len(F) == 0:
        return z
    order = F[np.lexsort((F, np.asarray(color)[F]))]
    Ap = A[order][:, order].tocsr()
    D = sp.diags(Ap.diagonal())
    L = sp.tril(Ap, k=-1)
    U = sp.triu(Ap, k=1)
    y = spl.spsolve_triangular((D + omega * L).tocsr(), np.asarray(r, np.float64)[order], lower=True)
    zp = spl.spsolve_triangular((D + omega * U).tocsr(), D @ y, lower=False)
    z[order] = omega * (2.0 - omega) * zp
    return z
