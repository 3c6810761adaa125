"""Seeded synthetic problem data for the non-negative diffusion QP.

This module only *describes problems*: mesh sizes, per-element coefficient
samples, per-element sources, Dirichlet masks/values, bounds and time
steps.  It holds none of the method's arithmetic (no element matrices, no
elimination, no solver).  It is the one module that both the FP64 oracle
and the CUDA path consume, so that both see bit-identical inputs.

The paper (arXiv 1506.08435) runs on unstructured tetrahedral meshes of a
cube with a hole (Sec. 5.1) and a site model (Sec. 5.2) that are not
available; these seeded structured workloads stand in for them, with the
paper's dispersion law and dispersivities (Sec. 5, alpha_L = 1,
alpha_T = 1e-3) and bounds 0 <= c <= 1 (Sec. 5 remark on the DMP).

Cell-wise coefficients are sampled at element centroids (Algorithm 1 takes
a cell-wise velocity as input).  Centroids of the canonical structured mesh
are formed from the lattice indices as exact rationals, e.g. the 2D
triangle T0 of square (i, j) has centroid ((3i+2)/(3n), (3j+1)/(3n)).

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), stream
(seed, k) starting from state seed ^ (k * 0xD1B54A32D192ED03) mod 2^64;
uniforms are the top 53 bits times 2^-53; normals use Box-Muller.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1

KIND_TENSOR = 0    # coef[e] = upper triangle of D_e (2D: xx, xy, yy; 3D: xx, xy, xz, yy, yz, zz)
KIND_VELOCITY = 1  # coef[e] = cell velocity v_e; D_e from the dispersion law


class SplitMix64:
    def __init__(self, seed: int, stream: int = 0):
        self.s = (seed ^ ((stream * 0xD1B54A32D192ED03) & MASK64)) & MASK64

    def u64(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & MASK64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        u1 = self.uniform()
        while u1 == 0.0:
            u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclass
class ProblemSpec:
    """One QP workload on a structured P1 mesh of [0,1]^dim."""
    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    coef_kind: int
    coef: np.ndarray                 # [E, 3|6] tensors or [E, dim] velocities, float64
    f_elem: np.ndarray | None        # [E] float64 or None (f = 0)
    dmask: np.ndarray                # [N] uint8, 1 = Dirichlet node
    dval: np.ndarray                 # [N] float64, value at Dirichlet nodes (0 elsewhere)
    lo: float
    hi: float
    aL: float = 0.0
    aT: float = 0.0
    DM: float = 0.0
    dt: float = 0.0                  # 0 = steady
    nsteps: int = 0
    c0: np.ndarray | None = None     # [N] initial state for the transient case
    meta: dict = field(default_factory=dict)
    coords: np.ndarray | None = None  # explicit mesh [N, dim] (None: the structured mesh nx, ny, nz)
    conn: np.ndarray | None = None    # explicit connectivity [E, dim+1] int32

    @property
    def n_nodes(self) -> int:
        if self.coords is not None:
            return int(self.coords.shape[0])
        if self.dim == 2:
            return (self.nx + 1) * (self.ny + 1)
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_elems(self) -> int:
        if self.conn is not None:
            return int(self.conn.shape[0])
        return 2 * self.nx * self.ny if self.dim == 2 else 6 * self.nx * self.ny * self.nz


# ---------------------------------------------------------------- lattice helpers

def element_lattice_2d(nx, ny):
    """Per element: (i, j, t) of its square and triangle index, element order."""
    j, i, t = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(2), indexing="ij")
    return i.ravel(), j.ravel(), t.ravel()


_PERMS = np.array([[0, 1, 2], [0, 2, 1], [1, 0, 2], [1, 2, 0], [2, 0, 1], [2, 1, 0]])


def element_lattice_3d(nx, ny, nz):
    """Per element: (i, j, k, p) of its hexahedron and tetrahedron index."""
    k, j, i, p = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), np.arange(6), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel(), p.ravel()


def centroid_numerators_2d(nx, ny):
    """Centroid of every triangle as integer numerators over (3nx, 3ny)."""
    i, j, t = element_lattice_2d(nx, ny)
    cx = 3 * i + np.where(t == 0, 2, 1)
    cy = 3 * j + np.where(t == 0, 1, 2)
    return cx, cy


def centroid_numerators_3d(nx, ny, nz):
    """Centroid of every tetrahedron as integer numerators over (4nx, 4ny, 4nz):
    the vertices are v0, v0+e_p0, v0+e_p0+e_p1, v0+e_p0+e_p1+e_p2, so the
    centroid is v0 + (3 e_p0 + 2 e_p1 + e_p2)/4."""
    i, j, k, p = element_lattice_3d(nx, ny, nz)
    off = np.zeros((len(p), 3), np.int64)
    for s, w in enumerate((3, 2, 1)):
        ax = _PERMS[p, s]
        off[np.arange(len(p)), ax] += w
    return 4 * i + off[:, 0], 4 * j + off[:, 1], 4 * k + off[:, 2]


def boundary_mask_2d(nx, ny):
    j, i = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return ((i == 0) | (i == nx) | (j == 0) | (j == ny)).ravel().astype(np.uint8)


def boundary_mask_3d(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    b = (i == 0) | (i == nx) | (j == 0) | (j == ny) | (k == 0) | (k == nz)
    return b.ravel().astype(np.uint8)


def patch_dirichlet_3d(nx, ny, nz):
    """c = 1 on the patch (y, z) in [1/4, 3/4]^2 of the face x = 0 and c = 0
    on the face x = 1; the other faces carry the natural zero-flux condition.
    Integer tests only (4j >= ny, 4j <= 3ny, same for k)."""
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    patch = (i == 0) & (4 * j >= ny) & (4 * j <= 3 * ny) & (4 * k >= nz) & (4 * k <= 3 * nz)
    far = i == nx
    mask = (patch | far).ravel().astype(np.uint8)
    val = np.where(patch.ravel(), 1.0, 0.0)
    return mask, val


def rotated_tensor(theta, lam1, lam2):
    """Upper triangle (xx, xy, yy) of R(theta) diag(lam1, lam2) R(theta)^T."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([lam1 * c * c + lam2 * s * s, (lam1 - lam2) * c * s, lam1 * s * s + lam2 * c * c])


def vortex_velocity(x, y):
    """v = (sin 2 pi x cos 2 pi y, -cos 2 pi x sin 2 pi y, 0.1): |v| >= 0.1."""
    tpx, tpy = 2.0 * np.pi * x, 2.0 * np.pi * y
    return np.stack([np.sin(tpx) * np.cos(tpy), -np.cos(tpx) * np.sin(tpy), np.full_like(x, 0.1)], axis=1)


def quaternion_rotation(rng: SplitMix64):
    q = np.array([rng.normal() for _ in range(4)])
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


# ---------------------------------------------------------------- the workloads

def square_box_source(nx, ny, x0, x1, y0, y1):
    """f_e = 1 where the centroid lies in [x0,x1] x [y0,y1] (closed), else 0."""
    cx, cy = centroid_numerators_2d(nx, ny)
    xc, yc = cx / (3.0 * nx), cy / (3.0 * ny)
    return ((xc >= x0) & (xc <= x1) & (yc >= y0) & (yc <= y1)).astype(np.float64)


def config1_steady_2d(n=50, theta=math.pi / 6, lam1=1000.0, lam2=1.0):
    """2D unit square, n x n squares split "/" into 2 n^2 triangles, constant
    D = R(theta) diag(lam1, lam2) R(theta)^T, f = 1 on [3/8, 5/8]^2 (centroid
    rule, integer test), c = 0 on the whole boundary, c >= 0."""
    E = 2 * n * n
    coef = np.tile(rotated_tensor(theta, lam1, lam2), (E, 1))
    cx, cy = centroid_numerators_2d(n, n)
    inside = (8 * cx >= 9 * n) & (8 * cx <= 15 * n) & (8 * cy >= 9 * n) & (8 * cy <= 15 * n)
    mask = boundary_mask_2d(n, n)
    return ProblemSpec("steady2d_n%d" % n, 2, n, n, 0, KIND_TENSOR, coef, inside.astype(np.float64),
                       mask, np.zeros(len(mask)), 0.0, math.inf)


def dispersion_velocities_3d(nx, ny, nz, rotate_seed=None, block=10):
    cx, cy, cz = centroid_numerators_3d(nx, ny, nz)
    v = vortex_velocity(cx / (4.0 * nx), cy / (4.0 * ny))
    if rotate_seed is not None:
        i, j, k, _ = element_lattice_3d(nx, ny, nz)
        nbx, nby, nbz = -(-nx // block), -(-ny // block), -(-nz // block)
        bid = (i // block) + nbx * ((j // block) + nby * (k // block))
        Q = np.stack([quaternion_rotation(SplitMix64(rotate_seed, b)) for b in range(nbx * nby * nbz)])
        v = np.einsum("eij,ej->ei", Q[bid], v)
    return np.ascontiguousarray(v)


def config2_transient_3d(n=40, dt=0.01, nsteps=50):
    """3D unit cube, n^3 hexes x 6 tets, dispersion law with the vortex
    velocity, alpha_L = 1, alpha_T = 1e-3, D_M = 1e-9; c = 1 on the x = 0
    patch, c = 0 on x = 1, 0 <= c <= 1, backward Euler with dt over nsteps
    steps from c0 = 0 (Dirichlet values at Dirichlet nodes)."""
    v = dispersion_velocities_3d(n, n, n)
    mask, val = patch_dirichlet_3d(n, n, n)
    c0 = np.where(mask == 1, val, 0.0)
    return ProblemSpec("transient3d_n%d" % n, 3, n, n, n, KIND_VELOCITY, v, None, mask, val, 0.0, 1.0,
                       aL=1.0, aT=1e-3, DM=1e-9, dt=dt, nsteps=nsteps, c0=c0)


def config3_steady_3d(n=150, seed=1506):
    """3D unit cube, n^3 hexes x 6 tets, the config-2 dispersion field with a
    seeded uniform random rotation of v per 10^3 block of hexes (alpha_L /
    alpha_T = 1e3), same boundary data, steady, 0 <= c <= 1."""
    v = dispersion_velocities_3d(n, n, n, rotate_seed=seed)
    mask, val = patch_dirichlet_3d(n, n, n)
    return ProblemSpec("steady3d_n%d" % n, 3, n, n, n, KIND_VELOCITY, v, None, mask, val, 0.0, 1.0,
                       aL=1.0, aT=1e-3, DM=1e-9)


def config4_instance(i, seed=8435, nmin=20, nmax=200):
    """Instance i of the batch: n ~ U{nmin..nmax}, theta ~ U(0, pi),
    ratio = 10^U(1,4), D = R(theta) diag(ratio, 1) R(theta)^T, box source with
    lower corner ~ U(0, 0.7)^2 and widths ~ U(0.1, 0.3) (clipped to [0,1]),
    c = 0 on the boundary, c >= 0."""
    r = SplitMix64(seed, i)
    n = nmin + int(r.uniform() * (nmax - nmin + 1))
    theta = math.pi * r.uniform()
    ratio = 10.0 ** (1.0 + 3.0 * r.uniform())
    a, c = 0.7 * r.uniform(), 0.7 * r.uniform()
    wx, wy = 0.1 + 0.2 * r.uniform(), 0.1 + 0.2 * r.uniform()
    E = 2 * n * n
    coef = np.tile(rotated_tensor(theta, ratio, 1.0), (E, 1))
    f = square_box_source(n, n, a, min(a + wx, 1.0), c, min(c + wy, 1.0))
    mask = boundary_mask_2d(n, n)
    return ProblemSpec("batch2d_%d_n%d" % (i, n), 2, n, n, 0, KIND_TENSOR, coef, f, mask,
                       np.zeros(len(mask)), 0.0, math.inf, meta=dict(theta=theta, ratio=ratio))


def config4_batch(count=512, seed=8435, nmin=20, nmax=200):
    return [config4_instance(i, seed, nmin, nmax) for i in range(count)]


def serve_request(r, seed=2015):
    """Request r of the serving stream: 2D or 3D with probability 1/2.
    2D: N ~ log-U[1e3, 2.5e5], n = round(sqrt N) - 1, boundary c = 0 and a
    random box source; per 10^2 block of squares a seeded direction theta_b
    and the dispersion law with |v| of the vortex field at (x, y, 0), i.e.
    v_e = |v(x_c)| (cos theta_b, sin theta_b).  3D: N ~ log-U[1e4, 1e6],
    n = round(cbrt N) - 1, the config-3 field with seed (seed, r), patch
    boundary data.  0 <= c <= 1 for both."""
    g = SplitMix64(seed, 1_000_000 + r)
    is3d = g.uniform() < 0.5
    if is3d:
        N = math.exp(math.log(1e4) + g.uniform() * (math.log(1e6) - math.log(1e4)))
        n = max(2, int(round(N ** (1.0 / 3.0))) - 1)
        v = dispersion_velocities_3d(n, n, n, rotate_seed=(seed * 1_000_003 + r) & MASK64)
        mask, val = patch_dirichlet_3d(n, n, n)
        return ProblemSpec("serve3d_%d_n%d" % (r, n), 3, n, n, n, KIND_VELOCITY, v, None, mask, val, 0.0, 1.0,
                           aL=1.0, aT=1e-3, DM=1e-9)
    N = math.exp(math.log(1e3) + g.uniform() * (math.log(2.5e5) - math.log(1e3)))
    n = max(2, int(round(math.sqrt(N))) - 1)
    cx, cy = centroid_numerators_2d(n, n)
    xc, yc = cx / (3.0 * n), cy / (3.0 * n)
    speed = np.linalg.norm(vortex_velocity(xc, yc), axis=1)
    i, j, _ = element_lattice_2d(n, n)
    nb = -(-n // 10)
    bid = (i // 10) + nb * (j // 10)
    th = np.array([math.pi * SplitMix64(seed * 7 + r, b).uniform() for b in range(nb * nb)])
    v = np.stack([speed * np.cos(th[bid]), speed * np.sin(th[bid])], axis=1)
    a, c = 0.7 * g.uniform(), 0.7 * g.uniform()
    wx, wy = 0.1 + 0.2 * g.uniform(), 0.1 + 0.2 * g.uniform()
    f = square_box_source(n, n, a, min(a + wx, 1.0), c, min(c + wy, 1.0))
    mask = boundary_mask_2d(n, n)
    return ProblemSpec("serve2d_%d_n%d" % (r, n), 2, n, n, 0, KIND_VELOCITY, np.ascontiguousarray(v), f,
                       mask, np.zeros(len(mask)), 0.0, 1.0, aL=1.0, aT=1e-3, DM=1e-9)


def serve_arrivals(rate=200.0, duration=60.0, seed=2015):
    """Poisson arrival times (s) at the given rate over [0, duration)."""
    g = SplitMix64(seed, 0)
    t, out = 0.0, []
    while True:
        u = g.uniform()
        t += -math.log(1.0 - u) / rate
        if t >= duration:
            return out
        out.append(t)


def tiny_2d(nx, ny, theta=math.pi / 6, lam1=1000.0, lam2=1.0, hi=math.inf, source_cell=(1, 1)):
    """Small 2D problem with every boundary node Dirichlet 0, a constant
    rotated tensor and f = 1 on the two triangles of one square (None: f = 1
    everywhere): the brute-force test meshes."""
    E = 2 * nx * ny
    coef = np.tile(rotated_tensor(theta, lam1, lam2), (E, 1))
    if source_cell is None:
        f = np.ones(E)
    else:
        f = np.zeros(E)
        q = source_cell[0] + nx * source_cell[1]
        f[2 * q:2 * q + 2] = 1.0
    mask = boundary_mask_2d(nx, ny)
    return ProblemSpec("tiny2d_%dx%d" % (nx, ny), 2, nx, ny, 0, KIND_TENSOR, coef, f, mask,
                       np.zeros(len(mask)), 0.0, hi)


def tiny_3d(n, tensor, hi=math.inf, source_cell=(0, 0, 0)):
    """Small 3D analogue of tiny_2d: f = 1 on the six tetrahedra of one hex."""
    E = 6 * n ** 3
    coef = np.tile(np.asarray(tensor, np.float64), (E, 1))
    if source_cell is None:
        f = np.ones(E)
    else:
        f = np.zeros(E)
        q = source_cell[0] + n * (source_cell[1] + n * source_cell[2])
        f[6 * q:6 * q + 6] = 1.0
    mask = boundary_mask_3d(n, n, n)
    return ProblemSpec("tiny3d_%d" % n, 3, n, n, n, KIND_TENSOR, coef, f, mask,
                       np.zeros(len(mask)), 0.0, hi)


def kuhn_mesh_without_box(n, box_lo, box_hi):
    """Explicit mesh of the unit cube cut into n^3 hexahedra, each split into
    the 6 Kuhn tetrahedra of the structured mesh (same vertex order), with the
    hexahedra (i, j, k) that have box_lo <= i, j, k < box_hi removed.  Nodes
    that no element uses (strictly inside the box) are dropped; the others
    keep the lattice order i + (n+1)(j + (n+1)k).  Returns (coords [N, 3],
    conn [E, 4] int32, lattice ids [N] of the kept nodes)."""
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    inside = ((ii >= box_lo) & (ii < box_hi) & (jj >= box_lo) & (jj < box_hi) &
              (kk >= box_lo) & (kk < box_hi))
    ii, jj, kk = ii[~inside], jj[~inside], kk[~inside]
    unit = np.eye(3, dtype=np.int64)
    m = n + 1
    tets = []
    for p in _PERMS:
        v = np.stack([ii, jj, kk], axis=1).astype(np.int64)
        verts = [v.copy()]
        for a in p:
            v = v + unit[a]
            verts.append(v.copy())
        tets.append(np.stack([w[:, 0] + m * (w[:, 1] + m * w[:, 2]) for w in verts], axis=1))
    lat = np.stack(tets, axis=1).reshape(-1, 4)      # hexahedron-major, then permutation
    used, conn = np.unique(lat, return_inverse=True)
    conn = conn.reshape(-1, 4).astype(np.int32)
    i = used % m
    j = (used // m) % m
    k = used // (m * m)
    coords = np.stack([i, j, k], axis=1).astype(np.float64) / n
    return coords, conn, used


def cube_with_hole(m, mesh="mirrored"):
    """Structured analogue of the cube with a cubic hole (Sec. 5.1): n = 9m
    hexahedra per side, the hole [4/9, 5/9]^3 = hexahedra 4m <= i, j, k < 5m
    removed; c = 0 on the outer boundary, c = 1 on the hole's boundary, f = 0,
    v = e_x + e_y + e_z on every element, alpha_L = 1, alpha_T = 1e-3,
    D_M = 0, bounds 0 <= c <= 1.  The paper's meshes are unstructured
    tetrahedral meshes (types A, B, C) that are not available; two
    structured types stand in:
      "kuhn":     the Kuhn split, whose hexahedron diagonals run along v;
      "mirrored": the same connectivity with x -> 1 - x, diagonals along
                  (-1, 1, 1) (the physical problem is symmetric under the
                  mirror, so only the mesh changes)."""
    if mesh not in ("kuhn", "mirrored"):
        raise ValueError("mesh must be 'kuhn' or 'mirrored'")
    n = 9 * m
    coords, conn, lat = kuhn_mesh_without_box(n, 4 * m, 5 * m)
    if mesh == "mirrored":
        coords[:, 0] = (n - lat % (n + 1)) / n
    N = len(coords)
    i, j, k = lat % (n + 1), (lat // (n + 1)) % (n + 1), lat // ((n + 1) ** 2)
    outer = (i == 0) | (i == n) | (j == 0) | (j == n) | (k == 0) | (k == n)
    hole = ((i >= 4 * m) & (i <= 5 * m) & (j >= 4 * m) & (j <= 5 * m) & (k >= 4 * m) & (k <= 5 * m))
    mask = (outer | hole).astype(np.uint8)
    val = np.where(hole, 1.0, 0.0)
    v = np.ones((len(conn), 3))
    return ProblemSpec("cube_hole_%s_m%d" % (mesh, m), 3, n, n, n, KIND_VELOCITY, v, None, mask, val, 0.0, 1.0,
                       aL=1.0, aT=1e-3, DM=0.0, coords=coords, conn=conn, meta={"mesh": mesh, "m": m})
