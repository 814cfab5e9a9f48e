"""Seeded synthetic inputs for cell-wise assembly: meshes, cell-node maps and coefficient Dats.

This module only *describes* inputs.  It holds none of the assembly arithmetic (no basis
functions, quadrature, Jacobians or element tensors) and is the one module shared by the
CUDA path's tests/benchmarks and the CPU oracle's tests.

Conventions (the paper uses unstructured meshes and leaves numbering to DMPlex, Sec. 3.4;
these structured stand-ins fix it as follows):

* UnitSquareMesh(n): vertices (i, j), 0 <= i, j <= n, id ``i + (n+1) j``, coordinates
  ``(i/n, j/n)``.  Square (i, j) (j outer, i inner) is split along its (0,0)-(1,1)
  diagonal into cell ``2(jn+i)`` = (v00, v10, v11) and cell ``2(jn+i)+1`` = (v00, v11, v01);
  both are counter-clockwise.
* UnitCubeMesh(n): vertices (i, j, k), id ``i + (n+1)(j + (n+1)k)``.  Cube (i, j, k)
  (k outer, i inner) is split into the 6 Kuhn tetrahedra, one per axis permutation
  ``pi`` in lexicographic order: v0 = (0,0,0), v1 = e_pi0, v2 = e_pi0 + e_pi1, v3 = (1,1,1).
* Jitter: every coordinate of every interior vertex moves by an independent
  uniform[-a h, a h] draw from ``numpy.random.default_rng(seed)``, drawn as one array of
  shape ``(n-1,)*dim + (dim,)`` indexed by ``(i-1, j-1[, k-1], c)``.  Boundary vertices stay
  put, so the domain stays the unit square/cube.  Inverted cells are refused.
* Lagrange P_p nodes of a cell are the lattice points ``sum_m alpha_m x_m / p`` with
  ``alpha`` a multi-index, ``|alpha| = p``.  Local order: vertices 0..d; then edges (a, b),
  a < b, in lexicographic order, each walked from a to b (alpha_a = p - t, alpha_b = t,
  t = 1..p-1); then faces (a, b, c), a < b < c, lexicographic, interior points by
  descending alpha_a then alpha_b; then (3D) cell-interior points by descending
  alpha_0, alpha_1, alpha_2.  Global node numbers are lexicographic on the fine grid of
  ``(p n + 1)^dim`` lattice points: fine coordinates ``sum_m alpha_m V_m`` with V_m the
  integer grid coordinates of the cell's vertices.
"""
from __future__ import annotations

from dataclasses import dataclass
from itertools import combinations, permutations

import numpy as np

__all__ = [
    "Mesh", "unit_square_mesh", "unit_cube_mesh", "lagrange_nodes", "cell_node_map",
    "node_coordinates", "uniform_dat", "lognormal_dat", "batch_mesh_sizes", "boundary_nodes",
    "manufactured_sine", "serve_requests", "face_nodes",
]


@dataclass
class Mesh:
    """A structured simplicial mesh of the unit square (dim 2) or cube (dim 3)."""
    dim: int
    n: int
    coords: np.ndarray       # [nvert, dim] float64
    cell_vertex: np.ndarray  # [ncell, dim+1] int32 (the coordinate map)
    vgrid: np.ndarray        # [nvert, dim] int64 integer grid coordinates of the vertices

    @property
    def ncell(self) -> int:
        return int(self.cell_vertex.shape[0])

    @property
    def nvert(self) -> int:
        return int(self.coords.shape[0])


def _jitter(n: int, dim: int, amount: float, seed: int | None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    return rng.uniform(-amount * h, amount * h, size=(n - 1,) * dim + (dim,))


def unit_square_mesh(n: int, jitter: float = 0.0, seed: int | None = None) -> Mesh:
    """Right-diagonal triangulation of [0,1]^2 with n x n squares (2 n^2 cells)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")  # [j, i]
    vgrid = np.stack([i.ravel(), j.ravel()], axis=1).astype(np.int64)       # id = i + (n+1) j
    coords = vgrid.astype(np.float64) / n
    if jitter > 0.0 and n > 1:
        d = _jitter(n, 2, jitter, seed)                                       # [i-1, j-1, c]
        ii, jj = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
        ids = (ii + (n + 1) * jj).ravel()
        coords[ids] += d.reshape(-1, 2)
    sq_i, sq_j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    sq_i, sq_j = sq_i.ravel(), sq_j.ravel()                                   # square index = j n + i
    v00 = sq_i + (n + 1) * sq_j
    v10, v01, v11 = v00 + 1, v00 + (n + 1), v00 + (n + 2)
    cells = np.empty((2 * n * n, 3), dtype=np.int32)
    cells[0::2] = np.stack([v00, v10, v11], axis=1)
    cells[1::2] = np.stack([v00, v11, v01], axis=1)
    mesh = Mesh(2, n, coords, cells, vgrid)
    _check_orientation(mesh)
    return mesh


_KUHN_PERMS = list(permutations(range(3)))  # lexicographic: (0,1,2), (0,2,1), ..., (2,1,0)


def unit_cube_mesh(n: int, jitter: float = 0.0, seed: int | None = None) -> Mesh:
    """Kuhn (6 tets per cube) triangulation of [0,1]^3 with n^3 cubes (6 n^3 cells)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    r = np.arange(n + 1)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")                              # id = i + (n+1)(j + (n+1)k)
    vgrid = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int64)
    coords = vgrid.astype(np.float64) / n
    if jitter > 0.0 and n > 1:
        d = _jitter(n, 3, jitter, seed)                                       # [i-1, j-1, k-1, c]
        ii, jj, kk = np.meshgrid(np.arange(1, n), np.arange(1, n), np.arange(1, n), indexing="ij")
        ids = (ii + (n + 1) * (jj + (n + 1) * kk)).ravel()
        coords[ids] += d.reshape(-1, 3)
    c = np.arange(n)
    ck, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    base = (ci + (n + 1) * (cj + (n + 1) * ck)).ravel()                       # cube order: k outer, i inner
    stride = np.array([1, n + 1, (n + 1) ** 2], dtype=np.int64)
    cells = np.empty((base.size, 6, 4), dtype=np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        off = np.zeros(3, dtype=np.int64)
        cells[:, t, 0] = base
        for m in range(3):
            off[perm[m]] += 1
            cells[:, t, m + 1] = base + int(off @ stride)
    mesh = Mesh(3, n, coords, cells.reshape(-1, 4).astype(np.int32), vgrid)
    _check_orientation(mesh)
    return mesh


def _signed_volumes(mesh: Mesh, coords: np.ndarray) -> np.ndarray:
    x = coords[mesh.cell_vertex]                                              # [ncell, d+1, d]
    e = x[:, 1:, :] - x[:, :1, :]
    return np.linalg.det(e)


def _check_orientation(mesh: Mesh) -> None:
    """Refuse meshes whose jitter inverted or flattened a cell (orientation must match the lattice)."""
    ref = np.sign(_signed_volumes(mesh, mesh.vgrid.astype(np.float64)))
    cur = _signed_volumes(mesh, mesh.coords)
    h = 1.0 / mesh.n
    if np.any(np.sign(cur) != ref) or np.any(np.abs(cur) < 1e-3 * h ** mesh.dim):
        raise ValueError("jitter produced an inverted or degenerate cell; use a smaller jitter")


def lagrange_nodes(dim: int, p: int) -> np.ndarray:
    """Multi-indices alpha (|alpha| = p) of the P_p lattice nodes of a dim-simplex, in local order."""
    if p < 1:
        raise ValueError("degree must be >= 1")
    nv = dim + 1
    out: list[tuple[int, ...]] = []
    for m in range(nv):
        a = [0] * nv
        a[m] = p
        out.append(tuple(a))
    for a_, b_ in combinations(range(nv), 2):
        for t in range(1, p):
            a = [0] * nv
            a[a_], a[b_] = p - t, t
            out.append(tuple(a))
    for face in combinations(range(nv), 3):
        if dim == 2 and face != (0, 1, 2):
            continue
        pts = []
        for aa in range(p - 2, 0, -1):
            for bb in range(p - 1 - aa, 0, -1):
                cc = p - aa - bb
                if cc >= 1:
                    pts.append((aa, bb, cc))
        for aa, bb, cc in pts:
            a = [0] * nv
            a[face[0]], a[face[1]], a[face[2]] = aa, bb, cc
            out.append(tuple(a))
    if dim == 3:
        for a0 in range(p - 3, 0, -1):
            for a1 in range(p - 2 - a0, 0, -1):
                for a2 in range(p - 1 - a0 - a1, 0, -1):
                    a3 = p - a0 - a1 - a2
                    if a3 >= 1:
                        out.append((a0, a1, a2, a3))
    return np.array(out, dtype=np.int64)


def cell_node_map(mesh: Mesh, p: int) -> tuple[np.ndarray, int]:
    """Cell -> P_p node map ``[ncell, nd]`` int32 and the number of nodes ``(p n + 1)^dim``."""
    alpha = lagrange_nodes(mesh.dim, p).astype(np.int64)                      # [nd, d+1]
    m = p * mesh.n + 1
    # node k of a cell sits at fine-grid point sum_v alpha[k, v] * vgrid[v]; its id is linear in it
    w = m ** np.arange(mesh.dim, dtype=np.int64)                              # [d]
    vid = mesh.vgrid.astype(np.int64) @ w                                     # fine-grid id / p per vertex
    ids = vid[mesh.cell_vertex] @ alpha.T                                     # [ncell, nd]
    return ids.astype(np.int32), m ** mesh.dim


def node_coordinates(mesh: Mesh, p: int) -> np.ndarray:
    """Physical coordinates ``[(p n+1)^dim, dim]`` of the P_p nodes (affine cells), for interpolation."""
    cmap, nnodes = cell_node_map(mesh, p)
    alpha = lagrange_nodes(mesh.dim, p).astype(np.float64) / p               # [nd, d+1]
    xv = mesh.coords[mesh.cell_vertex]                                        # [ncell, d+1, d]
    xn = np.einsum("km,cmx->ckx", alpha, xv)
    out = np.empty((nnodes, mesh.dim))
    out[cmap.ravel()] = xn.reshape(-1, mesh.dim)
    return out


def uniform_dat(size: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Nodal values uniform[lo, hi] from ``default_rng(seed)`` (float64)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=size)


def lognormal_dat(size: int, seed: int) -> np.ndarray:
    """Nodal values exp(z), z ~ N(0, 1), from ``default_rng(seed)`` (float64)."""
    return np.exp(np.random.default_rng(seed).standard_normal(size))


def batch_mesh_sizes(count: int, seed: int, lo: int = 8, hi: int = 256) -> tuple[np.ndarray, np.ndarray]:
    """Mesh sizes n = round(exp(U(ln lo, ln hi))) and degrees P1/P2 (Bernoulli 1/2) for many meshes."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    p = 1 + (rng.uniform(size=count) < 0.5).astype(np.int64)
    return n, p


def boundary_nodes(mesh: Mesh, p: int) -> np.ndarray:
    """uint8 mask over the P_p nodes: 1 where the node lies on the boundary of [0,1]^dim.

    Node ids enumerate the fine lattice (p n + 1)^dim with x fastest, so the test is exact
    integer arithmetic on the lattice index."""
    m = p * mesh.n + 1
    ids = np.arange(m ** mesh.dim, dtype=np.int64)
    on = np.zeros(ids.size, dtype=bool)
    for _ in range(mesh.dim):
        c = ids % m
        on |= (c == 0) | (c == m - 1)
        ids //= m
    return on.astype(np.uint8)


def manufactured_sine(mesh: Mesh, p: int, k: int, m: int) -> tuple[np.ndarray, np.ndarray]:
    """Nodal values of u = sin(k pi x) sin(m pi y) and of f = (k^2 + m^2) pi^2 u at the P_p nodes of
    a triangle mesh (-lap u = f in the unit square, u = 0 on its boundary)."""
    X = node_coordinates(mesh, p)
    u = np.sin(k * np.pi * X[:, 0]) * np.sin(m * np.pi * X[:, 1])
    return (k * k + m * m) * np.pi ** 2 * u, u


def serve_requests(count: int, seed: int, rate: float, lo: int = 16, hi: int = 512):
    """Poisson-process arrivals (exponential gaps, mean 1/rate seconds) of solve requests:
    (arrival_s, n log-uniform in [lo, hi], degree P1/P2 with probability 1/2, k, m uniform in 1..4)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count)) if rate > 0 else np.zeros(count)
    n = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    p = 1 + (rng.uniform(size=count) < 0.5).astype(np.int64)
    k = rng.integers(1, 5, size=count)
    mm = rng.integers(1, 5, size=count)
    return [(float(t[i]), int(n[i]), int(p[i]), int(k[i]), int(mm[i])) for i in range(count)]


def face_nodes(mesh: Mesh, p: int, axis: int, side: int) -> np.ndarray:
    """uint8 mask over the P_p nodes: 1 on the face x_axis = side (0 or 1) of the unit square/cube."""
    m = p * mesh.n + 1
    ids = np.arange(m ** mesh.dim, dtype=np.int64)
    c = (ids // m ** axis) % m
    return (c == (0 if side == 0 else m - 1)).astype(np.uint8)
