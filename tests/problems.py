"""Shared set-up for the GPU parity tests: a mesh with its maps and Dats on both sides.

Inputs come from the seeded generators only; the oracle and the CUDA path each receive the
same arrays and share nothing else.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from paper_1501_01809_gb300 import meshgen as mg

FORM_NAMES = {1: "mass", 2: "laplace", 3: "helmholtz", 4: "kappa"}


@dataclass
class Problem:
    dim: int
    p: int
    n: int
    mesh: mg.Mesh
    cmap: np.ndarray
    nnodes: int
    kappa: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def make(dim: int, p: int, n: int, jitter: float = 0.0, seed: int = 0, kappa_seed: int | None = None) -> Problem:
    mesh = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n, jitter, seed)
    cmap, nn = mg.cell_node_map(mesh, p)
    kap = mg.lognormal_dat(mesh.nvert, kappa_seed) if kappa_seed is not None else None
    return Problem(dim, p, n, mesh, cmap, nn, kap)


class GpuProblem:
    """The same problem as libfe objects (device tensors borrowed by the handles)."""

    def __init__(self, pr: Problem, ctx=None, checks=False):
        import torch
        from paper_1501_01809_gb300 import fe
        self.fe, self.torch, self.pr = fe, torch, pr
        dev = torch.device("cuda", 0)
        self.ctx = ctx or fe.ctx_create(0, checks=checks)
        self.cells = fe.set_create(self.ctx, pr.mesh.ncell)
        self.nodes = fe.set_create(self.ctx, pr.nnodes)
        self.verts = fe.set_create(self.ctx, pr.mesh.nvert)
        self.t_map = torch.from_numpy(np.ascontiguousarray(pr.cmap)).to(dev)
        self.t_cmap = torch.from_numpy(np.ascontiguousarray(pr.mesh.cell_vertex)).to(dev)
        self.t_coords = torch.from_numpy(np.ascontiguousarray(pr.mesh.coords)).to(dev)
        self.map = fe.map_create(self.ctx, self.cells, self.nodes, self.t_map)
        self.coord_map = fe.map_create(self.ctx, self.cells, self.verts, self.t_cmap)
        self.coords = fe.dat_create(self.ctx, self.verts, self.t_coords)
        self.kappa = None
        if pr.kappa is not None:
            self.t_kappa = torch.from_numpy(pr.kappa).to(dev)
            self.kappa = fe.dat_create(self.ctx, self.verts, self.t_kappa)
        self._sp = None

    def sparsity(self):
        if self._sp is None:
            self._sp = self.fe.sparsity_build(self.ctx, self.map, self.map)
        return self._sp

    def csr(self):
        nr, nc, nnz, rp, ci = self.fe.sparsity_csr(self.sparsity())
        return rp.cpu().numpy(), ci.cpu().numpy()

    def coeffs(self, form):
        if form == self.fe.FORM_KAPPA_DIFFUSION:
            return [(self.kappa, self.coord_map)]
        return []

    def assemble(self, form, precision=0, strategy=0):
        fe = self.fe
        k = fe.kernel_create(self.ctx, form, self.pr.dim, self.pr.p, precision=precision, strategy=strategy)
        A = fe.mat_create(self.ctx, self.sparsity())
        fe.assemble_mat(self.ctx, k, self.cells, A, self.coords, self.coord_map, self.coeffs(form), zero_first=True)
        fe.sync(self.ctx)
        return fe.mat_values(A).cpu().numpy()

    def action(self, form, x: np.ndarray, precision=0, strategy=0):
        fe, torch = self.fe, self.torch
        k = fe.kernel_create(self.ctx, form, self.pr.dim, self.pr.p, precision=precision, strategy=strategy)
        tx = torch.from_numpy(x).cuda()
        ty = torch.full_like(tx, np.nan)
        X, Y = fe.dat_create(self.ctx, self.nodes, tx), fe.dat_create(self.ctx, self.nodes, ty)
        fe.action(self.ctx, k, self.cells, X, Y, self.map, self.coords, self.coord_map, self.coeffs(form),
                  zero_first=True, sp=self.sparsity() if strategy == fe.STRATEGY_PULL else None)
        fe.sync(self.ctx)
        return ty.cpu().numpy()

    def fused(self, form, x: np.ndarray, precision=0):
        """fe_assemble_mat_action: the Mat values and y = A x of one pass (zero_first)."""
        fe, torch = self.fe, self.torch
        k = fe.kernel_create(self.ctx, form, self.pr.dim, self.pr.p, precision=precision)
        A = fe.mat_create(self.ctx, self.sparsity())
        tx = torch.from_numpy(x).cuda()
        ty = torch.full_like(tx, np.nan)
        X, Y = fe.dat_create(self.ctx, self.nodes, tx), fe.dat_create(self.ctx, self.nodes, ty)
        fe.assemble_mat_action(self.ctx, k, self.cells, A, X, Y, self.map, self.coords, self.coord_map,
                               self.coeffs(form), zero_first=True)
        fe.sync(self.ctx)
        return fe.mat_values(A).cpu().numpy(), ty.cpu().numpy()

    def rhs(self, f: np.ndarray, fmap: np.ndarray, pf: int, fset_size: int, precision=0, strategy=0):
        fe, torch = self.fe, self.torch
        k = fe.kernel_create(self.ctx, fe.FORM_SOURCE, self.pr.dim, self.pr.p, coeff_degree=pf,
                             precision=precision, strategy=strategy)
        fset = fe.set_create(self.ctx, fset_size)
        tf = torch.from_numpy(f).cuda()
        tfm = torch.from_numpy(np.ascontiguousarray(fmap)).cuda()
        F = fe.dat_create(self.ctx, fset, tf)
        Fm = fe.map_create(self.ctx, self.cells, fset, tfm)
        tb = torch.full((self.pr.nnodes,), np.nan, dtype=torch.float64, device="cuda")
        B = fe.dat_create(self.ctx, self.nodes, tb)
        fe.assemble_vec(self.ctx, k, self.cells, B, self.map, self.coords, self.coord_map, [(F, Fm)],
                        zero_first=True, sp=self.sparsity() if strategy == fe.STRATEGY_PULL else None)
        fe.sync(self.ctx)
        return tb.cpu().numpy()

    def functional(self, form, x: np.ndarray, precision=0, zero_first=True, g=None):
        """a(x, x) into a Global (fe_assemble_global with a bilinear kernel); returns (value, Global)."""
        fe, torch = self.fe, self.torch
        k = fe.kernel_create(self.ctx, form, self.pr.dim, self.pr.p, precision=precision)
        tx = torch.from_numpy(x).cuda()
        X = fe.dat_create(self.ctx, self.nodes, tx)
        g = g or fe.global_create(self.ctx)
        fe.assemble_global(self.ctx, k, self.cells, g, X, self.map, self.coords, self.coord_map, self.coeffs(form),
                           zero_first=zero_first)
        fe.sync(self.ctx)
        return float(fe.global_values(g)[0].item()), g

    def linear_functional(self, f: np.ndarray, fmap: np.ndarray, pf: int, fset_size: int, x: np.ndarray,
                          precision=0):
        """L(x) = integral of f x (fe_assemble_global with a linear kernel)."""
        fe, torch = self.fe, self.torch
        k = fe.kernel_create(self.ctx, fe.FORM_SOURCE, self.pr.dim, self.pr.p, coeff_degree=pf, precision=precision)
        fset = fe.set_create(self.ctx, fset_size)
        tf, tfm = torch.from_numpy(f).cuda(), torch.from_numpy(np.ascontiguousarray(fmap)).cuda()
        F, Fm = fe.dat_create(self.ctx, fset, tf), fe.map_create(self.ctx, self.cells, fset, tfm)
        tx = torch.from_numpy(x).cuda()
        X = fe.dat_create(self.ctx, self.nodes, tx)
        g = fe.global_create(self.ctx)
        fe.assemble_global(self.ctx, k, self.cells, g, X, self.map, self.coords, self.coord_map, [(F, Fm)])
        fe.sync(self.ctx)
        return float(fe.global_values(g)[0].item())

    def volume(self, op, g=None, zero_first=True):
        fe = self.fe
        g = g or fe.global_create(self.ctx)
        fe.reduce_cell_volume(self.ctx, self.cells, g, op, self.coords, self.coord_map, zero_first=zero_first)
        fe.sync(self.ctx)
        return float(fe.global_values(g)[0].item()), g


def assert_close_scaled(got, want, scale, rtol=1e-12, what=""):
    """Per-entry |got - want| <= rtol * scale (scale = sum of |contributions|) and relative Frobenius."""
    got, want, scale = np.asarray(got), np.asarray(want), np.asarray(scale)
    err = np.abs(got - want)
    bad = err > rtol * scale + 1e-300
    assert not np.any(bad), (f"{what}: {bad.sum()} entries beyond {rtol} x scale; worst ratio "
                             f"{np.max(err / np.maximum(scale, 1e-300)):.3e} at {int(np.argmax(err / np.maximum(scale, 1e-300)))}")
    nrm = np.linalg.norm(want)
    if nrm > 0:
        assert np.linalg.norm(got - want) <= rtol * nrm, what


class GpuBatch:
    """Several problems in one context, batched: bilinear form `forms[i]` plus f v dx with f in the
    same space (f = uniform_dat(nnodes, seed + i))."""

    def __init__(self, problems, forms, precisions, seed=11):
        import torch
        from paper_1501_01809_gb300 import fe
        self.fe, self.torch = fe, torch
        self.ctx = fe.ctx_create(0)
        self.gp = [GpuProblem(pr, ctx=self.ctx) for pr in problems]
        self.problems, self.forms, self.precisions = problems, forms, precisions
        self.f = [np.random.default_rng(seed + i).uniform(-1, 1, pr.nnodes) for i, pr in enumerate(problems)]
        items = []
        self._keep = []
        for g, pr, form, prec, f in zip(self.gp, problems, forms, precisions, self.f):
            kmat = fe.kernel_create(self.ctx, form, pr.dim, pr.p, precision=prec)
            kvec = fe.kernel_create(self.ctx, fe.FORM_SOURCE, pr.dim, pr.p, coeff_degree=pr.p, precision=prec)
            tf = torch.from_numpy(f).cuda()
            F = fe.dat_create(self.ctx, g.nodes, tf)
            self._keep += [kmat, kvec, tf, F]
            items.append(dict(kmat=kmat, kvec=kvec, cells=g.cells, sp=g.sparsity(), coords=g.coords,
                              coord_map=g.coord_map, f=(F, g.map)))
        self.batch = fe.batch_create(self.ctx, items)

    def results(self, i):
        v, r = self.fe.batch_values(self.batch, i)
        return v.cpu().numpy(), r.cpu().numpy()
