"""Stored element matrices (fe_elem_matrices + fe_action_stored) vs the CPU oracle.

The stored-matrix path must give what the matrix-free action gives: each stored upper triangle
matches the oracle's element matrix of that cell (per entry within 1e-12 of the cell's largest
entry), and the action from the stored matrices matches the oracle's action within the same
per-entry scaled bound as fe_action (1e-12 x the sum of |contributions|).  Sizes span several
128-thread blocks with ragged tails.
"""
import numpy as np
import pytest

import oracle as O
from tests import problems as PB

pytestmark = pytest.mark.gpu

CASES = [  # dim, p, n, jitter, form, precision (0 FP64, 1 FP32 pairs)
    (2, 1, 37, 0.2, 3, 0),
    (2, 2, 23, 0.2, 3, 1),
    (2, 2, 11, 0.2, 4, 1),
    (2, 4, 9, 0.2, 4, 0),
    (3, 1, 9, 0.2, 2, 1),
    (3, 2, 7, 0.2, 3, 0),
    (3, 2, 7, 0.2, 3, 1),
    (3, 2, 5, 0.2, 1, 1),
    (3, 3, 3, 0.2, 3, 0),
]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    return torch


def _stored(g, form, precision):
    fe, torch = g.fe, g.torch
    k = fe.kernel_create(g.ctx, form, g.pr.dim, g.pr.p, precision=precision)
    nup = k.nd * (k.nd + 1) // 2
    Ke = torch.full((nup, g.pr.mesh.ncell), np.nan, dtype=torch.float64, device="cuda")
    fe.elem_matrices(g.ctx, k, g.cells, Ke, g.coords, g.coord_map, g.coeffs(form))
    return k, Ke


def _upper(K):
    i, j = np.triu_indices(K.shape[0])
    return K[i, j]


@pytest.mark.parametrize("dim,p,n,jit,form,prec", CASES)
def test_stored_matrices_match_oracle(gpu, dim, p, n, jit, form, prec):
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    k, Ke = _stored(g, form, prec)
    g.fe.sync(g.ctx)
    got = Ke.cpu().numpy()
    cv = pr.mesh.cell_vertex
    for e in range(pr.mesh.ncell):
        kv = pr.kappa[cv[e]] if form == 4 else None
        want = _upper(O.element_matrix(dim, p, form, pr.mesh.coords[cv[e]], kv))
        tol = 1e-12 * np.max(np.abs(want))
        err = np.max(np.abs(got[:, e] - want))
        assert err <= tol, f"cell {e}: |K - K_oracle| = {err:.3e} > {tol:.3e}"


@pytest.mark.parametrize("dim,p,n,jit,form,prec", CASES)
def test_stored_action_matches_oracle(gpu, dim, p, n, jit, form, prec):
    torch = gpu
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    fe = g.fe
    k, Ke = _stored(g, form, prec)
    x = np.random.default_rng(2).uniform(-1, 1, pr.nnodes)
    tx = torch.from_numpy(x).cuda()
    ty = torch.full_like(tx, np.nan)
    X, Y = fe.dat_create(g.ctx, g.nodes, tx), fe.dat_create(g.ctx, g.nodes, ty)
    fe.action_stored(g.ctx, k, g.cells, Ke, X, Y, g.map, zero_first=True)
    fe.sync(g.ctx)
    want, scale = O.action(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x, kappa=pr.kappa)
    PB.assert_close_scaled(ty.cpu().numpy(), want, scale, 1e-12, "stored action")
    # INC: a second application without zeroing adds the same vector again
    fe.action_stored(g.ctx, k, g.cells, Ke, X, Y, g.map, zero_first=False)
    fe.sync(g.ctx)
    PB.assert_close_scaled(ty.cpu().numpy(), 2 * want, 2 * scale, 1e-12, "stored action, INC")
    # the stored matrices and x are READ: unchanged by the calls
    np.testing.assert_array_equal(tx.cpu().numpy(), x)


def test_stored_empty_mesh_and_refusals(gpu):
    torch = gpu
    pr = PB.make(2, 2, 5, 0.0, seed=3)
    g = PB.GpuProblem(pr)
    fe = g.fe
    # an empty iteration set stores nothing and leaves y zeroed
    cells0 = fe.set_create(g.ctx, 0)
    m0 = fe.map_create(g.ctx, cells0, g.nodes, torch.zeros((0, 6), dtype=torch.int32, device="cuda"))
    cm0 = fe.map_create(g.ctx, cells0, g.verts, torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    k = fe.kernel_create(g.ctx, fe.FORM_HELMHOLTZ, 2, 2)
    Ke0 = torch.zeros((21, 0), dtype=torch.float64, device="cuda")
    fe.elem_matrices(g.ctx, k, cells0, Ke0, g.coords, cm0)
    ty = torch.full((pr.nnodes,), 7.0, dtype=torch.float64, device="cuda")
    tx = torch.ones_like(ty)
    X, Y = fe.dat_create(g.ctx, g.nodes, tx), fe.dat_create(g.ctx, g.nodes, ty)
    fe.action_stored(g.ctx, k, cells0, Ke0, X, Y, m0, zero_first=True)
    fe.sync(g.ctx)
    assert float(ty.abs().max()) == 0.0
    Ke = torch.zeros((21, pr.mesh.ncell), dtype=torch.float64, device="cuda")
    # precisions without stored-matrix kernels (FP32 element tensors), and linear forms, are refused
    kp = fe.kernel_create(g.ctx, fe.FORM_HELMHOLTZ, 2, 2, precision=fe.PREC_FP32)
    with pytest.raises(fe.FeError) as ei:
        fe.elem_matrices(g.ctx, kp, g.cells, Ke, g.coords, g.coord_map)
    assert ei.value.code == fe.FE_EUNSUPPORTED
    with pytest.raises(fe.FeError) as ei:
        fe.action_stored(g.ctx, kp, g.cells, Ke, X, Y, g.map)
    assert ei.value.code == fe.FE_EUNSUPPORTED
    ks = fe.kernel_create(g.ctx, fe.FORM_SOURCE, 2, 2, coeff_degree=2)
    with pytest.raises(fe.FeError) as ei:
        fe.elem_matrices(g.ctx, ks, g.cells, torch.zeros((21, pr.mesh.ncell), dtype=torch.float64, device="cuda"),
                         g.coords, g.coord_map)
    assert ei.value.code == fe.FE_EUNSUPPORTED
    # x aliasing y is refused before any launch
    with pytest.raises(fe.FeError) as ei:
        fe.action_stored(g.ctx, k, g.cells, Ke, X, X, g.map)
    assert ei.value.code == fe.FE_EINVAL
    # a buffer of the wrong size is refused by the binding
    with pytest.raises(ValueError):
        fe.elem_matrices(g.ctx, k, g.cells, Ke[:, :-1].contiguous(), g.coords, g.coord_map)
