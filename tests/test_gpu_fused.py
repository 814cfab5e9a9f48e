"""The CSR assembly and the matrix-free action in one pass (fe_assemble_mat_action) against the
oracle: both outputs of every compiled bilinear form and element, per entry within 1e-12 of the
oracle's scale (the Mat's sum of |contributions|, the action's sum_e |K_e| |x_e|), in FP64 and in
double-float for P1/P2; INC semantics (zero_first = 0 adds a second pass onto the first); and in
check mode a lookup-table entry beyond its row flagged (FE_ERANGE at sync) with its write skipped,
y untouched by the skip."""
import numpy as np
import pytest

import oracle as O
from tests import problems as PB

pytestmark = pytest.mark.gpu

CASES = [(2, 1, 37, 0.2), (2, 2, 23, 0.2), (2, 3, 9, 0.2), (2, 4, 17, 0.2), (3, 1, 9, 0.2), (3, 2, 7, 0.2),
         (3, 3, 3, 0.2)]
KAPPA = [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    return torch


def _fused(g, form, x, precision=0, zero_first=True, A=None, ty=None):
    fe, torch = g.fe, g.torch
    k = fe.kernel_create(g.ctx, form, g.pr.dim, g.pr.p, precision=precision)
    A = A or fe.mat_create(g.ctx, g.sparsity())
    tx = torch.from_numpy(x).cuda()
    ty = ty if ty is not None else torch.full_like(tx, np.nan)
    X, Y = fe.dat_create(g.ctx, g.nodes, tx), fe.dat_create(g.ctx, g.nodes, ty)
    fe.assemble_mat_action(g.ctx, k, g.cells, A, X, Y, g.map, g.coords, g.coord_map, g.coeffs(form),
                           zero_first=zero_first)
    fe.sync(g.ctx)
    return fe.mat_values(A).cpu().numpy().copy(), ty.cpu().numpy().copy(), A, ty


def _check_against_oracle(pr, g, form, vals, y, x, rtol=1e-12):
    rp, ci = g.csr()
    want, scale = O.assemble_mat(pr.dim, pr.p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci,
                                 kappa=pr.kappa)
    PB.assert_close_scaled(vals, want, scale, rtol, f"Mat, form {form} P{pr.p} dim {pr.dim}")
    wy, sy = O.action(pr.dim, pr.p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x, kappa=pr.kappa)
    PB.assert_close_scaled(y, wy, sy, rtol, f"action, form {form} P{pr.p} dim {pr.dim}")


@pytest.mark.parametrize("dim,p,n,jit", CASES)
@pytest.mark.parametrize("form", [1, 2, 3, 4])
def test_fused_matches_oracle(gpu, dim, p, n, jit, form):
    if form == 4 and (dim, p) not in KAPPA:
        pytest.skip("kappa-diffusion built for P1/P2/P4 triangles and P1/P2 tets")
    pr = PB.make(dim, p, n, jit, seed=5, kappa_seed=4 if form == 4 else None)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(dim * 10 + p).uniform(-1, 1, pr.nnodes)
    vals, y, _, _ = _fused(g, form, x)
    _check_against_oracle(pr, g, form, vals, y, x)


@pytest.mark.parametrize("dim,p,n", [(2, 1, 37), (2, 2, 23), (3, 1, 9), (3, 2, 7)])
@pytest.mark.parametrize("form", [1, 3, 4])
def test_fused_double_float_matches_oracle(gpu, dim, p, n, form):
    if form == 4 and dim == 3:
        pytest.skip("kappa-diffusion in double-float on triangles only")
    pr = PB.make(dim, p, n, 0.2, seed=6, kappa_seed=5 if form == 4 else None)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(3).uniform(-1, 1, pr.nnodes)
    vals, y, _, _ = _fused(g, form, x, precision=1)
    _check_against_oracle(pr, g, form, vals, y, x)


def test_fused_inc_semantics(gpu):
    pr = PB.make(3, 2, 5, 0.2, seed=7)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(8).uniform(-1, 1, pr.nnodes)
    v1, y1, A, ty = _fused(g, 3, x)
    v2, y2, _, _ = _fused(g, 3, x, zero_first=False, A=A, ty=ty)
    assert np.abs(v2 - 2 * v1).max() <= 1e-14 * np.abs(v1).max()
    assert np.abs(y2 - 2 * y1).max() <= 1e-14 * np.abs(y1).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_fused_lookup_table_beyond_row_is_flagged(gpu, prec):
    """One byte of the library's lookup table is poked from the host: in check mode the fused
    kernel reports FE_ERANGE at sync and skips that write; no other Mat row changes, and y (whose
    reductions do not go through the table) is unchanged."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(3, 2, 4, 0.2, seed=6)
    g = PB.GpuProblem(pr, checks=True)
    x = np.random.default_rng(9).uniform(-1, 1, pr.nnodes)
    clean, yc, A, ty = _fused(g, 3, x, precision=prec)
    nd = pr.cmap.shape[1]
    lut = fe.sparsity_lut(g.sparsity(), pr.mesh.ncell, nd, nd)
    e, i, j = pr.mesh.ncell // 2, 1, nd - 2
    r = int(pr.cmap[e, i])
    rp, _ = g.csr()
    assert rp[r + 1] - rp[r] < 255
    lut[e * nd * nd + i * nd + j] = 255
    k = fe.kernel_create(g.ctx, 3, 3, 2, precision=prec)
    X, Y = fe.dat_create(g.ctx, g.nodes, g.torch.from_numpy(x).cuda()), fe.dat_create(g.ctx, g.nodes, ty)
    fe.assemble_mat_action(g.ctx, k, g.cells, A, X, Y, g.map, g.coords, g.coord_map, zero_first=True)
    with pytest.raises(fe.FeError) as ei:
        fe.sync(g.ctx)
    assert ei.value.code == fe.FE_ERANGE and "lookup-table entry" in str(ei.value)
    got = fe.mat_values(A).cpu().numpy()
    outside = np.ones(len(clean), dtype=bool)
    outside[rp[r]:rp[r + 1]] = False
    tol = 1e-13 * np.abs(clean).max()
    assert np.abs(got[outside] - clean[outside]).max() <= tol
    assert np.count_nonzero(np.abs(got[~outside] - clean[~outside]) > tol) <= 1
    assert np.abs(ty.cpu().numpy() - yc).max() <= 1e-13 * np.abs(yc).max()
