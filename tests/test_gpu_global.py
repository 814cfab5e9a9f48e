"""Globals on the GPU (Sec. 4.3; "Global arguments", Sec. 4.4) against the oracle.

* a(x, x) of every compiled bilinear form and element (FP64; double-float for P1/P2) within
  1e-12 of the oracle's scale (the sum of |x_i| (sum_e |K_e| |x_e|)_i), on meshes of several
  blocks of cells, and bitwise the same on a second call (a fixed order of reduction);
* the closed forms: a(x, x) = 4/3 for the Helmholtz form and u = x, L(u) = 1/2 for f = 1;
* L(x) = integral of f x against the oracle;
* SUM access adds to what the Global holds (zero_first = 0): exactly the FP64 sum of the two;
* cell volumes: SUM = 1 (jittered unit square and cube), MIN and MAX equal to the oracle's per-cell
  volumes, MIN keeps the smaller of what it held and the new minimum; with no cells the
  reductions give 0, +inf and -inf; in check mode a vertex index past the coordinates is flagged
  (FE_ERANGE at sync) and its cell skipped, never read.
"""
import numpy as np
import pytest

import oracle as O
from tests import problems as PB

pytestmark = pytest.mark.gpu

ELEMENTS = [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)]
KAPPA = [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    return torch


def _size(dim, p):
    # more than one block of 2048 cells, with a ragged last block
    return {(2, 1): 41, (2, 2): 37, (2, 3): 33, (2, 4): 33, (3, 1): 9, (3, 2): 8, (3, 3): 7}[(dim, p)]


@pytest.mark.parametrize("dim,p", ELEMENTS)
@pytest.mark.parametrize("form", [1, 2, 3])
def test_energy_matches_oracle(gpu, dim, p, form):
    pr = PB.make(dim, p, _size(dim, p), 0.2, seed=dim * 10 + p)
    assert pr.mesh.ncell > 2048 and pr.mesh.ncell % 2048
    x = np.random.default_rng(form).uniform(-1, 1, pr.nnodes)
    g = PB.GpuProblem(pr)
    got, _ = g.functional(form, x)
    want, scale = O.functional(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x)
    assert abs(got - want) <= 1e-12 * scale, (got, want, scale)
    again, _ = g.functional(form, x)
    assert again == got  # the same bits: the reduction order is fixed


@pytest.mark.parametrize("dim,p", KAPPA)
def test_kappa_energy_matches_oracle(gpu, dim, p):
    pr = PB.make(dim, p, _size(dim, p) // 2 + 2, 0.2, seed=5, kappa_seed=6)
    x = np.random.default_rng(9).uniform(-1, 1, pr.nnodes)
    got, _ = PB.GpuProblem(pr).functional(4, x)
    want, scale = O.functional(dim, p, 4, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x, kappa=pr.kappa)
    assert abs(got - want) <= 1e-12 * scale, (got, want, scale)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_energy_double_float_matches_oracle(gpu, dim, p):
    pr = PB.make(dim, p, _size(dim, p), 0.2, seed=3)
    x = np.random.default_rng(4).uniform(-1, 1, pr.nnodes)
    got, _ = PB.GpuProblem(pr).functional(3, x, precision=1)
    want, scale = O.functional(dim, p, 3, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x)
    assert abs(got - want) <= 1e-12 * scale, (got, want, scale)


@pytest.mark.parametrize("dim,p", ELEMENTS)
def test_closed_forms(gpu, dim, p):
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(dim, p, 6 if dim == 2 else 3, 0.2, seed=1)
    u = mg.node_coordinates(pr.mesh, p)[:, 0].copy()
    g = PB.GpuProblem(pr)
    got, _ = g.functional(3, u)
    _, scale = O.functional(dim, p, 3, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, u)
    assert abs(got - 4 / 3) <= 1e-14 * scale, got
    if p <= 2:
        one = np.ones(pr.mesh.nvert)
        got = g.linear_functional(one, pr.mesh.cell_vertex, 1, pr.mesh.nvert, u)
        assert abs(got - 0.5) <= 1e-14, got


@pytest.mark.parametrize("dim,p,pf", [(2, 1, 1), (2, 2, 2), (2, 2, 1), (2, 4, 1), (3, 1, 1), (3, 2, 2), (3, 2, 1)])
def test_linear_functional_matches_oracle(gpu, dim, p, pf):
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(dim, p, _size(dim, p), 0.2, seed=8)
    fmap, nf = mg.cell_node_map(pr.mesh, pf)
    f = np.random.default_rng(10).uniform(-1, 1, nf)
    x = np.random.default_rng(11).uniform(-1, 1, pr.nnodes)
    got = PB.GpuProblem(pr).linear_functional(f, fmap, pf, nf, x)
    want, scale = O.linear_functional(dim, p, pf, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, f, fmap, x)
    assert abs(got - want) <= 1e-12 * scale, (got, want, scale)


def test_sum_access_adds(gpu):
    pr = PB.make(2, 2, 20, 0.2, seed=2)
    x = np.random.default_rng(12).uniform(-1, 1, pr.nnodes)
    g = PB.GpuProblem(pr)
    a, _ = g.functional(1, x)
    b, _ = g.functional(2, x)
    first, G = g.functional(1, x)
    both, _ = g.functional(2, x, zero_first=False, g=G)
    assert first == a and both == a + b


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_volume_reductions(gpu, dim):
    from paper_1501_01809_gb300 import fe
    pr = PB.make(dim, 1, 40 if dim == 2 else 10, 0.2, seed=4)
    g = PB.GpuProblem(pr)
    vol = O.cell_volumes(dim, pr.mesh.coords, pr.mesh.cell_vertex)
    total, _ = g.volume(fe.REDUCE_SUM)
    assert abs(total - 1.0) <= 1e-16 * pr.mesh.ncell, total
    lo, G = g.volume(fe.REDUCE_MIN)
    hi, _ = g.volume(fe.REDUCE_MAX)
    assert abs(lo - vol.min()) <= 1e-14 * vol.min() and abs(hi - vol.max()) <= 1e-14 * vol.max()
    # MIN access keeps the smaller value: a Global holding less than every cell stays where it is
    fe.global_values(G).fill_(lo / 2)
    gpu.cuda.synchronize()  # the fill (torch's stream) before the library's launch
    kept, _ = g.volume(fe.REDUCE_MIN, g=G, zero_first=False)
    assert kept == lo / 2
    fe.global_values(G).fill_(1.0)
    gpu.cuda.synchronize()
    now, _ = g.volume(fe.REDUCE_MIN, g=G, zero_first=False)
    assert now == lo


def test_empty_reductions(gpu):
    from paper_1501_01809_gb300 import fe
    torch = gpu
    ctx = fe.ctx_create(0)
    cells, verts = fe.set_create(ctx, 0), fe.set_create(ctx, 3)
    cm = fe.map_create(ctx, cells, verts, torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    xy = fe.dat_create(ctx, verts, torch.zeros((3, 2), dtype=torch.float64, device="cuda"))
    g = fe.global_create(ctx)
    out = []
    for op in (fe.REDUCE_SUM, fe.REDUCE_MIN, fe.REDUCE_MAX):
        fe.reduce_cell_volume(ctx, cells, g, op, xy, cm)
        fe.sync(ctx)
        out.append(float(fe.global_values(g)[0].item()))
    assert out == [0.0, np.inf, -np.inf]
    nodes = fe.set_create(ctx, 3)
    m = fe.map_create(ctx, cells, nodes, torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    X = fe.dat_create(ctx, nodes, torch.ones(3, dtype=torch.float64, device="cuda"))
    k = fe.kernel_create(ctx, fe.FORM_HELMHOLTZ, 2, 1)
    fe.global_values(g).fill_(7.0)
    torch.cuda.synchronize()
    fe.assemble_global(ctx, k, cells, g, X, m, xy, cm)
    fe.sync(ctx)
    assert float(fe.global_values(g)[0].item()) == 0.0


def test_bad_vertex_index_is_flagged_in_check_mode(gpu):
    from paper_1501_01809_gb300 import fe
    torch = gpu
    pr = PB.make(2, 1, 6, 0.0)
    ctx = fe.ctx_create(0, checks=True)
    cv = pr.mesh.cell_vertex.copy()
    cv[7, 2] = pr.mesh.nvert + 5  # past the coordinates: the check skips the cell, never reads it
    cells, verts = fe.set_create(ctx, pr.mesh.ncell), fe.set_create(ctx, pr.mesh.nvert)
    tcv = torch.from_numpy(cv).cuda()
    cm = fe.map_create(ctx, cells, verts, tcv)
    xy = fe.dat_create(ctx, verts, torch.from_numpy(pr.mesh.coords).cuda())
    g = fe.global_create(ctx)
    fe.reduce_cell_volume(ctx, cells, g, fe.REDUCE_SUM, xy, cm)
    with pytest.raises(fe.FeError) as ei:
        fe.sync(ctx)
    assert ei.value.code == fe.FE_ERANGE
    h = 1 / 6
    assert abs(float(fe.global_values(g)[0].item()) - (1 - h * h / 2)) <= 1e-15  # all cells but the flagged one
