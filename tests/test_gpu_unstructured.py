"""Unstructured inputs on the GPU vs the CPU oracle (runs on the GB300 machine).

The mesh generators number nodes, vertices and cells lexicographically; real meshes do not.
These tests relabel all three at random (values must permute exactly with the relabelling and
match the oracle), build patterns from random maps with long and ragged rows (the hash path of
the row kernel), and check that rows beyond the documented limits are refused with an error
status rather than written.
"""
import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg
from tests import problems as PB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    return torch


def _relabel(pr, seed):
    """The same mesh with nodes, vertices and cells renumbered by random permutations."""
    rng = np.random.default_rng(seed)
    pn = rng.permutation(pr.nnodes).astype(np.int32)
    pv = rng.permutation(pr.mesh.nvert).astype(np.int32)
    pc = rng.permutation(pr.mesh.ncell)
    cmap = np.ascontiguousarray(pn[pr.cmap[pc]])
    cv = np.ascontiguousarray(pv[pr.mesh.cell_vertex[pc]])
    coords = np.empty_like(pr.mesh.coords)
    coords[pv] = pr.mesh.coords
    mesh = mg.Mesh(pr.mesh.dim, pr.mesh.n, coords, cv, pr.mesh.vgrid[np.argsort(pv)])
    return PB.Problem(pr.dim, pr.p, pr.n, mesh, cmap, pr.nnodes, None), pn


def _csr_dict(rp, ci, v):
    return {(r, int(c)): v[k] for r in range(len(rp) - 1) for k, c in zip(range(rp[r], rp[r + 1]), ci[rp[r]:rp[r + 1]])}


@pytest.mark.parametrize("dim,p,n", [(3, 2, 5), (2, 4, 7), (2, 1, 20)])
def test_relabelled_mesh(gpu, dim, p, n):
    from paper_1501_01809_gb300 import fe
    base = PB.make(dim, p, n, 0.2, seed=4)
    pr, pn = _relabel(base, seed=n)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    orp, oci = O.sparsity(pr.cmap, pr.cmap, pr.nnodes, pr.nnodes)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    nd = pr.cmap.shape[1]
    lut = g.fe.sparsity_lut(g.sparsity(), pr.mesh.ncell, nd, nd).cpu().numpy().reshape(-1, nd, nd).astype(np.int64)
    pos = rp[pr.cmap][:, :, None] + lut
    np.testing.assert_array_equal(ci[pos], np.broadcast_to(pr.cmap[:, None, :], pos.shape))
    got = g.assemble(fe.FORM_HELMHOLTZ, strategy=fe.STRATEGY_PUSH)
    want, scale = O.assemble_mat(dim, p, 3, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci)
    PB.assert_close_scaled(got, want, scale, 1e-12, "relabelled mesh")
    # the same operator as on the lexicographic numbering, entry for entry
    gb = PB.GpuProblem(base)
    brp, bci = gb.csr()
    bvals = gb.assemble(fe.FORM_HELMHOLTZ, strategy=fe.STRATEGY_PUSH)
    B = _csr_dict(brp, bci, bvals)
    Rl = _csr_dict(rp, ci, got)
    assert len(B) == len(Rl)
    for (r, c), v in B.items():
        assert abs(Rl[(int(pn[r]), int(pn[c]))] - v) <= 1e-12 * max(1.0, abs(v))


def _random_map(ncell, arity, nto, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(np.argsort(rng.random((ncell, nto)), axis=1)[:, :arity].astype(np.int32))


@pytest.mark.parametrize("ncell,ar,ac,nr,nc", [(2500, 6, 6, 700, 700), (2000, 10, 4, 800, 900), (500, 3, 12, 100, 2000)])
def test_random_maps_sparsity(gpu, ncell, ar, ac, nr, nc):
    """Random maps (no target repeated within a cell): rows of up to about 200 candidates, most of
    them distinct (the hash path of the row kernel), square and rectangular."""
    from paper_1501_01809_gb300 import fe
    torch = gpu
    rmap = _random_map(ncell, ar, nr, 1)
    cmap = _random_map(ncell, ac, nc, 2)
    ctx = fe.ctx_create(0)
    cells, rows, cols = fe.set_create(ctx, ncell), fe.set_create(ctx, nr), fe.set_create(ctx, nc)
    tr, tc = torch.from_numpy(rmap).cuda(), torch.from_numpy(cmap).cuda()
    R = fe.map_create(ctx, cells, rows, tr, validate=True)
    Cm = fe.map_create(ctx, cells, cols, tc, validate=True)
    sp = fe.sparsity_build(ctx, R, Cm)
    _, _, nnz, rp, ci = fe.sparsity_csr(sp)
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    orp, oci = O.sparsity(rmap, cmap, nr, nc)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    lut = fe.sparsity_lut(sp, ncell, ar, ac).cpu().numpy().reshape(-1, ar, ac).astype(np.int64)
    pos = rp[rmap][:, :, None] + lut
    np.testing.assert_array_equal(ci[pos], np.broadcast_to(cmap[:, None, :], pos.shape))


@pytest.mark.parametrize("ncell,ar,ac,nr,nc,nhub", [(3000, 3, 5, 3000, 400, 0), (2000, 4, 6, 1500, 1500, 12),
                                                    (1200, 2, 9, 900, 300, 6)])
def test_random_maps_small_rows_with_repeats(gpu, ncell, ar, ac, nr, nc, nhub):
    """Random maps whose rows mostly hold a few incidences (the row kernel sorts those four at a
    time, one per quarter-warp), targets repeated within a cell in both maps, and nhub rows that
    appear in 20 more cells each (those take the whole warp, beside small rows of their chunk of
    eight).  Pattern bitwise equal to the oracle's; every lookup-table entry names its column."""
    from paper_1501_01809_gb300 import fe
    torch = gpu
    rng = np.random.default_rng(ncell + ar)
    rmap = rng.integers(0, nr, (ncell, ar)).astype(np.int32)
    cmap = rng.integers(0, nc, (ncell, ac)).astype(np.int32)
    if nhub:
        hubs = 8 * rng.choice(nr // 8, nhub, replace=False) + rng.integers(0, 8, nhub)
        rmap[:20 * nhub, 0] = np.repeat(hubs, 20)
    assert (rmap[:, :1] == rmap[:, 1:]).any() and (cmap[:, :1] == cmap[:, 1:]).any()  # repeats occur
    ctx = fe.ctx_create(0)
    cells, rows, cols = fe.set_create(ctx, ncell), fe.set_create(ctx, nr), fe.set_create(ctx, nc)
    R = fe.map_create(ctx, cells, rows, torch.from_numpy(rmap).cuda(), validate=True)
    Cm = fe.map_create(ctx, cells, cols, torch.from_numpy(cmap).cuda(), validate=True)
    sp = fe.sparsity_build(ctx, R, Cm)
    _, _, nnz, rp, ci = fe.sparsity_csr(sp)
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    orp, oci = O.sparsity(rmap, cmap, nr, nc)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    lut = fe.sparsity_lut(sp, ncell, ar, ac).cpu().numpy().reshape(-1, ar, ac).astype(np.int64)
    pos = rp[rmap][:, :, None] + lut
    assert (lut < (rp[rmap + 1] - rp[rmap])[:, :, None]).all()
    np.testing.assert_array_equal(ci[pos], np.broadcast_to(cmap[:, None, :], pos.shape))
    # a rebuild from the same maps (in-place pass, counts checked) gives the same pattern and table
    fe.sparsity_rebuild(sp)
    _, _, _, rp2, ci2 = fe.sparsity_csr(sp)
    np.testing.assert_array_equal(rp2.cpu().numpy(), orp)
    np.testing.assert_array_equal(ci2.cpu().numpy(), oci)
    lut2 = fe.sparsity_lut(sp, ncell, ar, ac).cpu().numpy().reshape(-1, ar, ac).astype(np.int64)
    np.testing.assert_array_equal(lut2, lut)


def test_rows_beyond_the_limits_are_refused(gpu):
    from paper_1501_01809_gb300 import fe
    torch = gpu
    ctx = fe.ctx_create(0)
    # node 0 in 300 cells with 5 distinct other nodes each: a row of 1501 columns (> 256)
    ncell = 300
    m = np.zeros((ncell, 6), dtype=np.int32)
    m[:, 1:] = 1 + np.arange(ncell * 5, dtype=np.int32).reshape(ncell, 5)
    nodes = 1 + ncell * 5
    cells, ns = fe.set_create(ctx, ncell), fe.set_create(ctx, nodes)
    M = fe.map_create(ctx, cells, ns, torch.from_numpy(m).cuda(), validate=True)
    with pytest.raises(fe.FeError) as ei:
        fe.sparsity_build(ctx, M, M)
    assert ei.value.code == fe.FE_EUNSUPPORTED
    # node 0 in 800 cells: 4800 candidates (> 4096)
    ncell = 800
    m = np.zeros((ncell, 6), dtype=np.int32)
    m[:, 1:] = 1 + (np.arange(ncell * 5, dtype=np.int32).reshape(ncell, 5) % 200)
    cells, ns = fe.set_create(ctx, ncell), fe.set_create(ctx, 201)
    M = fe.map_create(ctx, cells, ns, torch.from_numpy(m).cuda(), validate=True)
    with pytest.raises(fe.FeError) as ei:
        fe.sparsity_build(ctx, M, M)
    assert ei.value.code == fe.FE_EUNSUPPORTED
