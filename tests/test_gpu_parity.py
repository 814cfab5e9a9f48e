"""CUDA path vs the CPU oracle on the same seeded inputs (runs on the GB300 machine).

Sparsity: bitwise identical CSR.  Lookup table: exhaustive check that every (e, i, j) points at
column map(e)[j] of row map(e)[i].  Values: per entry |a - a_ref| <= 1e-12 * S_ij with S_ij the
sum of |element contributions| (the oracle accumulates S), and relative Frobenius <= 1e-12.
Sizes span several CTAs and leave ragged tails (cell counts not multiples of the block size).
"""
import numpy as np
import pytest

import oracle as O
from tests import problems as PB

pytestmark = pytest.mark.gpu

CASES = [  # dim, p, n, jitter
    (2, 1, 64, 0.0),    # the P1 UnitSquareMesh 64x64 workload (8192 cells)
    (2, 1, 37, 0.2),
    (2, 2, 23, 0.2),
    (2, 3, 9, 0.2),
    (2, 4, 17, 0.2),
    (3, 1, 9, 0.2),
    (3, 2, 7, 0.2),
    (3, 3, 3, 0.2),
]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("dim,p,n,jit", CASES)
def test_sparsity_bitwise_and_lut(gpu, dim, p, n, jit):
    pr = PB.make(dim, p, n, jit, seed=3)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    orp, oci = O.sparsity(pr.cmap, pr.cmap, pr.nnodes, pr.nnodes)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    nd = pr.cmap.shape[1]
    lut = g.fe.sparsity_lut(g.sparsity(), pr.mesh.ncell, nd, nd).cpu().numpy().reshape(-1, nd, nd).astype(np.int64)
    pos = rp[pr.cmap][:, :, None] + lut
    np.testing.assert_array_equal(ci[pos], np.broadcast_to(pr.cmap[:, None, :], pos.shape))


@pytest.mark.parametrize("dim,p,n,jit", CASES)
@pytest.mark.parametrize("form", [1, 2, 3, 4])
def test_assemble_mat_matches_oracle(gpu, dim, p, n, jit, form):
    """FP64 push (FP64 atomics through the lookup table)."""
    from paper_1501_01809_gb300 import fe
    if form == 4 and (dim, p) not in [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)]:
        pytest.skip("kappa-diffusion built for P1/P2/P4 triangles and P1/P2 tets")
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    got = g.assemble(form, strategy=fe.STRATEGY_PUSH)
    want, scale = O.assemble_mat(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci, kappa=pr.kappa)
    PB.assert_close_scaled(got, want, scale, 1e-12, f"form {form} P{p} dim {dim}")


@pytest.mark.parametrize("dim,p,n,jit", CASES[:1] + CASES[2:3] + CASES[6:7])
@pytest.mark.parametrize("form", [3, 4])
def test_action_matches_oracle(gpu, dim, p, n, jit, form):
    if form == 4 and (dim, p) not in [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)]:
        pytest.skip("kappa-diffusion built for P1/P2/P4 triangles and P1/P2 tets")
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(2).uniform(-1, 1, pr.nnodes)
    got = g.action(form, x)
    want, scale = O.action(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x, kappa=pr.kappa)
    PB.assert_close_scaled(got, want, scale, 1e-12, "action")


@pytest.mark.parametrize("dim,p,pf,n", [(2, 1, 1, 64), (2, 2, 2, 11), (2, 2, 1, 11), (2, 4, 1, 6), (3, 1, 1, 5),
                                         (3, 2, 2, 4), (3, 2, 1, 4)])
def test_assemble_vec_matches_oracle(gpu, dim, p, pf, n):
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(dim, p, n, 0.2 if n > 6 else 0.0, seed=4)
    g = PB.GpuProblem(pr)
    fmap, nf = mg.cell_node_map(pr.mesh, pf)
    f = mg.uniform_dat(nf, 1)
    got = g.rhs(f, fmap, pf, nf)
    want, scale = O.assemble_vec(dim, p, pf, pr.cmap, pr.nnodes, pr.mesh.coords, pr.mesh.cell_vertex, f, fmap)
    PB.assert_close_scaled(got, want, scale, 1e-12, "rhs")


def test_rebuild_is_bitwise_stable(gpu):
    pr = PB.make(3, 2, 5, 0.2, seed=0)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    lut0 = g.fe.sparsity_lut(g.sparsity(), pr.mesh.ncell, 10, 10).cpu().numpy().copy()
    for _ in range(2):
        g.fe.sparsity_rebuild(g.sparsity())
        g.fe.sync(g.ctx)
        rp2, ci2 = g.csr()
        np.testing.assert_array_equal(rp, rp2)
        np.testing.assert_array_equal(ci, ci2)
        np.testing.assert_array_equal(lut0, g.fe.sparsity_lut(g.sparsity(), pr.mesh.ncell, 10, 10).cpu().numpy())


def _check_pattern(g, cmap, nnodes):
    """CSR bitwise equal to the oracle's for cmap, and every lookup-table entry points at its column."""
    rp, ci = g.csr()
    orp, oci = O.sparsity(cmap, cmap, nnodes, nnodes)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    nd = cmap.shape[1]
    lut = g.fe.sparsity_lut(g.sparsity(), cmap.shape[0], nd, nd).cpu().numpy().reshape(-1, nd, nd).astype(np.int64)
    pos = orp[cmap][:, :, None] + lut
    np.testing.assert_array_equal(oci[pos], np.broadcast_to(cmap[:, None, :], pos.shape))


def _rewrite_map(g, cmap):
    g.t_map.copy_(g.torch.from_numpy(np.ascontiguousarray(cmap)))


@pytest.mark.parametrize("dim,p,n", [(3, 2, 5), (2, 2, 9)])
def test_map_values_not_8_byte_aligned(gpu, dim, p, n):
    """Map values that start 4 bytes past an 8-byte boundary (a view one int32 into a larger tensor):
    the row pass then loads candidates one at a time instead of in 8-byte pairs (even ndc).  The
    pattern and every lookup-table entry still match the oracle, after the build and a rebuild."""
    pr = PB.make(dim, p, n, 0.2, seed=3)
    g = PB.GpuProblem(pr)
    torch = g.torch
    flat = torch.empty(pr.cmap.size + 1, dtype=torch.int32, device="cuda")
    view = flat[1:].view(pr.cmap.shape)
    view.copy_(torch.from_numpy(np.ascontiguousarray(pr.cmap)))
    torch.cuda.synchronize()
    assert view.data_ptr() % 8 == 4 and pr.cmap.shape[1] % 2 == 0
    g.t_map, g.map = view, g.fe.map_create(g.ctx, g.cells, g.nodes, view)
    _check_pattern(g, pr.cmap, pr.nnodes)
    g.fe.sparsity_rebuild(g.sparsity())
    g.fe.sync(g.ctx)
    _check_pattern(g, pr.cmap, pr.nnodes)


def test_rebuild_same_row_lengths_in_place(gpu):
    """Local node order permuted within each cell: the pattern is unchanged (rows keep their
    lengths, the in-place pass writes colidx directly) while the lookup table changes."""
    pr = PB.make(3, 2, 5, 0.2, seed=0)
    g = PB.GpuProblem(pr)
    g.sparsity()
    rng = np.random.default_rng(11)
    perm = np.argsort(rng.random(pr.cmap.shape), axis=1)
    m2 = np.take_along_axis(pr.cmap, perm, axis=1)
    _rewrite_map(g, m2)
    g.fe.sparsity_rebuild(g.sparsity())
    g.fe.sync(g.ctx)
    _check_pattern(g, m2, pr.nnodes)


def test_rebuild_changed_row_lengths(gpu):
    """Nodes relabelled: the same nnz, but rows change length, so the full row pass, the scan and
    the compaction must run after the in-place pass."""
    pr = PB.make(3, 2, 5, 0.2, seed=0)
    g = PB.GpuProblem(pr)
    g.sparsity()
    relabel = np.random.default_rng(12).permutation(pr.nnodes).astype(np.int32)
    m2 = relabel[pr.cmap]
    rp0, _ = g.csr()
    orp2, _ = O.sparsity(m2, m2, pr.nnodes, pr.nnodes)
    assert orp2[-1] == rp0[-1] and np.any(np.diff(orp2) != np.diff(rp0))
    _rewrite_map(g, m2)
    g.fe.sparsity_rebuild(g.sparsity())
    g.fe.sync(g.ctx)
    _check_pattern(g, m2, pr.nnodes)
    # and back: rebuilding with the original map restores the original pattern
    _rewrite_map(g, pr.cmap)
    g.fe.sparsity_rebuild(g.sparsity())
    g.fe.sync(g.ctx)
    _check_pattern(g, pr.cmap, pr.nnodes)


def _flags(g):
    g.fe.sync(g.ctx)
    return g.fe.sparsity_changed(g.sparsity()).cpu().tolist()


@pytest.mark.parametrize("dim,p,n", [(3, 2, 5), (2, 1, 9), (3, 3, 3)])
def test_rebuild_reports_whether_the_pattern_changed(gpu, dim, p, n):
    """fe_sparsity_changed after each rebuild with column tracking on: [0, 0] after the build, for
    the same map, and for a permuted local node order (the same pattern, a new lookup table);
    [0, 1] when two nodes whose rows have the same length swap labels (every row keeps its length,
    some columns change), and again when they swap back; flags[0] set when relabelled nodes change
    row lengths.  With tracking off, flags[1] is set by every rebuild.  The pattern matches the
    oracle's every time.  P2 tetrahedra have whole-warp and quarter-warp rows, P1 triangles only
    quarter-warp rows, P3 tetrahedra hashed vertex rows (480 candidates)."""
    pr = PB.make(dim, p, n, 0.2, seed=0)
    g = PB.GpuProblem(pr)
    g.fe.sparsity_track_columns(g.sparsity(), True)
    assert _flags(g) == [0, 0]
    g.fe.sparsity_rebuild(g.sparsity())
    assert _flags(g) == [0, 0]
    perm = np.argsort(np.random.default_rng(11).random(pr.cmap.shape), axis=1)
    m_local = np.take_along_axis(pr.cmap, perm, axis=1)
    _rewrite_map(g, m_local)
    g.fe.sparsity_rebuild(g.sparsity())
    assert _flags(g) == [0, 0]
    _check_pattern(g, m_local, pr.nnodes)
    rp, ci = g.csr()
    lens = np.diff(rp)
    a = int(np.argmax(lens))  # a vertex node; b: the farthest node with a row of the same length
    b = int(np.nonzero(lens == lens[a])[0][-1])
    assert a != b
    relabel = np.arange(pr.nnodes, dtype=np.int32)
    relabel[a], relabel[b] = b, a
    m_swap = relabel[pr.cmap]
    orp, oci = O.sparsity(m_swap, m_swap, pr.nnodes, pr.nnodes)
    assert np.array_equal(orp, rp) and not np.array_equal(oci, ci)
    _rewrite_map(g, m_swap)
    g.fe.sparsity_rebuild(g.sparsity())
    assert _flags(g) == [0, 1]
    _check_pattern(g, m_swap, pr.nnodes)
    _rewrite_map(g, pr.cmap)
    g.fe.sparsity_rebuild(g.sparsity())
    assert _flags(g) == [0, 1]
    _check_pattern(g, pr.cmap, pr.nnodes)
    g.fe.sparsity_track_columns(g.sparsity(), False)
    g.fe.sparsity_rebuild(g.sparsity())
    f = _flags(g)
    assert f[0] == 0 and f[1] != 0
    _check_pattern(g, pr.cmap, pr.nnodes)
    g.fe.sparsity_track_columns(g.sparsity(), True)
    m_rel = np.random.default_rng(12).permutation(pr.nnodes).astype(np.int32)[pr.cmap]
    _rewrite_map(g, m_rel)
    g.fe.sparsity_rebuild(g.sparsity())
    assert _flags(g)[0] == 1
    _check_pattern(g, m_rel, pr.nnodes)


def test_rebuild_changed_nnz_is_reported(gpu):
    """A map whose pattern has another nnz is reported at the next sync, every time it is rebuilt
    (also when the previous failed rebuild left rowptr at that map's lengths); rebuilding with the
    original map then gives the original pattern."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(3, 2, 5, 0.2, seed=0)
    g = PB.GpuProblem(pr)
    g.sparsity()
    counts = np.bincount(pr.cmap.ravel(), minlength=pr.nnodes)
    # cell 0 takes the nodes of a cell whose nodes all have fewer incidences than the longest list,
    # so the row kernel's capacities still hold
    donor = next(e for e in range(1, pr.cmap.shape[0])
                 if counts[pr.cmap[e]].max() < counts.max() and not np.intersect1d(pr.cmap[e], pr.cmap[0]).size)
    m2 = pr.cmap.copy()
    m2[0] = pr.cmap[donor]
    orp2, _ = O.sparsity(m2, m2, pr.nnodes, pr.nnodes)
    rp0, _ = g.csr()
    assert orp2[-1] != rp0[-1]
    _rewrite_map(g, m2)
    for _ in range(2):
        g.fe.sparsity_rebuild(g.sparsity())
        with pytest.raises(fe.FeError) as ei:
            g.fe.sync(g.ctx)
        assert ei.value.code == fe.FE_EINVAL
    _rewrite_map(g, pr.cmap)
    g.fe.sparsity_rebuild(g.sparsity())
    g.fe.sync(g.ctx)
    _check_pattern(g, pr.cmap, pr.nnodes)


def test_rectangular_sparsity(gpu):
    """Rows from P2 nodes, columns from P1 nodes (Sec. 4.4.3: two different maps)."""
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(2, 2, 6, 0.0)
    g = PB.GpuProblem(pr)
    c1, n1 = mg.cell_node_map(pr.mesh, 1)
    s1 = g.fe.set_create(g.ctx, n1)
    t1 = g.torch.from_numpy(c1).cuda()
    m1 = g.fe.map_create(g.ctx, g.cells, s1, t1)
    sp = g.fe.sparsity_build(g.ctx, g.map, m1)
    nr, nc, nnz, rp, ci = g.fe.sparsity_csr(sp)
    orp, oci = O.sparsity(pr.cmap, c1, pr.nnodes, n1)
    assert (nr, nc) == (pr.nnodes, n1)
    np.testing.assert_array_equal(rp.cpu().numpy(), orp)
    np.testing.assert_array_equal(ci.cpu().numpy(), oci)
    lut = g.fe.sparsity_lut(sp, pr.mesh.ncell, 6, 3).cpu().numpy().reshape(-1, 6, 3).astype(np.int64)
    pos = orp[pr.cmap][:, :, None] + lut
    np.testing.assert_array_equal(oci[pos], np.broadcast_to(c1[:, None, :], pos.shape))


def test_single_cell_and_empty_mesh(gpu):
    from paper_1501_01809_gb300 import fe
    pr = PB.make(2, 2, 1, 0.0)
    pr.mesh.cell_vertex = pr.mesh.cell_vertex[:1].copy()
    pr.cmap = pr.cmap[:1].copy()
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    got = g.assemble(fe.FORM_HELMHOLTZ)
    want, scale = O.assemble_mat(2, 2, 3, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci)
    PB.assert_close_scaled(got, want, scale, 1e-12, "one cell")
    # an empty iteration set assembles nothing and builds an empty pattern over the nodes
    ctx = g.ctx
    cells0 = fe.set_create(ctx, 0)
    import torch
    m0 = fe.map_create(ctx, cells0, g.nodes, torch.zeros((0, 6), dtype=torch.int32, device="cuda"))
    sp0 = fe.sparsity_build(ctx, m0, m0)
    nr, nc, nnz, rp0, ci0 = fe.sparsity_csr(sp0)
    assert nnz == 0 and int(rp0[-1]) == 0 and nr == pr.nnodes


# ------------------------------------------------------------------ double-float (FP32 pair) element tensors
DD_CASES = [(2, 1, 64, 0.0), (2, 1, 37, 0.2), (2, 2, 23, 0.2), (3, 1, 9, 0.2), (3, 2, 7, 0.2)]


@pytest.mark.parametrize("dim,p,n,jit", DD_CASES)
@pytest.mark.parametrize("form", [1, 2, 3, 4])
def test_assemble_mat_f32x2_matches_oracle(gpu, dim, p, n, jit, form):
    """FP32-pair element tensors, FP64 global accumulation: same 1e-12 per-entry bound."""
    from paper_1501_01809_gb300 import fe
    if form == 4 and dim == 3:
        pytest.skip("kappa-diffusion on tetrahedra is compiled in FP64 only")
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    got = g.assemble(form, precision=fe.PREC_F32X2, strategy=fe.STRATEGY_PUSH)
    want, scale = O.assemble_mat(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci, kappa=pr.kappa)
    PB.assert_close_scaled(got, want, scale, 1e-12, f"f32x2 form {form} P{p} dim {dim}")


@pytest.mark.parametrize("dim,p,n,jit", DD_CASES)
@pytest.mark.parametrize("form", [3, 4])
def test_action_f32x2_matches_oracle(gpu, dim, p, n, jit, form):
    from paper_1501_01809_gb300 import fe
    if form == 4 and dim == 3:
        pytest.skip("kappa-diffusion on tetrahedra is compiled in FP64 only")
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(2).uniform(-1, 1, pr.nnodes)
    got = g.action(form, x, precision=fe.PREC_F32X2)
    want, scale = O.action(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x, kappa=pr.kappa)
    PB.assert_close_scaled(got, want, scale, 1e-12, "f32x2 action")


@pytest.mark.parametrize("dim,p,pf,n", [(2, 1, 1, 64), (2, 2, 2, 11), (3, 2, 2, 4), (3, 2, 1, 4)])
def test_assemble_vec_f32x2_matches_oracle(gpu, dim, p, pf, n):
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(dim, p, n, 0.2 if n > 6 else 0.0, seed=4)
    g = PB.GpuProblem(pr)
    fmap, nf = mg.cell_node_map(pr.mesh, pf)
    f = mg.uniform_dat(nf, 1)
    got = g.rhs(f, fmap, pf, nf, precision=fe.PREC_F32X2)
    want, scale = O.assemble_vec(dim, p, pf, pr.cmap, pr.nnodes, pr.mesh.coords, pr.mesh.cell_vertex, f, fmap)
    PB.assert_close_scaled(got, want, scale, 1e-12, "f32x2 rhs")


def test_f32x2_extreme_scales(gpu):
    """Tiny and huge cell sizes (coordinates scaled by 2^-30 and 2^20): relative accuracy holds."""
    from paper_1501_01809_gb300 import fe
    for scale_x in [2.0 ** -30, 3.0e-7, 2.0 ** 20]:
        pr = PB.make(3, 2, 3, 0.2, seed=3)
        pr.mesh.coords = pr.mesh.coords * scale_x
        g = PB.GpuProblem(pr)
        rp, ci = g.csr()
        got = g.assemble(3, precision=fe.PREC_F32X2)
        want, scale = O.assemble_mat(3, 2, 3, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci)
        PB.assert_close_scaled(got, want, scale, 1e-12, f"f32x2 coordinates x {scale_x}")


# ------------------------------------------------------------------ pull strategy (row owners, no atomics)
PULL_CASES = [(2, 1, 64, 0.0), (2, 2, 23, 0.2), (2, 4, 9, 0.2), (3, 1, 9, 0.2), (3, 2, 7, 0.2), (3, 3, 3, 0.2)]


def _dd_ok(dim, p, form):
    return p <= 2 and not (form == 4 and dim == 3)


@pytest.mark.parametrize("dim,p,n,jit", PULL_CASES)
@pytest.mark.parametrize("form", [1, 3, 4])
@pytest.mark.parametrize("prec", [0, 1])
def test_pull_mat_matches_oracle(gpu, dim, p, n, jit, form, prec):
    from paper_1501_01809_gb300 import fe
    if form == 4 and (dim, p) not in [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)]:
        pytest.skip("kappa-diffusion built for P1/P2/P4 triangles and P1/P2 tets")
    if prec == 1 and not _dd_ok(dim, p, form):
        pytest.skip("double-float kernels built for P1/P2 (kappa on triangles)")
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    got = g.assemble(form, precision=prec, strategy=fe.STRATEGY_PULL)
    want, scale = O.assemble_mat(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci, kappa=pr.kappa)
    PB.assert_close_scaled(got, want, scale, 1e-12, f"pull form {form} P{p} dim {dim} prec {prec}")


@pytest.mark.parametrize("dim,p,n,jit", [(2, 2, 23, 0.2), (3, 2, 7, 0.2), (3, 1, 9, 0.2)])
@pytest.mark.parametrize("prec", [0, 1])
def test_pull_action_and_rhs_match_oracle(gpu, dim, p, n, jit, prec):
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(dim, p, n, jit, seed=3)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(2).uniform(-1, 1, pr.nnodes)
    got = g.action(3, x, precision=prec, strategy=fe.STRATEGY_PULL)
    want, scale = O.action(dim, p, 3, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x)
    PB.assert_close_scaled(got, want, scale, 1e-12, "pull action")
    fmap, nf = mg.cell_node_map(pr.mesh, p)
    f = mg.uniform_dat(nf, 1)
    got = g.rhs(f, fmap, p, nf, precision=prec, strategy=fe.STRATEGY_PULL)
    want, scale = O.assemble_vec(dim, p, p, pr.cmap, pr.nnodes, pr.mesh.coords, pr.mesh.cell_vertex, f, fmap)
    PB.assert_close_scaled(got, want, scale, 1e-12, "pull rhs")


@pytest.mark.parametrize("dim,n", [(2, 37), (3, 9)])
@pytest.mark.parametrize("prec", [0, 1])
def test_pull_p1_laplace_action(gpu, dim, n, prec):
    """The P1 Laplace element stage (formed through grad(u), without the element matrix) against the
    oracle per entry within 1e-12 of its scale; and for u = x, the assembled action vanishes at
    every interior node (the integral of d(phi_i)/dx over the support of phi_i is zero)."""
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(dim, 1, n, 0.2, seed=4)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(5).uniform(-1, 1, pr.nnodes)
    got = g.action(fe.FORM_LAPLACE, x, precision=prec, strategy=fe.STRATEGY_PULL)
    want, scale = O.action(dim, 1, O.LAPLACE, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x)
    PB.assert_close_scaled(got, want, scale, 1e-12, f"P1 Laplace pull action dim {dim} prec {prec}")
    xn = mg.node_coordinates(pr.mesh, 1)
    u = xn[:, 0].copy()
    y = g.action(fe.FORM_LAPLACE, u, precision=prec, strategy=fe.STRATEGY_PULL)
    _, su = O.action(dim, 1, O.LAPLACE, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, u)
    interior = np.all((xn > 1e-12) & (xn < 1 - 1e-12), axis=1)
    assert interior.sum() > 0
    assert np.all(np.abs(y[interior]) <= 1e-13 * su[interior]), np.max(np.abs(y[interior]) / su[interior])


def test_pull_is_bitwise_reproducible(gpu):
    """Row owners sum in the fixed incidence order: repeated assemblies and actions are bitwise equal."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(3, 2, 6, 0.2, seed=1)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(2).uniform(-1, 1, pr.nnodes)
    for prec in (0, 1):
        a1 = g.assemble(3, precision=prec, strategy=fe.STRATEGY_PULL)
        a2 = g.assemble(3, precision=prec, strategy=fe.STRATEGY_PULL)
        np.testing.assert_array_equal(a1, a2)
        y1 = g.action(3, x, precision=prec, strategy=fe.STRATEGY_PULL)
        y2 = g.action(3, x, precision=prec, strategy=fe.STRATEGY_PULL)
        np.testing.assert_array_equal(y1, y2)
        # after a rebuild (incidence lists refilled by atomics, in a run-dependent order) and from a
        # fresh build in another context, the sums run in the same order again
        g.fe.sparsity_rebuild(g.sparsity())
        np.testing.assert_array_equal(g.assemble(3, precision=prec, strategy=fe.STRATEGY_PULL), a1)
        np.testing.assert_array_equal(g.action(3, x, precision=prec, strategy=fe.STRATEGY_PULL), y1)
        g2 = PB.GpuProblem(pr)
        np.testing.assert_array_equal(g2.assemble(3, precision=prec, strategy=fe.STRATEGY_PULL), a1)
        np.testing.assert_array_equal(g2.action(3, x, precision=prec, strategy=fe.STRATEGY_PULL), y1)


def test_pull_inc_semantics(gpu):
    """zero_first = 0 adds to what the Mat and y hold (INC), for the pull strategy too."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(2, 2, 9, 0.2, seed=1)
    g = PB.GpuProblem(pr)
    k = fe.kernel_create(g.ctx, 3, 2, 2, strategy=fe.STRATEGY_PULL)
    A = fe.mat_create(g.ctx, g.sparsity())
    fe.assemble_mat(g.ctx, k, g.cells, A, g.coords, g.coord_map, zero_first=True)
    fe.assemble_mat(g.ctx, k, g.cells, A, g.coords, g.coord_map, zero_first=False)
    fe.sync(g.ctx)
    twice = fe.mat_values(A).cpu().numpy()
    once = g.assemble(3, strategy=fe.STRATEGY_PULL)
    np.testing.assert_allclose(twice, 2 * once, rtol=1e-15, atol=0)


@pytest.mark.parametrize("dim,p,n,jit", [(2, 1, 37, 0.2), (2, 2, 23, 0.2), (2, 4, 17, 0.2)])
@pytest.mark.parametrize("form", [1, 3, 4])
def test_fp32_element_tensors_frobenius(gpu, dim, p, n, jit, form):
    """FP32 element tensors with FP64 accumulation: relative Frobenius error <= 1e-5 (stated bound)."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(dim, p, n, jit, seed=3, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    got = g.assemble(form, precision=fe.PREC_FP32)
    want, scale = O.assemble_mat(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci, kappa=pr.kappa)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-5, err
    assert np.max(np.abs(got - want) / np.maximum(scale, 1e-300)) <= 1e-5


# ------------------------------------------------------------------ tensor cores (tcgen05, three TF32 products)
@pytest.mark.parametrize("n,jit", [(17, 0.2), (9, 0.0), (1, 0.0)])
def test_tensor_core_p4_kappa(gpu, n, jit):
    """P4 kappa-diffusion element tensors as a [cells x 18] x [18 x 120] product on the tensor cores
    (hi/lo TF32 splits, three products, FP32 accumulation in TMEM), FP64 CSR accumulation:
    relative Frobenius <= 1e-5 and per entry <= 1e-5 of the contribution scale.  Cell counts
    578, 162 and 2 leave full, partial and nearly empty 128-cell tiles."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(2, 4, n, jit, seed=3, kappa_seed=3)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    got = g.assemble(fe.FORM_KAPPA_DIFFUSION, precision=fe.PREC_TF32X3)
    want, scale = O.assemble_mat(2, 4, 4, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci, kappa=pr.kappa)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-5, err
    assert np.max(np.abs(got - want) / np.maximum(scale, 1e-300)) <= 1e-5


def test_tensor_core_refuses_other_elements(gpu):
    from paper_1501_01809_gb300 import fe
    ctx = fe.ctx_create(0)
    for form, dim, p in [(fe.FORM_HELMHOLTZ, 2, 4), (fe.FORM_KAPPA_DIFFUSION, 2, 2), (fe.FORM_KAPPA_DIFFUSION, 3, 2)]:
        with pytest.raises(fe.FeError) as ei:
            fe.kernel_create(ctx, form, dim, p, precision=fe.PREC_TF32X3)
        assert ei.value.code == fe.FE_EUNSUPPORTED
