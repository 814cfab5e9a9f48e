"""Access descriptors of the par_loops (Sec. 4.4): READ arguments (maps, coordinates, coefficients,
the action's x) come back bitwise unchanged from every call, and INC adds to what the output holds
(zero_first = 0) for the push strategy as for pull.  Runs on the GB300 machine."""
import numpy as np
import pytest

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


def test_read_arguments_unchanged(gpu):
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(3, 2, 5, 0.2, seed=4, kappa_seed=4)
    g = PB.GpuProblem(pr)
    x = np.random.default_rng(5).uniform(-1, 1, pr.nnodes)
    reads = {"map": g.t_map, "coord map": g.t_cmap, "coords": g.t_coords, "kappa": g.t_kappa}
    before = {k: v.clone() for k, v in reads.items()}
    runs = [(fe.FORM_HELMHOLTZ, fe.PREC_FP64), (fe.FORM_HELMHOLTZ, fe.PREC_F32X2),
            (fe.FORM_KAPPA_DIFFUSION, fe.PREC_FP64)]  # kappa on tetrahedra is built in FP64
    for strategy in (fe.STRATEGY_PUSH, fe.STRATEGY_PULL):
        for form, prec in runs:
            g.assemble(form, precision=prec, strategy=strategy)
            y = g.action(form, x.copy(), precision=prec, strategy=strategy)
            assert np.isfinite(y).all()
    fmap, nf = mg.cell_node_map(pr.mesh, 2)
    f = mg.uniform_dat(nf, 1)
    f0 = f.copy()
    g.rhs(f, fmap, 2, nf, strategy=fe.STRATEGY_PUSH)
    g.rhs(f, fmap, 2, nf, strategy=fe.STRATEGY_PULL)
    g.fe.sparsity_rebuild(g.sparsity())
    g.fe.sync(g.ctx)
    for k, v in reads.items():
        assert g.torch.equal(v, before[k]), k
    np.testing.assert_array_equal(f, f0)
    # the action's x: a device Dat read by the kernel, checked on the device copy
    tx = g.torch.from_numpy(x).cuda()
    tx0 = tx.clone()
    ty = g.torch.zeros_like(tx)
    k = fe.kernel_create(g.ctx, fe.FORM_HELMHOLTZ, 3, 2, precision=fe.PREC_F32X2)
    fe.action(g.ctx, k, g.cells, fe.dat_create(g.ctx, g.nodes, tx), fe.dat_create(g.ctx, g.nodes, ty), g.map,
              g.coords, g.coord_map, zero_first=True)
    fe.sync(g.ctx)
    assert g.torch.equal(tx, tx0)


@pytest.mark.parametrize("prec", [0, 1])
def test_push_inc_semantics(gpu, prec):
    """zero_first = 0 adds to what the Mat and y hold; the atomics run in another order the second
    time, so the sum agrees with twice the first to rounding."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(3, 2, 5, 0.2, seed=2)
    g = PB.GpuProblem(pr)
    k = fe.kernel_create(g.ctx, fe.FORM_HELMHOLTZ, 3, 2, precision=prec, strategy=fe.STRATEGY_PUSH)
    A = fe.mat_create(g.ctx, g.sparsity())
    fe.assemble_mat(g.ctx, k, g.cells, A, g.coords, g.coord_map, zero_first=True)
    fe.sync(g.ctx)
    once = fe.mat_values(A).cpu().numpy().copy()
    fe.assemble_mat(g.ctx, k, g.cells, A, g.coords, g.coord_map, zero_first=False)
    fe.sync(g.ctx)
    twice = fe.mat_values(A).cpu().numpy()
    scale = np.abs(once).max()
    assert np.abs(twice - 2 * once).max() <= 1e-14 * scale
    x = np.random.default_rng(3).uniform(-1, 1, pr.nnodes)
    tx = g.torch.from_numpy(x).cuda()
    ty = g.torch.zeros_like(tx)
    X, Y = fe.dat_create(g.ctx, g.nodes, tx), fe.dat_create(g.ctx, g.nodes, ty)
    fe.action(g.ctx, k, g.cells, X, Y, g.map, g.coords, g.coord_map, zero_first=True)
    fe.sync(g.ctx)
    y1 = ty.cpu().numpy().copy()
    fe.action(g.ctx, k, g.cells, X, Y, g.map, g.coords, g.coord_map, zero_first=False)
    fe.sync(g.ctx)
    y2 = ty.cpu().numpy()
    assert np.abs(y2 - 2 * y1).max() <= 1e-14 * np.abs(y1).max()


@pytest.mark.parametrize("dim,p,form,prec,strategy", [  # push FP64, push double-float, pull, tensor cores
    (3, 2, 3, 0, 1), (3, 2, 3, 1, 1), (3, 2, 3, 0, 2), (2, 4, 4, 3, 1)])
def test_lookup_table_beyond_row_is_flagged(gpu, dim, p, form, prec, strategy):
    """Check mode (fe_ctx_set_checks): a lookup-table entry that points beyond its CSR row is
    reported as FE_ERANGE at fe_sync and its write is skipped, so no other row changes (the INC of
    Sec. 4.4.1 stays inside the row the map names).  One byte of the library's table is poked from
    the host side; this is a bounds check in the kernels, not a fault."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(dim, p, 4 if dim == 3 else 3, 0.2, seed=6, kappa_seed=3 if form == 4 else None)
    g = PB.GpuProblem(pr, checks=True)
    k = fe.kernel_create(g.ctx, form, dim, p, precision=prec, strategy=strategy)
    A = fe.mat_create(g.ctx, g.sparsity())
    fe.assemble_mat(g.ctx, k, g.cells, A, g.coords, g.coord_map, g.coeffs(form), zero_first=True)
    fe.sync(g.ctx)
    clean = fe.mat_values(A).cpu().numpy().copy()
    nd = pr.cmap.shape[1]
    lut = fe.sparsity_lut(g.sparsity(), pr.mesh.ncell, nd, nd)
    e, i, j = pr.mesh.ncell // 2, 1, nd - 2
    r = int(pr.cmap[e, i])
    rp, _ = g.csr()
    assert rp[r + 1] - rp[r] < 255
    lut[e * nd * nd + i * nd + j] = 255
    fe.assemble_mat(g.ctx, k, g.cells, A, g.coords, g.coord_map, g.coeffs(form), zero_first=True)
    with pytest.raises(fe.FeError) as ei:
        fe.sync(g.ctx)
    assert ei.value.code == fe.FE_ERANGE and "lookup-table entry" in str(ei.value)
    got = fe.mat_values(A).cpu().numpy()
    outside = np.ones(len(clean), dtype=bool)
    outside[rp[r]:rp[r + 1]] = False
    tol = 0 if strategy == fe.STRATEGY_PULL else 1e-13 * np.abs(clean).max()
    assert np.abs(got[outside] - clean[outside]).max() <= tol
    # the skipped contribution is the only difference inside the row
    assert np.count_nonzero(np.abs(got[~outside] - clean[~outside]) > 1e-13 * np.abs(clean).max()) <= 1
