"""Batches of many meshes in one persistent launch vs the CPU oracle (runs on the GB300 machine).

Every item of a batch (its Mat and its right-hand side) is held to the same per-entry bound as a
single assembly: |a - a_ref| <= 1e-12 * S_ij, relative Frobenius <= 1e-12.  Mesh sizes follow the
log-uniform mix of the batched workload, at sizes the oracle finishes in seconds; the batch mixes
P1/P2, Mass/Laplace/Helmholtz, FP64 and double-float element tensors, and single-cell and empty
meshes.
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


def _mixed(count, seed, lo=2, hi=40):
    ns, ps = mg.batch_mesh_sizes(count, seed, lo, hi)
    probs, forms, precs = [], [], []
    for i, (n, p) in enumerate(zip(ns, ps)):
        probs.append(PB.make(2, int(p), int(n), 0.2 if n > 2 else 0.0, seed=seed + i))
        forms.append((1, 2, 3)[i % 3])
        precs.append(i % 2)
    return probs, forms, precs


def _check_item(b, i, what):
    pr, form = b.problems[i], b.forms[i]
    rp, ci = b.gp[i].csr()
    vals, rhs = b.results(i)
    want, scale = O.assemble_mat(2, pr.p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci)
    PB.assert_close_scaled(vals, want, scale, 1e-12, f"{what}: item {i} Mat (P{pr.p} form {form})")
    wv, sv = O.assemble_vec(2, pr.p, pr.p, pr.cmap, pr.nnodes, pr.mesh.coords, pr.mesh.cell_vertex, b.f[i], pr.cmap)
    PB.assert_close_scaled(rhs, wv, sv, 1e-12, f"{what}: item {i} rhs")


def test_batch_matches_oracle_direct_graph_and_tuned(gpu):
    from paper_1501_01809_gb300 import fe
    probs, forms, precs = _mixed(24, 5)
    b = PB.GpuBatch(probs, forms, precs)
    # poison the outputs: assembly must zero them itself
    for i in range(len(probs)):
        v, r = fe.batch_values(b.batch, i)
        v.fill_(np.nan)
        r.fill_(np.nan)
    fe.batch_assemble(b.batch, use_graph=False)
    fe.sync(b.ctx)
    for i in range(len(probs)):
        _check_item(b, i, "direct")
    for _ in range(3):  # graph replays re-zero every time
        fe.batch_assemble(b.batch, use_graph=True)
    fe.sync(b.ctx)
    for i in range(len(probs)):
        _check_item(b, i, "graph")
    tile, grid, ms = fe.batch_tune(b.batch, reps=2)
    assert tile in (256, 1024, 4096, 16384) and grid % 152 == 0 and ms > 0
    fe.batch_assemble(b.batch, use_graph=True)
    fe.sync(b.ctx)
    for i in range(len(probs)):
        _check_item(b, i, f"tuned tile {tile} grid {grid}")


def test_batch_equals_single_assemblies(gpu):
    """Batched results equal the per-mesh push assemblies of the same problems (same bound)."""
    from paper_1501_01809_gb300 import fe
    probs, forms, precs = _mixed(8, 21, lo=4, hi=30)
    b = PB.GpuBatch(probs, forms, precs)
    fe.batch_assemble(b.batch, use_graph=True)
    fe.sync(b.ctx)
    for i, (pr, form, prec) in enumerate(zip(probs, forms, precs)):
        vals, rhs = b.results(i)
        single = b.gp[i].assemble(form, precision=prec, strategy=fe.STRATEGY_PUSH)
        rp, ci = b.gp[i].csr()
        _, scale = O.assemble_mat(2, pr.p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci)
        PB.assert_close_scaled(vals, single, scale, 1e-12, f"item {i} batched vs single")


def test_batch_single_cell_and_empty_meshes(gpu):
    from paper_1501_01809_gb300 import fe
    one = PB.make(2, 2, 1, 0.0)
    one.mesh.cell_vertex = one.mesh.cell_vertex[:1].copy()
    one.cmap = one.cmap[:1].copy()
    probs = [one, PB.make(2, 1, 3, 0.0)]
    b = PB.GpuBatch(probs, [3, 2], [0, 1])
    fe.batch_assemble(b.batch, use_graph=True)
    fe.sync(b.ctx)
    for i in range(2):
        _check_item(b, i, "small")
    empty = fe.batch_create(b.ctx, [])
    fe.batch_assemble(empty, use_graph=True)
    fe.batch_assemble(empty, use_graph=False)
    fe.sync(b.ctx)
    with pytest.raises(fe.FeError):
        fe.batch_values(empty, 0)


def test_batch_rejects_unbatched_elements(gpu):
    from paper_1501_01809_gb300 import fe
    for dim, p, prec, form in [(3, 1, 0, 3), (2, 3, 0, 3), (2, 1, fe.PREC_FP32, 3), (2, 1, 0, fe.FORM_KAPPA_DIFFUSION)]:
        pr = PB.make(dim, p, 2, 0.0)
        g = PB.GpuProblem(pr)
        k = fe.kernel_create(g.ctx, form, dim, p, precision=prec)
        with pytest.raises(fe.FeError) as ei:
            fe.batch_create(g.ctx, [dict(kmat=k, cells=g.cells, sp=g.sparsity(), coords=g.coords,
                                         coord_map=g.coord_map)])
        assert ei.value.code == fe.FE_EUNSUPPORTED, (dim, p, prec, form)


def test_batch_buffers_are_the_items_back_to_back(gpu):
    from paper_1501_01809_gb300 import fe
    probs, forms, precs = _mixed(5, 33, lo=3, hi=12)
    b = PB.GpuBatch(probs, forms, precs)
    fe.batch_assemble(b.batch, use_graph=False)
    fe.sync(b.ctx)
    va, ra = (t.cpu().numpy() for t in fe.batch_buffers(b.batch))
    vs = np.concatenate([b.results(i)[0] for i in range(5)])
    rs = np.concatenate([b.results(i)[1] for i in range(5)])
    np.testing.assert_array_equal(va, vs)
    np.testing.assert_array_equal(ra, rs)
