"""Parity at the workloads' full sizes, in the launch configuration bench.py times (GB300).

The oracle cannot assemble 1.5M P2 tetrahedra in seconds, so it computes sampled rows one by one:
each sampled row's pattern by brute force from the input map (the nodes of the cells incident to
the row), its values with the oracle restricted to those cells.  The GPU's full pattern is also
checked against the nnz closed form, and the action against the oracle on the incident cells.
"""
import numpy as np
import pytest

import oracle as O
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


def _sample_rows(nn, rng, k=160):
    rows = set([0, 1, nn // 2, nn - 2, nn - 1])
    rows.update(rng.integers(0, nn, size=k).tolist())
    return np.array(sorted(rows), dtype=np.int64)


def _oracle_rows(pr, rows, form, kappa=None):
    """Brute-force pattern of the sampled rows and their oracle values (cells touching them only)."""
    cmap = pr.cmap
    hit = np.isin(cmap, rows)
    cells = np.nonzero(hit.any(axis=1))[0]
    sub = cmap[cells]
    pattern = {int(r): set() for r in rows}
    for e in range(sub.shape[0]):
        for r in sub[e]:
            if int(r) in pattern:
                pattern[int(r)].update(int(c) for c in sub[e])
    srp = np.zeros(len(rows) + 1, dtype=np.int64)
    cols = []
    for t, r in enumerate(rows):
        cs = sorted(pattern[int(r)])
        cols.extend(cs)
        srp[t + 1] = srp[t] + len(cs)
    sci = np.array(cols, dtype=np.int32)
    vals, absv = O.assemble_rows(pr.dim, pr.p, form, np.ascontiguousarray(sub), pr.mesh.coords,
                                 np.ascontiguousarray(pr.mesh.cell_vertex[cells]), pr.nnodes, rows, srp, sci,
                                 kappa=kappa)
    return srp, sci, vals, absv, cells


def _check_rows(g, rows, srp, sci, vals, absv, got_vals, rtol, what):
    rp, ci = g.csr()
    for t, r in enumerate(rows):
        np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], sci[srp[t]:srp[t + 1]], err_msg=f"{what}: row {r}")
    got = np.concatenate([got_vals[rp[r]:rp[r + 1]] for r in rows])
    PB.assert_close_scaled(got, vals, absv, rtol, what)


def test_p2_cube_64_assembly_and_action_sampled(gpu):
    """P2 UnitCubeMesh 64^3, jitter 0.2h seed 0 (1,572,864 cells): nnz closed form, sampled rows in
    FP64 and double-float push (the timed configuration) and pull, and sampled action entries."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(3, 2, 64, 0.2, seed=0)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    n = 64
    assert len(ci) == 230 * n ** 3 + 138 * n ** 2 + 24 * n + 1 == 60859905
    rng = np.random.default_rng(7)
    rows = _sample_rows(pr.nnodes, rng)
    srp, sci, vals, absv, cells = _oracle_rows(pr, rows, O.HELMHOLTZ)
    for prec, strat in [(fe.PREC_F32X2, fe.STRATEGY_PUSH), (fe.PREC_FP64, fe.STRATEGY_PUSH),
                        (fe.PREC_F32X2, fe.STRATEGY_PULL)]:
        got = g.assemble(fe.FORM_HELMHOLTZ, precision=prec, strategy=strat)
        _check_rows(g, rows, srp, sci, vals, absv, got, 1e-12, f"P2 64^3 prec {prec} strategy {strat}")
    x = np.random.default_rng(2).uniform(-1, 1, pr.nnodes)
    ysub, yabs = O.action(3, 2, O.HELMHOLTZ, np.ascontiguousarray(pr.cmap[cells]), pr.mesh.coords,
                          np.ascontiguousarray(pr.mesh.cell_vertex[cells]), x)
    for prec in (fe.PREC_F32X2, fe.PREC_FP64):
        y = g.action(fe.FORM_HELMHOLTZ, x, precision=prec)
        PB.assert_close_scaled(y[rows], ysub[rows], yabs[rows], 1e-12, f"P2 64^3 action prec {prec}")


def test_p1_square_64_full(gpu):
    """P1 UnitSquareMesh 64x64 Helmholtz (the whole matrix) and the RHS of f in P1, push and pull."""
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg
    pr = PB.make(2, 1, 64, 0.0)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    want, scale = O.assemble_mat(2, 1, O.HELMHOLTZ, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci)
    f = mg.uniform_dat(pr.nnodes, 1)
    bw, bs = O.assemble_vec(2, 1, 1, pr.cmap, pr.nnodes, pr.mesh.coords, pr.mesh.cell_vertex, f, pr.cmap)
    for strat in (fe.STRATEGY_PUSH, fe.STRATEGY_PULL):
        PB.assert_close_scaled(g.assemble(3, strategy=strat), want, scale, 1e-12, "P1 64x64")
        PB.assert_close_scaled(g.rhs(f, pr.cmap, 1, pr.nnodes, strategy=strat), bw, bs, 1e-12, "P1 64x64 RHS")


def test_p4_square_512_kappa_fp32_sampled(gpu):
    """P4 UnitSquareMesh 512x512 kappa-diffusion (kappa = exp(N(0,1)) per P1 node, seed 3): FP32
    element tensors (CUDA cores, and three TF32 tensor-core products), FP64 accumulation -- relative
    Frobenius error <= 1e-5 over sampled rows; the
    double-float variant of P2 and FP64 P4 stay at 1e-12."""
    from paper_1501_01809_gb300 import fe
    pr = PB.make(2, 4, 512, 0.0, kappa_seed=3)
    g = PB.GpuProblem(pr)
    rp, ci = g.csr()
    assert len(ci) == 376 * 512 ** 2 + 48 * 512 + 1
    rows = _sample_rows(pr.nnodes, np.random.default_rng(9))
    srp, sci, vals, absv, _ = _oracle_rows(pr, rows, O.KAPPA_DIFFUSION, kappa=pr.kappa)
    got32 = g.assemble(fe.FORM_KAPPA_DIFFUSION, precision=fe.PREC_FP32)
    got = np.concatenate([got32[rp[r]:rp[r + 1]] for r in rows])
    err = np.linalg.norm(got - vals) / np.linalg.norm(vals)
    assert err <= 1e-5, err
    gottc = g.assemble(fe.FORM_KAPPA_DIFFUSION, precision=fe.PREC_TF32X3)  # tensor cores
    got = np.concatenate([gottc[rp[r]:rp[r + 1]] for r in rows])
    err = np.linalg.norm(got - vals) / np.linalg.norm(vals)
    assert err <= 1e-5, err
    got64 = g.assemble(fe.FORM_KAPPA_DIFFUSION, precision=fe.PREC_FP64)
    _check_rows(g, rows, srp, sci, vals, absv, got64, 1e-12, "P4 512^2 kappa FP64")
