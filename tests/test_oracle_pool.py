"""The many-core oracle driver (tests/oracle_pool.py) gives exactly the single-process oracle's
results: the same pattern slices, values, scales and action, bit for bit (no GPU)."""
import numpy as np

import oracle as O
from tests import oracle_pool as OP
from tests import problems as PB


def test_pool_matches_single_process():
    pr = PB.make(3, 2, 3, 0.2, seed=1)
    rp, ci = O.sparsity(pr.cmap, pr.cmap, pr.nnodes, pr.nnodes)
    want_v, want_a = O.assemble_mat(3, 2, O.HELMHOLTZ, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci)
    got_v, got_a = OP.assemble_mat_full(3, 2, O.HELMHOLTZ, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci,
                                        procs=2)
    np.testing.assert_array_equal(got_v, want_v)
    np.testing.assert_array_equal(got_a, want_a)
    x = np.random.default_rng(2).uniform(-1, 1, pr.nnodes)
    wy, wa = O.action(3, 2, O.HELMHOLTZ, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x)
    gy, ga = OP.action_full(3, 2, O.HELMHOLTZ, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x, procs=2)
    np.testing.assert_array_equal(gy, wy)
    np.testing.assert_array_equal(ga, wa)


def test_pool_kappa_and_items():
    pr = PB.make(2, 4, 3, 0.2, seed=2, kappa_seed=3)
    rp, ci = O.sparsity(pr.cmap, pr.cmap, pr.nnodes, pr.nnodes)
    want = O.assemble_mat(2, 4, O.KAPPA_DIFFUSION, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci,
                          kappa=pr.kappa)
    got = OP.assemble_mat_full(2, 4, O.KAPPA_DIFFUSION, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci,
                               kappa=pr.kappa, procs=2)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
    f = np.random.default_rng(3).uniform(-1, 1, pr.nnodes)
    (v, a, b, ba), = OP.assemble_items([(2, 4, O.HELMHOLTZ, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, rp, ci, f)],
                                       procs=1)
    np.testing.assert_array_equal(v, O.assemble_mat(2, 4, O.HELMHOLTZ, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex,
                                                    rp, ci)[0])
    np.testing.assert_array_equal(b, O.assemble_vec(2, 4, 4, pr.cmap, pr.nnodes, pr.mesh.coords, pr.mesh.cell_vertex,
                                                    f, pr.cmap)[0])
