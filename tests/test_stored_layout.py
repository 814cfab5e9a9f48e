"""The stored-element-matrix layout of fe_elem_matrices / fe_action_stored, on the CPU.

Ke holds entry u of the upper triangle of cell e at Ke[u * ncell + e], u counting the pairs
(i, j), i <= j, row by row.  Applying matrices stored that way, in the order the CUDA kernel
walks them (y_i += K_ij x_j and, off the diagonal, y_j += K_ij x_i), must give the oracle's
action: this pins the layout convention itself to the oracle, independently of any GPU code.
"""
import numpy as np
import pytest

import oracle as O
from tests import problems as PB


def _stored_from_oracle(pr, form):
    nd = pr.cmap.shape[1]
    nup = nd * (nd + 1) // 2
    Ke = np.empty(nup * pr.mesh.ncell)
    cv = pr.mesh.cell_vertex
    for e in range(pr.mesh.ncell):
        K = O.element_matrix(pr.dim, pr.p, form, pr.mesh.coords[cv[e]], pr.kappa[cv[e]] if form == 4 else None)
        u = 0
        for i in range(nd):
            for j in range(i, nd):
                Ke[u * pr.mesh.ncell + e] = K[i, j]
                u += 1
    return Ke


def _apply_stored(pr, Ke, x):
    nd, ncell = pr.cmap.shape[1], pr.mesh.ncell
    y = np.zeros(pr.nnodes)
    for e in range(ncell):
        rows = pr.cmap[e]
        ye = np.zeros(nd)
        u = 0
        for i in range(nd):
            for j in range(i, nd):
                k = Ke[u * ncell + e]
                ye[i] += k * x[rows[j]]
                if i != j:
                    ye[j] += k * x[rows[i]]
                u += 1
        np.add.at(y, rows, ye)
    return y


@pytest.mark.parametrize("dim,p,n,form", [(2, 2, 4, 3), (2, 1, 5, 4), (3, 2, 2, 3)])
def test_stored_layout_gives_the_oracle_action(dim, p, n, form):
    pr = PB.make(dim, p, n, 0.2, seed=5, kappa_seed=5 if form == 4 else None)
    x = np.random.default_rng(7).uniform(-1, 1, pr.nnodes)
    y = _apply_stored(pr, _stored_from_oracle(pr, form), x)
    want, scale = O.action(dim, p, form, pr.cmap, pr.mesh.coords, pr.mesh.cell_vertex, x, kappa=pr.kappa)
    PB.assert_close_scaled(y, want, scale, 1e-12, "stored layout")


def test_element_matrices_are_symmetric():
    """Storing only the upper triangle assumes K_e = K_e^T (every bilinear form here is symmetric)."""
    pr = PB.make(3, 2, 1, 0.2, seed=5, kappa_seed=5)
    cv = pr.mesh.cell_vertex
    for form in (1, 2, 3, 4):
        for e in range(pr.mesh.ncell):
            K = O.element_matrix(3, 2, form, pr.mesh.coords[cv[e]], pr.kappa[cv[e]] if form == 4 else None)
            np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-14 * np.abs(K).max())
