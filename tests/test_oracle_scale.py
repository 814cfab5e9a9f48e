"""Pins of the oracle's per-entry error scale, the tolerance of every parity test (no GPU).

Every GPU parity assertion is |got - want| <= 1e-12 * scale, with ``scale`` accumulated by the
oracle next to the values (the INC of Sec. 4.4.1 adds one contribution per cell; the scale adds
that contribution's conditioning).  A mistake in the scale would loosen every check without
failing any value pin, so it is pinned here against exact rationals:

* element matrix entries: scale_ij = sqrt(K_ii K_jj) of the exact element matrix.  The forms
  here are symmetric positive semi-definite (kappa > 0), the diagonal sums of absolute
  quadrature terms equal K_ii (all terms are non-negative), and by Cauchy-Schwarz over the
  quadrature points and components the off-diagonal sums never exceed sqrt(K_ii K_jj), so the
  floor decides every off-diagonal entry whatever rule the oracle uses;
* the action: scale_i = sum_j sqrt(K_ii K_jj) |x_j|;
* the P1 linear form f v dx with f in P1: every quadrature term has the sign of f_k (the
  barycentric products are non-negative), so scale_i = sum_k |f_k| int(lambda_k lambda_i), i.e.
  M_e |f_e| exactly;
* on jittered meshes: |value| <= scale for every entry, and the row's largest scale is at most
  the sum over the row's cells of their largest |K_e| entry.
"""
from __future__ import annotations

from fractions import Fraction as F

import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg
from tests import exact_fe

_FORMS = {O.MASS: dict(stiff=False), O.LAPLACE: dict(mass=False), O.HELMHOLTZ: {},
          O.KAPPA_DIFFUSION: dict(mass=False)}


def _one_cell_scale(dim, p, form, xv, kv=None):
    """Values and scale of a single cell assembled through the oracle's par_loop (dense pattern)."""
    nd = O.num_nodes(dim, p)
    cmap = np.arange(nd, dtype=np.int32)[None, :]
    cv = np.arange(dim + 1, dtype=np.int32)[None, :]
    rp = np.arange(0, nd * nd + 1, nd, dtype=np.int64)
    ci = np.tile(np.arange(nd, dtype=np.int32), nd)
    kap = None if kv is None else np.asarray(kv, dtype=np.float64)
    vals, absv = O.assemble_mat(dim, p, form, cmap, np.asarray(xv, dtype=np.float64), cv, rp, ci, kappa=kap)
    return vals.reshape(nd, nd), absv.reshape(nd, nd)


def _dyadic_cells(dim, count, seed):
    """Reference-shaped cells with dyadic vertex perturbations (exact in binary)."""
    rng = np.random.default_rng(seed)
    ref = np.vstack([np.zeros(dim), np.eye(dim)])
    out = [ref]
    for _ in range(count):
        xv = ref + rng.integers(-3, 4, size=ref.shape) / 16.0
        J = (xv[1:] - xv[0]).T
        if abs(np.linalg.det(J)) > 0.05:
            out.append(xv)
    return out


def _exact_scale(K):
    d = np.sqrt(np.diag(K))
    return np.outer(d, d)


def pin_scale_element(dim, p, cells=3, seed=0):
    """scale_ij == sqrt(K_ii K_jj) of the exact element matrix, all four forms."""
    kv = [1.5, 0.25, 2.0, 0.75][: dim + 1]
    for xv in _dyadic_cells(dim, cells, seed):
        xf = [[F(float(c)) for c in row] for row in xv]
        for form, kw in _FORMS.items():
            kap = kv if form == O.KAPPA_DIFFUSION else None
            ex = np.array(exact_fe.element_matrix(dim, p, xf, kappa=kap, **kw), dtype=float)
            want = _exact_scale(ex)
            _, got = _one_cell_scale(dim, p, form, xv, kap)
            assert np.all(np.abs(got - want) <= 1e-14 * want.max()), (dim, p, form, np.max(np.abs(got - want)))


def pin_scale_reference_triangle():
    """Hand-computed P1 Helmholtz scale on the reference triangle (0,0),(1,0),(0,1):
    K = stiffness 1/2[[2,-1,-1],[-1,1,0],[-1,0,1]] + mass 1/24[[2,1,1],[1,2,1],[1,1,2]], so the
    diagonal is (13/12, 7/12, 7/12) and scale = sqrt of its outer product; e.g. the (0,1) entry
    sqrt(91)/12 and the (1,2) entry 7/12."""
    _, s = _one_cell_scale(2, 1, O.HELMHOLTZ, [[0, 0], [1, 0], [0, 1]])
    diag = np.array([13 / 12, 7 / 12, 7 / 12])
    np.testing.assert_allclose(s, np.sqrt(np.outer(diag, diag)), rtol=1e-15, atol=0)
    assert abs(s[0, 1] - np.sqrt(91) / 12) <= 1e-15 and abs(s[1, 2] - 7 / 12) <= 1e-15


def pin_scale_action(dim, p, n=2, seed=3):
    """Action scale on a dyadically jittered mesh: sum over cells of sum_j sqrt(K_ii K_jj)|x_j|."""
    m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n)
    coords = m.coords.copy()
    rng = np.random.default_rng(seed)
    interior = np.all((m.vgrid > 0) & (m.vgrid < n), axis=1)
    coords[interior] += rng.integers(-1, 2, size=(interior.sum(), dim)) / (8.0 * n)
    cmap, nn = mg.cell_node_map(m, p)
    x = np.random.default_rng(seed + 1).uniform(-1, 1, nn)
    _, ay = O.action(dim, p, O.HELMHOLTZ, cmap, coords, m.cell_vertex, x)
    want = np.zeros(nn)
    for e in range(m.ncell):
        xf = [[F(float(c)) for c in row] for row in coords[m.cell_vertex[e]]]
        K = np.array(exact_fe.element_matrix(dim, p, xf), dtype=float)
        want[cmap[e]] += _exact_scale(K) @ np.abs(x[cmap[e]])
    assert np.all(np.abs(ay - want) <= 1e-14 * want.max()), np.max(np.abs(ay - want))


def pin_scale_vector_p1(dim, seed=4):
    """P1 linear form with f in P1: scale = M_e |f_e| per cell (exact mass matrix)."""
    for xv in _dyadic_cells(dim, 2, seed):
        fe = np.random.default_rng(seed).uniform(-1, 1, dim + 1)
        fe[0] = -abs(fe[0])  # mixed signs, so that signed and absolute terms differ
        fe[1] = abs(fe[1])
        nd = dim + 1
        _, babs = O.assemble_vec(dim, 1, 1, np.arange(nd, dtype=np.int32)[None, :], nd, np.asarray(xv, float),
                                 np.arange(nd, dtype=np.int32)[None, :], fe, np.arange(nd, dtype=np.int32)[None, :])
        xf = [[F(float(c)) for c in row] for row in xv]
        M = np.array(exact_fe.element_matrix(dim, 1, xf, stiff=False), dtype=float)
        want = M @ np.abs(fe)
        assert np.all(np.abs(babs - want) <= 1e-14 * want.max()), (babs, want)


def pin_scale_bounds(dim, p, n, jitter, kappa_seed=None):
    """On a jittered mesh: |A_rc| <= scale_rc; max_c scale_rc <= sum over the cells of row r of
    max |K_e| (each contribution's scale is at most its element's largest diagonal entry)."""
    m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n, jitter, 13)
    cmap, nn = mg.cell_node_map(m, p)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    form = O.HELMHOLTZ if kappa_seed is None else O.KAPPA_DIFFUSION
    kap = None if kappa_seed is None else mg.lognormal_dat(m.nvert, kappa_seed)
    v, a = O.assemble_mat(dim, p, form, cmap, m.coords, m.cell_vertex, rp, ci, kappa=kap)
    assert np.all(np.abs(v) <= a * (1 + 1e-15))
    kmax = np.array([np.abs(O.element_matrix(dim, p, form, m.coords[m.cell_vertex[e]],
                                             None if kap is None else kap[m.cell_vertex[e]])).max()
                     for e in range(m.ncell)])
    bound = np.zeros(nn)
    for e in range(m.ncell):
        bound[cmap[e]] += kmax[e]
    rowmax = np.maximum.reduceat(a, rp[:-1])
    assert np.all(rowmax <= bound * (1 + 1e-14)), np.max(rowmax / bound)


# ---------------------------------------------------------------------------------------------

def test_scale_reference_triangle():
    pin_scale_reference_triangle()


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_scale_element(dim, p):
    pin_scale_element(dim, p, cells=2 if p >= 3 else 3)


@pytest.mark.parametrize("dim,p,n", [(2, 1, 3), (2, 2, 2), (3, 2, 1)])
def test_scale_action(dim, p, n):
    pin_scale_action(dim, p, n)


@pytest.mark.parametrize("dim", [2, 3])
def test_scale_vector_p1(dim):
    pin_scale_vector_p1(dim)


@pytest.mark.parametrize("dim,p,n,jitter,ks", [(2, 2, 6, 0.2, None), (2, 4, 3, 0.2, 3), (3, 2, 3, 0.2, None),
                                               (3, 1, 4, 0.2, 5)])
def test_scale_bounds(dim, p, n, jitter, ks):
    pin_scale_bounds(dim, p, n, jitter, ks)


def test_signed_off_diagonal_terms_leave_the_scale_unchanged():
    """The off-diagonal absolute-term sums never reach the Cauchy-Schwarz floor, so summing them
    signed (planted mistake 14) must not change any scale: the floor decides every off-diagonal
    entry, as the proof in the module docstring says."""
    xv = _dyadic_cells(3, 2, 9)[-1]
    ref = [_one_cell_scale(d, p, f, xv[: d + 1, :d] if d == 2 else xv, [1.5, 0.25, 2.0, 0.75][: d + 1]
                           if f == O.KAPPA_DIFFUSION else None)[1]
           for d, p in [(2, 2), (3, 2)] for f in _FORMS]
    O.set_mutation(14)
    try:
        got = [_one_cell_scale(d, p, f, xv[: d + 1, :d] if d == 2 else xv, [1.5, 0.25, 2.0, 0.75][: d + 1]
                               if f == O.KAPPA_DIFFUSION else None)[1]
               for d, p in [(2, 2), (3, 2)] for f in _FORMS]
    finally:
        O.set_mutation(0)
    for r, g in zip(ref, got):
        np.testing.assert_array_equal(r, g)
