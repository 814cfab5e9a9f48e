"""Pins of the oracle's rank-0 forms and cell-volume reductions (no GPU).

A Global (Sec. 4.3) receives a form of rank 0: here a bilinear form with both arguments the same
Function, a(u, u), or a linear form with its test argument a Function, L(u).  For u the
interpolant of a polynomial the element reproduces exactly, these are integrals with closed
forms on the unit square and cube, whatever the (jittered, affine) mesh:
  u = x:       int |grad u|^2 + u^2 = 1 + 1/3,  int u^2 = 1/3,  int |grad u|^2 = 1;
  u = x^2:     int u^2 = 1/5,  int |grad u|^2 = 4/3                          (P2 and up);
  u = x y:     int |grad u|^2 = 2/3 (square), int u^2 = 1/9 (square)        (P2 and up);
  f = 1, u=x:  int f u = 1/2;  f = x (P1), u = x:  int f u = 1/3.
Cell volumes add up to the domain's volume, 1, jittered or not, and on the unjittered lattice
every cell has volume h^d / d!.  Each value must match within 1e-14 of the oracle's own scale
(the sum of absolute contributions): the value is a sum of a few hundred rounded terms, each
rounding at most one ulp of a partial sum no larger than the scale, so about 90 ulp of the scale
bounds it; a wrong term or coefficient misses by a fixed fraction of the value instead.
"""
import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg

ELEMENTS = [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)]


def _mesh(dim, n, jitter=0.2, seed=3):
    return mg.unit_square_mesh(n, jitter, seed) if dim == 2 else mg.unit_cube_mesh(n, jitter, seed)


def _interp(mesh, p, fn):
    xn = mg.node_coordinates(mesh, p)
    return fn(*[xn[:, k] for k in range(mesh.dim)])


@pytest.mark.parametrize("dim,p", ELEMENTS)
def test_energy_of_x_is_four_thirds(dim, p):
    m = _mesh(dim, 5 if dim == 2 else 3)
    cmap, _ = mg.cell_node_map(m, p)
    u = _interp(m, p, lambda x, *r: x)
    for form, exact in ((O.HELMHOLTZ, 4 / 3), (O.MASS, 1 / 3), (O.LAPLACE, 1.0)):
        val, scale = O.functional(dim, p, form, cmap, m.coords, m.cell_vertex, u)
        assert abs(val - exact) <= 1e-14 * scale, (form, val, exact, scale)


@pytest.mark.parametrize("dim,p", [e for e in ELEMENTS if e[1] >= 2])
def test_quadratics_are_integrated_exactly(dim, p):
    m = _mesh(dim, 4 if dim == 2 else 2)
    cmap, _ = mg.cell_node_map(m, p)
    u = _interp(m, p, lambda x, *r: x * x)
    val, scale = O.functional(dim, p, O.MASS, cmap, m.coords, m.cell_vertex, u)
    assert abs(val - 1 / 5) <= 1e-14 * scale
    val, scale = O.functional(dim, p, O.LAPLACE, cmap, m.coords, m.cell_vertex, u)
    assert abs(val - 4 / 3) <= 1e-14 * scale
    if dim == 2:
        u = _interp(m, p, lambda x, y: x * y)
        val, scale = O.functional(dim, p, O.LAPLACE, cmap, m.coords, m.cell_vertex, u)
        assert abs(val - 2 / 3) <= 1e-14 * scale
        val, scale = O.functional(dim, p, O.MASS, cmap, m.coords, m.cell_vertex, u)
        assert abs(val - 1 / 9) <= 1e-14 * scale


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_kappa_one_is_the_laplacian(dim, p):
    m = _mesh(dim, 4 if dim == 2 else 2)
    cmap, _ = mg.cell_node_map(m, p)
    u = np.random.default_rng(7).uniform(-1, 1, cmap.max() + 1)
    a, sa = O.functional(dim, p, O.KAPPA_DIFFUSION, cmap, m.coords, m.cell_vertex, u, kappa=np.ones(m.nvert))
    b, sb = O.functional(dim, p, O.LAPLACE, cmap, m.coords, m.cell_vertex, u)
    assert abs(a - b) <= 1e-14 * (sa + sb) and a > 0


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_linear_functionals(dim, p):
    m = _mesh(dim, 5 if dim == 2 else 3)
    cmap, _ = mg.cell_node_map(m, p)
    u = _interp(m, p, lambda x, *r: x)
    one = np.ones(m.nvert)
    val, scale = O.linear_functional(dim, p, 1, cmap, m.coords, m.cell_vertex, one, m.cell_vertex, u)
    assert abs(val - 1 / 2) <= 1e-14 * scale
    fx = m.coords[:, 0].copy()
    val, scale = O.linear_functional(dim, p, 1, cmap, m.coords, m.cell_vertex, fx, m.cell_vertex, u)
    assert abs(val - 1 / 3) <= 1e-14 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_volumes(dim):
    n = 8 if dim == 2 else 4
    v = O.cell_volumes(dim, _mesh(dim, n).coords, _mesh(dim, n).cell_vertex)
    assert v.size == (2 * n * n if dim == 2 else 6 * n ** 3) and v.min() > 0
    assert abs(v.sum() - 1.0) <= 1e-16 * v.size
    flat = _mesh(dim, n, jitter=0.0)
    w = O.cell_volumes(dim, flat.coords, flat.cell_vertex)
    h = 1.0 / n
    np.testing.assert_allclose(w, h ** dim / (2 if dim == 2 else 6), rtol=1e-15, atol=0)
