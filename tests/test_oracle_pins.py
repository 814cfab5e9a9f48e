"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each check compares the oracle with something other than itself: hand-computed element
matrices, closed forms of the structured-mesh stencils, exact-rational brute force,
polynomial reproduction, conservation identities, quadrature exactness on monomials, the
O(h^2)/O(h^3) convergence of Poisson's problem to a manufactured solution (the paper's
Poisson experiment, Sec. 6.2), and brute-force sparsity sets.  The ``pin_*`` functions are
also run with planted mistakes (tests/test_oracle_mutations.py).
"""
from __future__ import annotations

import os
from fractions import Fraction as F
from itertools import product
from math import factorial

import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg
from tests import exact_fe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if not _isnum(tok[0]):
                cur = tok[0]
                out[cur] = []
            else:
                out[cur].append([float(F(t)) for t in tok])
    return {k: np.array(v) for k, v in out.items()}


def _isnum(t):
    try:
        F(t)
        return True
    except ValueError:
        return False


def _scipy_csr(rowptr, colidx, vals, n, m=None):
    sp = pytest.importorskip("scipy.sparse")
    return sp.csr_matrix((vals, colidx, rowptr), shape=(n, m or n))


# ---------------------------------------------------------------------------------------------
# pins as plain functions (raise AssertionError) so the mutation tests can reuse them
# ---------------------------------------------------------------------------------------------

def pin_reference_elements():
    """Hand-computed P1 element matrices on the reference triangle and tetrahedron."""
    g = _read_golden("p1_reference_elements.txt")
    tri = [[0, 0], [1, 0], [0, 1]]
    tet = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    np.testing.assert_allclose(O.element_matrix(2, 1, O.LAPLACE, tri), g["triangle_stiffness"], atol=1e-15)
    np.testing.assert_allclose(O.element_matrix(2, 1, O.MASS, tri), g["triangle_mass"], atol=1e-15)
    np.testing.assert_allclose(O.element_matrix(3, 1, O.LAPLACE, tet), g["tet_stiffness"], atol=1e-15)
    np.testing.assert_allclose(O.element_matrix(3, 1, O.MASS, tet), g["tet_mass"], atol=1e-15)
    np.testing.assert_allclose(O.element_matrix(2, 1, O.HELMHOLTZ, tri),
                               g["triangle_stiffness"] + g["triangle_mass"], atol=1e-15)


def pin_p1_interior_row(n=64):
    """P1 Helmholtz on the right-diagonal mesh: interior row = 4 + h^2/2 on the diagonal,
    -1 + h^2/12 at the 4 axis neighbours, h^2/12 at the 2 diagonal neighbours, row sum h^2."""
    m = mg.unit_square_mesh(n)
    cmap, nn = mg.cell_node_map(m, 1)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    v, _ = O.assemble_mat(2, 1, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, rp, ci)
    h = 1.0 / n
    for (i, j) in [(1, 1), (n // 2, n // 3), (n - 1, n - 1)]:
        r = i + (n + 1) * j
        cols, vals = ci[rp[r]:rp[r + 1]], v[rp[r]:rp[r + 1]]
        want = {r: 4 + h * h / 2,
                r - 1: -1 + h * h / 12, r + 1: -1 + h * h / 12,
                r - (n + 1): -1 + h * h / 12, r + (n + 1): -1 + h * h / 12,
                r + (n + 2): h * h / 12, r - (n + 2): h * h / 12}
        assert sorted(cols.tolist()) == sorted(want)
        for c, x in zip(cols, vals):
            assert abs(x - want[int(c)]) <= 1e-14, (r, c, x, want[int(c)])
        assert abs(vals.sum() - h * h) <= 1e-14


def pin_mass_sum_and_stiffness_rows(dim, p, n, jitter):
    """sum of all mass entries = |Omega| = 1; stiffness (Laplace, kappa-diffusion) rows sum to 0."""
    m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n, jitter, 7)
    cmap, nn = mg.cell_node_map(m, p)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    vm, am = O.assemble_mat(dim, p, O.MASS, cmap, m.coords, m.cell_vertex, rp, ci)
    assert abs(vm.sum() - 1.0) <= 1e-13 * am.sum()
    kappa = mg.lognormal_dat(m.nvert, 3)
    for form, kap in [(O.LAPLACE, None), (O.KAPPA_DIFFUSION, kappa)]:
        vs, ab = O.assemble_mat(dim, p, form, cmap, m.coords, m.cell_vertex, rp, ci, kappa=kap)
        rows = np.add.reduceat(vs, rp[:-1])
        scale = np.add.reduceat(ab, rp[:-1])
        assert np.all(np.abs(rows) <= 1e-13 * scale)


def _poly_eval(poly, X):
    out = np.zeros(X.shape[0])
    for e, c in poly.items():
        t = np.full(X.shape[0], float(c))
        for k, a in enumerate(e):
            t = t * X[:, k] ** a
        out += t
    return out


def _cube_integral(poly):
    s = F(0)
    for e, c in poly.items():
        t = F(c)
        for a in e:
            t /= (a + 1)
        s += t
    return s


def _random_poly(dim, deg, rng):
    return {e: F(int(rng.integers(-3, 4))) for e in exact_fe.monomials(dim, deg)}


def pin_polynomial_reproduction(dim, p, n, jitter, seed=0):
    """For u, v polynomials of degree <= p (exactly represented in P_p), U^T A V equals
    int grad u . grad v + u v over the unit square/cube in closed form, on jittered meshes too;
    likewise v^T b = int f v for the linear form and v^T (A u) for the action."""
    rng = np.random.default_rng(seed)
    m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n, jitter, 11)
    cmap, nn = mg.cell_node_map(m, p)
    X = mg.node_coordinates(m, p)
    u, v = _random_poly(dim, p, rng), _random_poly(dim, p, rng)
    U, V = _poly_eval(u, X), _poly_eval(v, X)
    exact = _cube_integral(exact_fe.poly_mul(u, v))
    for k in range(dim):
        exact += _cube_integral(exact_fe.poly_mul(exact_fe.poly_diff(u, k), exact_fe.poly_diff(v, k)))
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    vals, absv = O.assemble_mat(dim, p, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, rp, ci)
    A = _scipy_csr(rp, ci, vals, nn)
    got = V @ (A @ U)
    scale = np.abs(V) @ (_scipy_csr(rp, ci, absv, nn) @ np.abs(U))
    assert abs(got - float(exact)) <= 1e-12 * scale, (got, float(exact))
    y, _ = O.action(dim, p, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, U)
    assert abs(V @ y - float(exact)) <= 1e-12 * scale
    # linear form with f in P_p: v^T b = int f v
    f = _random_poly(dim, p, rng)
    Fv = _poly_eval(f, X)
    b, babs = O.assemble_vec(dim, p, p, cmap, nn, m.coords, m.cell_vertex, Fv, cmap)
    exact_b = _cube_integral(exact_fe.poly_mul(f, v))
    assert abs(V @ b - float(exact_b)) <= 1e-12 * (np.abs(V) @ babs)


def pin_exact_rational(dim, p, n):
    """Oracle element matrices on a dyadically jittered mesh against exact rational integrals."""
    m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n)
    rng = np.random.default_rng(5)
    coords = m.coords.copy()
    interior = np.all((m.vgrid > 0) & (m.vgrid < n), axis=1)
    coords[interior] += rng.integers(-1, 2, size=(interior.sum(), dim)) / (8.0 * n)  # exact binary
    kap = [1.5, 0.25, 2.0, 0.75][: dim + 1]
    for e in range(m.ncell):
        xv = coords[m.cell_vertex[e]]
        xf = [[F(float(c)) for c in row] for row in xv]
        for form, kw in [(O.HELMHOLTZ, {}), (O.MASS, dict(stiff=False)), (O.LAPLACE, dict(mass=False)),
                         (O.KAPPA_DIFFUSION, dict(mass=False, kappa=kap))]:
            ex = np.array(exact_fe.element_matrix(dim, p, xf, **kw), dtype=float)
            got = O.element_matrix(dim, p, form, xv, kap if form == O.KAPPA_DIFFUSION else None)
            assert np.max(np.abs(got - ex)) <= 1e-14 * np.max(np.abs(ex)), (e, form)


def pin_quadrature_monomials(dim, m):
    """Collapsed Gauss rule integrates xi^a (total degree <= 2m-dim) exactly on the reference simplex."""
    pts, wts = O.quadrature(dim, m)
    deg = 2 * m - dim
    for e in product(range(deg + 1), repeat=dim):
        if sum(e) > deg:
            continue
        exact = np.prod([factorial(a) for a in e]) / factorial(sum(e) + dim)
        got = np.sum(wts * np.prod(pts ** np.array(e), axis=1))
        assert abs(got - exact) <= 1e-15, (e, got, exact)


def pin_sparsity_bruteforce(dim, p, n, pr=None):
    """CSR pattern == sorted set of (rmap(e)[i], cmap(e)[j]) pairs (also rectangular: P_p x P_pr)."""
    m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n)
    rmap, nr = mg.cell_node_map(m, p)
    cmap, nc = mg.cell_node_map(m, pr or p)
    rp, ci = O.sparsity(rmap, cmap, nr, nc)
    pairs = sorted({(int(r), int(c)) for e in range(m.ncell) for r in rmap[e] for c in cmap[e]})
    assert len(pairs) == len(ci)
    rows = np.repeat(np.arange(nr), np.diff(rp))
    assert list(zip(rows.tolist(), ci.tolist())) == pairs


# ---------------------------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------------------------

def test_reference_elements():
    pin_reference_elements()


def test_p1_interior_row_closed_form():
    pin_p1_interior_row()


@pytest.mark.parametrize("dim,p,n,jitter", [(2, 1, 16, 0.0), (2, 2, 8, 0.2), (2, 4, 4, 0.2),
                                            (3, 1, 4, 0.2), (3, 2, 3, 0.2)])
def test_mass_sum_and_stiffness_rows(dim, p, n, jitter):
    pin_mass_sum_and_stiffness_rows(dim, p, n, jitter)


@pytest.mark.parametrize("dim,p,n,jitter", [(2, 1, 8, 0.2), (2, 2, 6, 0.2), (2, 3, 4, 0.2), (2, 4, 3, 0.2),
                                            (3, 1, 3, 0.2), (3, 2, 3, 0.2)])
def test_polynomial_reproduction(dim, p, n, jitter):
    pin_polynomial_reproduction(dim, p, n, jitter)


@pytest.mark.parametrize("dim,p,n", [(2, 1, 2), (2, 2, 2), (2, 4, 1), (3, 1, 1), (3, 2, 1)])
def test_exact_rational(dim, p, n):
    pin_exact_rational(dim, p, n)


@pytest.mark.parametrize("dim,m", [(2, 1), (2, 2), (2, 4), (2, 7), (3, 2), (3, 3), (3, 5)])
def test_quadrature_monomials(dim, m):
    pin_quadrature_monomials(dim, m)


def test_gauss_legendre_textbook():
    """m = 2 Gauss-Legendre on [0,1]: nodes (1 -+ 1/sqrt 3)/2, weights 1/2."""
    x, w = O.gauss_legendre01(2)
    np.testing.assert_allclose(sorted(x), [(1 - 3 ** -0.5) / 2, (1 + 3 ** -0.5) / 2], atol=1e-16)
    np.testing.assert_allclose(w, [0.5, 0.5], atol=1e-16)


@pytest.mark.parametrize("dim,p,n,pr", [(2, 1, 3, None), (2, 2, 3, None), (2, 4, 2, None), (3, 2, 2, None),
                                        (2, 2, 2, 1), (3, 1, 2, 2)])
def test_sparsity_bruteforce(dim, p, n, pr):
    pin_sparsity_bruteforce(dim, p, n, pr)


@pytest.mark.parametrize("dim,p,formula", [
    (2, 1, lambda n: 7 * n * n + 6 * n + 1),
    (2, 2, lambda n: 46 * n * n + 16 * n + 1),
    (2, 4, lambda n: 376 * n * n + 48 * n + 1),
    (3, 2, lambda n: 230 * n ** 3 + 138 * n * n + 24 * n + 1)])
def test_nnz_closed_forms(dim, p, formula):
    """nnz of the structured patterns.  P1-2D: N + 2E = (n+1)^2 + 2(3n^2+2n) (vertex + edge
    neighbours); the others are polynomial in n and checked at several n."""
    for n in ([2, 3, 5, 64] if dim == 2 and p == 1 else [2, 3, 4] if dim == 3 else [2, 3, 5]):
        m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n)
        cmap, nn = mg.cell_node_map(m, p)
        _, ci = O.sparsity(cmap, cmap, nn, nn)
        assert len(ci) == formula(n), (n, len(ci), formula(n))


def test_symmetry():
    """Structure symmetric bit-exact; values symmetric within rounding (jittered P2 tets)."""
    m = mg.unit_cube_mesh(3, 0.2, 1)
    cmap, nn = mg.cell_node_map(m, 2)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    v, a = O.assemble_mat(3, 2, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, rp, ci)
    A = _scipy_csr(rp, ci, v, nn)
    At = A.T.tocsr()
    At.sort_indices()
    # structure: the transpose has exactly the same (rowptr, colidx)
    np.testing.assert_array_equal(At.indptr, rp)
    np.testing.assert_array_equal(At.indices, ci)
    # values: A_ij - A_ji within rounding of the contributions
    St = _scipy_csr(rp, ci, a, nn).T.tocsr()
    St.sort_indices()
    assert np.all(np.abs(At.data - v) <= 1e-14 * np.maximum(a, St.data))


def test_kappa_one_is_stiffness():
    """kappa = 1 diffusion equals the Laplace (stiffness) matrix; P4 triangles."""
    m = mg.unit_square_mesh(4, 0.2, 2)
    cmap, nn = mg.cell_node_map(m, 4)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    k1, a1 = O.assemble_mat(2, 4, O.KAPPA_DIFFUSION, cmap, m.coords, m.cell_vertex, rp, ci,
                            kappa=np.ones(m.nvert))
    st, _ = O.assemble_mat(2, 4, O.LAPLACE, cmap, m.coords, m.cell_vertex, rp, ci)
    assert np.all(np.abs(k1 - st) <= 1e-13 * a1)


def test_rhs_sum_is_mass_times_f():
    """Sum of the P1 RHS b = M f equals 1^T M f and the integral of f (C1-style inputs)."""
    m = mg.unit_square_mesh(16)
    cmap, nn = mg.cell_node_map(m, 1)
    f = mg.uniform_dat(nn, 1)
    b, babs = O.assemble_vec(2, 1, 1, cmap, nn, m.coords, m.cell_vertex, f, cmap)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    mv, _ = O.assemble_mat(2, 1, O.MASS, cmap, m.coords, m.cell_vertex, rp, ci)
    M = _scipy_csr(rp, ci, mv, nn)
    np.testing.assert_allclose(b, M @ f, rtol=0, atol=1e-15)
    assert abs(b.sum() - np.ones(nn) @ (M @ f)) <= 1e-14 * babs.sum()


def test_action_equals_csr_spmv():
    """The cell-wise action equals the assembled CSR matrix times x (two routes)."""
    m = mg.unit_cube_mesh(3, 0.2, 0)
    cmap, nn = mg.cell_node_map(m, 2)
    x = mg.uniform_dat(nn, 2)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    v, a = O.assemble_mat(3, 2, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, rp, ci)
    y, ay = O.action(3, 2, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, x)
    y2 = _scipy_csr(rp, ci, v, nn) @ x
    assert np.all(np.abs(y - y2) <= 1e-13 * ay)


def test_assemble_rows_matches_full():
    m = mg.unit_cube_mesh(3, 0.2, 0)
    cmap, nn = mg.cell_node_map(m, 2)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    v, a = O.assemble_mat(3, 2, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, rp, ci)
    rows = np.array([0, 5, 17, nn // 2, nn - 1], dtype=np.int64)
    srp = np.concatenate([[0], np.cumsum(np.diff(rp)[rows])]).astype(np.int64)
    sci = np.concatenate([ci[rp[r]:rp[r + 1]] for r in rows]).astype(np.int32)
    sv, sa = O.assemble_rows(3, 2, O.HELMHOLTZ, cmap, m.coords, m.cell_vertex, nn, rows, srp, sci)
    full = np.concatenate([v[rp[r]:rp[r + 1]] for r in rows])
    np.testing.assert_array_equal(sv, full)


def _poisson_l2_error(dim, p, n, problem):
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n)
    cmap, nn = mg.cell_node_map(m, p)
    X = mg.node_coordinates(m, p)
    u_ex, f_ex, on_dirichlet = problem
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    v, _ = O.assemble_mat(dim, p, O.LAPLACE, cmap, m.coords, m.cell_vertex, rp, ci)
    b, _ = O.assemble_vec(dim, p, p, cmap, nn, m.coords, m.cell_vertex, f_ex(X), cmap)
    A = sp.csr_matrix((v, ci, rp), shape=(nn, nn))
    free = ~on_dirichlet(X)
    uh = np.zeros(nn)
    uh[free] = spla.spsolve(A[free][:, free].tocsc(), b[free])
    xq, wq, uq = O.eval_function(dim, p, 2 * p + 6, cmap, m.coords, m.cell_vertex, uh)
    return np.sqrt(np.sum(wq * (uq - u_ex(xq)) ** 2))


_K, _M = 1, 2
_SQUARE = (lambda X: np.sin(_K * np.pi * X[:, 0]) * np.sin(_M * np.pi * X[:, 1]),
           lambda X: (_K ** 2 + _M ** 2) * np.pi ** 2 * np.sin(_K * np.pi * X[:, 0]) * np.sin(_M * np.pi * X[:, 1]),
           lambda X: np.any((np.abs(X) < 1e-12) | (np.abs(X - 1) < 1e-12), axis=1))
# the paper's Poisson problem (Sec. 6.2): u = cos(4 pi x) sin(4 pi y) cos(4 pi z), f = 48 pi^2 u,
# u = 0 on y = 0 and y = 1, natural (zero-flux) condition elsewhere
_CUBE = (lambda X: np.cos(4 * np.pi * X[:, 0]) * np.sin(4 * np.pi * X[:, 1]) * np.cos(4 * np.pi * X[:, 2]),
         lambda X: 48 * np.pi ** 2 * np.cos(4 * np.pi * X[:, 0]) * np.sin(4 * np.pi * X[:, 1])
         * np.cos(4 * np.pi * X[:, 2]),
         lambda X: (np.abs(X[:, 1]) < 1e-12) | (np.abs(X[:, 1] - 1) < 1e-12))


@pytest.mark.parametrize("dim,p,ns,min_rate,problem", [
    (2, 1, [16, 32, 64, 128], 1.9, _SQUARE),
    (2, 2, [8, 16, 32, 64], 2.9, _SQUARE),
    (3, 2, [8, 16], 2.8, _CUBE)])
def test_poisson_convergence(dim, p, ns, min_rate, problem):
    """O(h^{p+1}) L2 convergence of Poisson to a manufactured solution (oracle + sparse solve);
    the observed rates over the finest two refinements must reach min_rate."""
    errs = [_poisson_l2_error(dim, p, n, problem) for n in ns]
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(len(errs) - 1)]
    assert min(rates[-2:]) >= min_rate, (errs, rates)
