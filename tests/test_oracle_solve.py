"""Pins of the oracle's Dirichlet elimination and Jacobi-preconditioned CG (CPU only).

What fixes them independently of the oracle's own code:
* symmetric elimination of u = g must give the solution of the reduced system
  A_II x_I = b_I - A_IB g_B (dense slicing of the un-eliminated matrix, dense solve);
* P_p reproduces harmonic polynomials of degree <= p exactly: with f = 0 and g = u on the
  boundary, the discrete solution equals u at every node (Laplace assembly, elimination, CG);
* CG on a dense SPD system agrees with a dense LU solve within the conditioning bound;
* on a diagonal matrix Jacobi-CG converges in one iteration;
* the returned residual satisfies ||r|| <= rtol ||b|| and equals the true residual;
* manufactured sin(k pi x) sin(m pi y): O(h^2) (P1) and O(h^3) (P2) L2 convergence through the
  whole chain (oracle assembly + elimination + CG).
"""
import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg


def _poisson(n, p, jitter=0.0, seed=0, f=None):
    m = mg.unit_square_mesh(n, jitter, seed)
    cmap, nn = mg.cell_node_map(m, p)
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    v, _ = O.assemble_mat(2, p, O.LAPLACE, cmap, m.coords, m.cell_vertex, rp, ci)
    fv = np.zeros(nn) if f is None else f
    b, _ = O.assemble_vec(2, p, p, cmap, nn, m.coords, m.cell_vertex, fv, cmap)
    return m, cmap, nn, rp, ci, v, b


def _dense(rp, ci, v, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    return A


def pin_reduced_system(n=5, p=2):
    rng = np.random.default_rng(7)
    m, cmap, nn, rp, ci, v, b = _poisson(n, p, 0.2, 3, f=rng.uniform(-1, 1, (p * n + 1) ** 2))
    bc = mg.boundary_nodes(m, p)
    g = rng.uniform(-1, 1, nn)
    ve, be = O.dirichlet_apply(rp, ci, v, b, bc, g)
    A, Ae = _dense(rp, ci, v, nn), _dense(rp, ci, ve, nn)
    B, I = bc.astype(bool), ~bc.astype(bool)
    assert np.array_equal(Ae, Ae.T), "elimination must keep the matrix symmetric"
    assert np.array_equal(Ae[B], np.eye(nn)[B]), "boundary rows must be identity rows"
    x = np.linalg.solve(Ae, be)
    xr = np.zeros(nn)
    xr[B] = g[B]
    xr[I] = np.linalg.solve(A[np.ix_(I, I)], b[I] - A[np.ix_(I, B)] @ g[B])
    assert np.allclose(x, xr, rtol=0, atol=1e-12 * np.abs(xr).max()), np.abs(x - xr).max()


def pin_harmonic_reproduction(p, n=6):
    u = {1: lambda x, y: 1 + 2 * x - 3 * y,
         2: lambda x, y: x * x - y * y + 0.5 * x * y - x,
         3: lambda x, y: x ** 3 - 3 * x * y * y + y}[p]
    m, cmap, nn, rp, ci, v, b = _poisson(n, p, 0.25, 5)
    X = mg.node_coordinates(m, p)
    ue = u(X[:, 0], X[:, 1])
    bc = mg.boundary_nodes(m, p)
    ve, be = O.dirichlet_apply(rp, ci, v, b, bc, ue)
    x, it, rn, bn = O.cg_jacobi(rp, ci, ve, be, rtol=1e-14)
    assert it > 0
    assert np.abs(x - ue).max() <= 1e-11, (p, np.abs(x - ue).max())


def pin_cg_dense_spd(n=40):
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + np.diag(rng.uniform(1, 50, n))
    rp = np.arange(0, n * n + 1, n, dtype=np.int64)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    b = rng.standard_normal(n)
    x, it, rn, bn = O.cg_jacobi(rp, ci, A.ravel(), b, rtol=1e-14)
    xd = np.linalg.solve(A, b)
    bound = 2e-14 * np.linalg.norm(b) / np.linalg.eigvalsh(A)[0]
    assert it > 0 and np.linalg.norm(x - xd) <= bound, (np.linalg.norm(x - xd), bound)


def pin_cg_diagonal():
    d = np.array([1.0, 4.0, 9.0, 0.5, 3.0])
    rp = np.arange(6, dtype=np.int64)
    ci = np.arange(5, dtype=np.int32)
    b = np.array([2.0, -1.0, 3.0, 0.25, 1.0])
    x, it, rn, bn = O.cg_jacobi(rp, ci, d, b, rtol=1e-15)
    assert it == 1 and np.allclose(x, b / d, rtol=1e-15, atol=0)


def test_reduced_system():
    pin_reduced_system()
    pin_reduced_system(6, 1)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_harmonic_reproduction(p):
    pin_harmonic_reproduction(p)


def test_cg_dense_spd():
    pin_cg_dense_spd()


def test_cg_diagonal():
    pin_cg_diagonal()


def test_cg_residual_and_zero_rhs():
    m, cmap, nn, rp, ci, v, b = _poisson(16, 1, f=mg.manufactured_sine(mg.unit_square_mesh(16), 1, 2, 3)[0])
    ve, be = O.dirichlet_apply(rp, ci, v, b, mg.boundary_nodes(m, 1))
    x, it, rn, bn = O.cg_jacobi(rp, ci, ve, be, rtol=1e-8)
    A = _dense(rp, ci, ve, nn)
    true_r = np.linalg.norm(be - A @ x)
    assert rn <= 1e-8 * bn and abs(true_r - rn) <= 1e-3 * rn + 1e-14 * bn, (rn, true_r, bn)
    assert 0 < it < nn
    # zero right-hand side and zero guess: converged before the first iteration
    x0, it0, rn0, bn0 = O.cg_jacobi(rp, ci, ve, np.zeros(nn), rtol=1e-8)
    assert it0 == 0 and rn0 == 0 and not x0.any()
    # a matrix that is not SPD (negated) is reported
    assert O.cg_jacobi(rp, ci, -ve, be)[1] == -1


@pytest.mark.parametrize("p,ns,min_rate", [(1, [8, 16, 32, 64], 1.9), (2, [4, 8, 16, 32], 2.85)])
def test_sine_convergence_through_cg(p, ns, min_rate):
    errs = []
    for n in ns:
        mesh = mg.unit_square_mesh(n)
        f, u = mg.manufactured_sine(mesh, p, 1, 2)
        m, cmap, nn, rp, ci, v, b = _poisson(n, p, f=f)
        ve, be = O.dirichlet_apply(rp, ci, v, b, mg.boundary_nodes(m, p))
        x, it, rn, bn = O.cg_jacobi(rp, ci, ve, be, rtol=1e-12)
        xq, wq, uq = O.eval_function(2, p, 2 * p + 6, cmap, m.coords, m.cell_vertex, x)
        ue = np.sin(np.pi * xq[:, 0]) * np.sin(2 * np.pi * xq[:, 1])
        errs.append(np.sqrt(np.sum(wq * (uq - ue) ** 2)))
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(2) for i in range(len(errs) - 1)]
    assert min(rates[-2:]) >= min_rate, (errs, rates)


def test_boundary_nodes_and_requests():
    m = mg.unit_square_mesh(3)
    X = mg.node_coordinates(m, 2)
    want = np.any((np.abs(X) < 1e-12) | (np.abs(X - 1) < 1e-12), axis=1)
    assert np.array_equal(mg.boundary_nodes(m, 2).astype(bool), want)
    m3 = mg.unit_cube_mesh(2)
    X3 = mg.node_coordinates(m3, 1)
    want3 = np.any((np.abs(X3) < 1e-12) | (np.abs(X3 - 1) < 1e-12), axis=1)
    assert np.array_equal(mg.boundary_nodes(m3, 1).astype(bool), want3)
    reqs = mg.serve_requests(200, 1, rate=50.0)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) >= 0) and 2.0 < t[-1] < 6.0
    assert all(16 <= r[1] <= 512 and r[2] in (1, 2) and 1 <= r[3] <= 4 and 1 <= r[4] <= 4 for r in reqs)
