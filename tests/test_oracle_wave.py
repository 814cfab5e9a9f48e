"""Pins of the oracle's explicit lumped-mass wave steps (CPU only).

* Without Dirichlet nodes the scheme acts on each eigenmode of the lumped-mass pencil
  K v = lam M_L v separately.  Writing the state as phi = a v, p = b v, one step is the 2x2 map
  a <- a - dt/2 b, b <- b + dt lam a, a <- a - dt/2 b (the half-step structure and the signs of
  the paper's scheme).  Starting from a mode, the oracle's vector state after N steps must equal
  that map's N-th power applied to (1, 0), with the modes from a dense eigensolver.
* A constant phi is a zero mode: nothing moves.
* With Dirichlet nodes, p equals sin(10 pi t) on them after every step, and the interior
  evolves (the forcing enters).
"""
import numpy as np

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg


def _setup(n, dim=2, jitter=0.2, seed=3):
    mesh = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n, jitter, seed)
    cmap, nn = mg.cell_node_map(mesh, 1)
    return mesh, cmap, nn


def _dense_pencil(mesh, cmap, nn, dim):
    rp, ci = O.sparsity(cmap, cmap, nn, nn)
    v, _ = O.assemble_mat(dim, 1, O.LAPLACE, cmap, mesh.coords, mesh.cell_vertex, rp, ci)
    K = np.zeros((nn, nn))
    for i in range(nn):
        K[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    m, _ = O.assemble_vec(dim, 1, 1, cmap, nn, mesh.coords, mesh.cell_vertex, np.ones(nn), cmap)
    return K, m


def pin_modes(n=5, dim=2, nsteps=40, dt=0.01):
    mesh, cmap, nn = _setup(n, dim)
    K, m = _dense_pencil(mesh, cmap, nn, dim)
    s = 1.0 / np.sqrt(m)
    lam, U = np.linalg.eigh(s[:, None] * K * s[None, :])
    for k in (1, nn // 2, nn - 1):
        vk = s * U[:, k]
        G = np.array([[1.0, -dt / 2], [0.0, 1.0]]) @ np.array([[1.0, 0.0], [dt * lam[k], 1.0]]) @ \
            np.array([[1.0, -dt / 2], [0.0, 1.0]])
        a, b = np.linalg.matrix_power(G, nsteps) @ np.array([1.0, 0.0])
        phi, p = O.wave_steps(dim, 1, cmap, mesh.coords, mesh.cell_vertex, nn, vk, np.zeros(nn), 0.0, dt, nsteps)
        scale = np.abs(vk).max()
        assert np.abs(phi - a * vk).max() <= 1e-10 * scale, (k, np.abs(phi - a * vk).max())
        assert np.abs(p - b * vk).max() <= 1e-10 * scale * max(1.0, np.sqrt(lam[k])), k


def test_modes_2d():
    pin_modes()


def test_modes_3d():
    pin_modes(2, dim=3, nsteps=25, dt=0.02)


def test_constant_is_at_rest():
    mesh, cmap, nn = _setup(6)
    phi, p = O.wave_steps(2, 1, cmap, mesh.coords, mesh.cell_vertex, nn, np.full(nn, 0.7), np.zeros(nn), 0.0, 0.01, 30)
    assert np.abs(phi - 0.7).max() <= 1e-13 and np.abs(p).max() <= 1e-12


def test_dirichlet_forcing():
    mesh, cmap, nn = _setup(8)
    bc = mg.face_nodes(mesh, 1, 1, 0)
    phi, p = np.zeros(nn), np.zeros(nn)
    dt = 0.003
    for k in range(5):
        phi, p = O.wave_steps(2, 1, cmap, mesh.coords, mesh.cell_vertex, nn, phi, p, k * dt, dt, 1, is_bc=bc)
        assert np.all(p[bc == 1] == np.sin(10 * np.pi * k * dt))
    assert np.abs(phi[bc == 0]).max() > 0 and np.abs(p[bc == 0]).max() > 0


def test_face_nodes():
    m = mg.unit_cube_mesh(2)
    X = mg.node_coordinates(m, 1)
    assert np.array_equal(mg.face_nodes(m, 1, 1, 0).astype(bool), np.abs(X[:, 1]) < 1e-12)
    assert np.array_equal(mg.face_nodes(m, 1, 2, 1).astype(bool), np.abs(X[:, 2] - 1) < 1e-12)
