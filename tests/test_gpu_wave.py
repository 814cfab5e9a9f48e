"""Explicit lumped-mass wave steps on the GPU vs the CPU oracle (runs on the GB300 machine).

The scheme is stable at these time steps (dt below 2 / sqrt(lambda_max) of the lumped-mass
pencil), so per-step rounding differences between the two implementations (below 1e-14 of the
state's size per step in FP64, below 2^-44 in double-float) grow at most linearly: after 40 steps
they stay below 1e-11 of the state; the bound checked is 1e-10 of max |phi| + max |p|.  Same
inputs on both sides: a jittered P1 mesh, random initial phi and p, Dirichlet forcing on y = 0.
"""
import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    return torch


def _run_gpu(torch, dim, mesh, cmap, nn, phi0, p0, bc, t0, dt, nsteps, prec):
    from paper_1501_01809_gb300 import fe
    dev = torch.device("cuda", 0)
    ctx = fe.ctx_create(0)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
         dict(map=cmap, cv=mesh.cell_vertex, xy=mesh.coords, phi=phi0, p=p0, bc=bc, one=np.ones(nn)).items()}
    mass = torch.zeros(nn, dtype=torch.float64, device=dev)
    cells, nodes, verts = fe.set_create(ctx, mesh.ncell), fe.set_create(ctx, nn), fe.set_create(ctx, mesh.nvert)
    M, CM = fe.map_create(ctx, cells, nodes, t["map"]), fe.map_create(ctx, cells, verts, t["cv"])
    XY = fe.dat_create(ctx, verts, t["xy"])
    PHI, P = fe.dat_create(ctx, nodes, t["phi"]), fe.dat_create(ctx, nodes, t["p"])
    ONE, MASS = fe.dat_create(ctx, nodes, t["one"]), fe.dat_create(ctx, nodes, mass)
    sp = fe.sparsity_build(ctx, M, M)
    ks = fe.kernel_create(ctx, fe.FORM_SOURCE, dim, 1, coeff_degree=1, strategy=fe.STRATEGY_PULL)
    fe.assemble_vec(ctx, ks, cells, MASS, M, XY, CM, [(ONE, M)], zero_first=True, sp=sp)  # deterministic
    kl = fe.kernel_create(ctx, fe.FORM_LAPLACE, dim, 1, precision=prec)
    fe.wave_steps(ctx, kl, cells, PHI, P, mass, t["bc"], M, XY, CM, sp, t0, dt, nsteps)
    fe.sync(ctx)
    return t["phi"].cpu().numpy(), t["p"].cpu().numpy()


@pytest.mark.parametrize("dim,n,prec", [(2, 33, 0), (3, 7, 0), (2, 33, 1), (3, 7, 1)])
def test_wave_matches_oracle(gpu, dim, n, prec):
    mesh = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n, 0.2, 5)
    cmap, nn = mg.cell_node_map(mesh, 1)
    rng = np.random.default_rng(9)
    phi0, p0 = rng.uniform(-1, 1, nn), rng.uniform(-1, 1, nn)
    bc = mg.face_nodes(mesh, 1, 1, 0)
    t0, dt, nsteps = 0.01, 0.002, 40
    phi_g, p_g = _run_gpu(gpu, dim, mesh, cmap, nn, phi0, p0, bc, t0, dt, nsteps, prec)
    phi_o, p_o = O.wave_steps(dim, 1, cmap, mesh.coords, mesh.cell_vertex, nn, phi0, p0, t0, dt, nsteps, is_bc=bc)
    scale = np.abs(phi_o).max() + np.abs(p_o).max()
    assert np.abs(phi_g - phi_o).max() <= 1e-10 * scale, np.abs(phi_g - phi_o).max() / scale
    assert np.abs(p_g - p_o).max() <= 1e-10 * scale, np.abs(p_g - p_o).max() / scale
    np.testing.assert_array_equal(p_g[bc == 1], p_o[bc == 1])  # the same host sin on both sides


def test_wave_is_deterministic_and_splits(gpu):
    """Bitwise equal on repeat; 30 steps equal 10 + 20 steps within the rounding bound (the merged
    half steps are split at the call boundary)."""
    mesh = mg.unit_cube_mesh(6, 0.2, 1)
    cmap, nn = mg.cell_node_map(mesh, 1)
    rng = np.random.default_rng(2)
    phi0, p0 = rng.uniform(-1, 1, nn), rng.uniform(-1, 1, nn)
    bc = mg.face_nodes(mesh, 1, 1, 0)
    a = _run_gpu(gpu, 3, mesh, cmap, nn, phi0, p0, bc, 0.0, 0.002, 30, 0)
    b = _run_gpu(gpu, 3, mesh, cmap, nn, phi0, p0, bc, 0.0, 0.002, 30, 0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    c1 = _run_gpu(gpu, 3, mesh, cmap, nn, phi0, p0, bc, 0.0, 0.002, 10, 0)
    c = _run_gpu(gpu, 3, mesh, cmap, nn, c1[0], c1[1], bc, 0.02, 0.002, 20, 0)
    scale = np.abs(a[0]).max() + np.abs(a[1]).max()
    assert np.abs(c[0] - a[0]).max() <= 1e-12 * scale and np.abs(c[1] - a[1]).max() <= 1e-12 * scale
