"""The seeded input generators: sizes, determinism, boundary, orientation, node numbering."""
import numpy as np
import pytest

from paper_1501_01809_gb300 import meshgen as mg


def test_sizes_of_the_named_workloads():
    m = mg.unit_square_mesh(64)
    cm, nn = mg.cell_node_map(m, 1)
    assert (m.ncell, nn) == (8192, 4225)
    m = mg.unit_square_mesh(8)
    cm, nn = mg.cell_node_map(m, 4)
    assert cm.shape == (128, 15) and nn == 33 * 33
    m = mg.unit_cube_mesh(4, 0.2, 0)
    cm, nn = mg.cell_node_map(m, 2)
    assert cm.shape == (6 * 64, 10) and nn == 9 ** 3


def test_jitter_is_seeded_and_keeps_boundary():
    a = mg.unit_cube_mesh(5, 0.2, 0)
    b = mg.unit_cube_mesh(5, 0.2, 0)
    c = mg.unit_cube_mesh(5, 0.2, 1)
    np.testing.assert_array_equal(a.coords, b.coords)
    assert not np.array_equal(a.coords, c.coords)
    bnd = np.any((a.vgrid == 0) | (a.vgrid == 5), axis=1)
    np.testing.assert_array_equal(a.coords[bnd], a.vgrid[bnd] / 5.0)
    assert np.max(np.abs(a.coords - a.vgrid / 5.0)) <= 0.2 / 5 + 1e-15


def test_refuses_inverted_cells():
    with pytest.raises(ValueError):
        mg.unit_square_mesh(4, 0.9, 0)


def test_every_node_is_used_and_numbering_is_lexicographic():
    for dim, p, n in [(2, 1, 3), (2, 2, 3), (2, 4, 2), (3, 2, 2), (3, 3, 2)]:
        m = (mg.unit_square_mesh if dim == 2 else mg.unit_cube_mesh)(n)
        cm, nn = mg.cell_node_map(m, p)
        assert set(np.unique(cm).tolist()) == set(range(nn))
        X = mg.node_coordinates(m, p)
        g = np.rint(X * (p * n)).astype(np.int64)          # unjittered: fine-grid coordinates
        ids = g[:, 0] + (p * n + 1) * g[:, 1] + ((p * n + 1) ** 2 * g[:, 2] if dim == 3 else 0)
        np.testing.assert_array_equal(ids, np.arange(nn))
        assert all(len(set(row)) == len(row) for row in cm.tolist())  # no repeated node in a cell


def test_batch_sizes():
    n, p = mg.batch_mesh_sizes(2048, 4)
    assert n.min() >= 8 and n.max() <= 256 and set(p.tolist()) == {1, 2}
