"""The synthetic meshes' geometry: every cell is closed (its outward vector
areas sum to zero), normals are unit vectors, volumes are positive and fill
the unit cube.  Closure is what the step scheme's uniform-solution invariant
rests on, so a generator mistake (a flipped or dropped face) shows here first."""

import numpy as np
import pytest

from inputs import column_mesh, hex_grid, kuhn_tets


def _closure(mesh):
    fc = np.asarray(mesh["face_cells"])
    a = np.asarray(mesh["areas"])[:, None] * np.asarray(mesh["normals"])
    n = mesh["n_cells"]
    acc = np.zeros((n, 3))
    area = np.zeros(n)
    np.add.at(acc, fc[:, 0], a)
    np.add.at(area, fc[:, 0], np.asarray(mesh["areas"]))
    inner = fc[:, 1] >= 0
    np.add.at(acc, fc[inner, 1], -a[inner])
    np.add.at(area, fc[inner, 1], np.asarray(mesh["areas"])[inner])
    return np.linalg.norm(acc, axis=1), area


@pytest.mark.parametrize("mesh_fn", [
    lambda: hex_grid(6, 0.3, 5),
    lambda: hex_grid(jitter=0.2, seed=9, shape=(30, 5, 4)),
    lambda: kuhn_tets(5, 0.2, 2),
    lambda: column_mesh(40),
])
def test_cells_close_and_fill_the_unit_cube(mesh_fn):
    mesh = mesh_fn()
    res, area = _closure(mesh)
    assert np.all(res <= 1e-14 * area)
    assert np.allclose(np.linalg.norm(np.asarray(mesh["normals"]), axis=1), 1.0, rtol=0, atol=1e-14)
    vol = np.asarray(mesh["volumes"])
    assert vol.min() > 0
    assert abs(vol.sum() - 1.0) < 1e-12


def test_closure_check_catches_a_flipped_face():
    mesh = dict(hex_grid(4, 0.2, 1))
    normals = np.array(mesh["normals"], copy=True)
    normals[7] = -normals[7]
    mesh["normals"] = normals
    res, area = _closure(mesh)
    assert np.any(res > 1e-6 * area)
