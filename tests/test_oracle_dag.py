"""Pins of the oracle's dependency graphs: brute force, validity, a worked example."""

import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle
from inputs import hex_grid, kuhn_tets, pinwheel_mesh
from _bruteforce import edges, lag_rule, relaxed_levels

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pinwheel_worked_example():
    gold = json.load(open(os.path.join(HERE, "golden", "pinwheel.json")))
    mesh = pinwheel_mesh()
    for case in gold["cases"]:
        g = oracle.build_dags(mesh, np.array([case["omega"]]))
        assert g.lagged(0).tolist() == case["lagged"]
        assert g.levels(0).tolist() == case["levels"]
        order, ptr = g.order(0)
        assert order.tolist() == case["order"]
        assert ptr.tolist() == case["level_ptr"]


@pytest.mark.parametrize("kind,n,jit,seed", [("hex", 4, 0.3, 7), ("hex", 5, 0.3, 11), ("tet", 3, 0.3, 5)])
def test_bruteforce_lags_and_levels(kind, n, jit, seed):
    mesh = hex_grid(n, jit, seed) if kind == "hex" else kuhn_tets(n, jit, seed)
    dirs, _ = oracle.product_quadrature(6, 6)
    g = oracle.build_dags(mesh, dirs)
    N = mesh["n_cells"]
    n_cyclic = 0
    for m in range(dirs.shape[0]):
        e = edges(mesh, dirs[m])
        lag_bf, active = lag_rule(N, e)
        lag = [tuple(r) for r in g.lagged(m).tolist()]
        assert lag == lag_bf, f"direction {m}"
        n_cyclic += bool(lag)
        lev_bf = relaxed_levels(N, active)
        lev = g.levels(m)
        assert np.array_equal(lev, lev_bf), f"direction {m}"
        order, ptr = g.order(m)
        assert np.array_equal(order, np.lexsort((np.arange(N), lev)))
        assert ptr[0] == 0 and ptr[-1] == N and len(ptr) == lev.max() + 2
        assert np.array_equal(np.diff(ptr), np.bincount(lev))
    if kind == "hex":
        assert n_cyclic > 10  # these meshes are chosen to have cyclic directions


def test_acyclic_after_lagging_and_edge_validity():
    mesh = hex_grid(8, 0.25, 3)
    dirs, _ = oracle.product_quadrature(6, 6)
    g = oracle.build_dags(mesh, dirs)
    N = mesh["n_cells"]
    total = 0
    for m in range(0, dirs.shape[0], 5):
        lagged = {tuple(r) for r in g.lagged(m).tolist()}
        total += len(lagged)
        active = [e for e in edges(mesh, dirs[m]) if e not in lagged]
        G = sp.csr_matrix((np.ones(len(active)), ([e[1] for e in active], [e[2] for e in active])),
                          shape=(N, N))
        nc, _ = connected_components(G, directed=True, connection="strong")
        assert nc == N  # every component a single cell: acyclic
        lev = g.levels(m)
        for _, u, v in active:
            assert lev[u] < lev[v]
        # every lagged face joins two cells and was a real dependency
        for f, u, v in lagged:
            assert (f, u, v) in set(edges(mesh, dirs[m]))
    assert total > 0


def test_unjittered_grid_levels_are_manhattan():
    # Regular grid, direction in the (+,+,+) octant: level(i,j,k) = i + j + k.
    mesh = hex_grid(5, 0.0, 0)
    dirs, _ = oracle.product_quadrature(2, 3)
    g = oracle.build_dags(mesh, dirs[:6])
    i, j, k = np.meshgrid(np.arange(5), np.arange(5), np.arange(5), indexing="ij")
    ref = (i + j + k).transpose(2, 1, 0).ravel()  # cell id = i + 5 (j + 5 k)
    for m in range(6):
        assert np.array_equal(g.levels(m), ref)
        assert g.nlevels(m) == 13
