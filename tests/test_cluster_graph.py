"""Coarsened graph (Sec. V-E, Theorem 1), checked on the oracle's graphs.

A coarsened graph merges the vertices of a direction's dependency graph into
clusters and keeps one edge between two clusters wherever a vertex of one is
upwind of a vertex of the other.  Theorem 1: if the graph is acyclic, so is a
coarsened graph whose clusters were collected along a topological traversal.
The library's work units are such clusters: up to 32 consecutive cells of one
layer of a direction's level-major order, an interval of a topological order.
These tests rebuild each direction's active edges from the mesh (the face
signs, minus the faces the oracle lagged), take the oracle's order, cut it
into intervals (inside one level, and across levels), and check the cluster
graph by a topological sort.  The converse is shown too: clusters cut by
space (cubic patches of a jittered hex grid) give a cyclic cluster graph for
some grazing directions, which is why the sweeps cluster along the order.
"""

import numpy as np

import oracle
from inputs import hex_grid, kuhn_tets
from _bruteforce import edges

ODD = [0, 5, 37, 100, 143, 200, 250, 287]


def _active_edges(mesh, omega, lagged_faces):
    lag = set(int(f) for f in lagged_faces)
    return [(u, v) for f, u, v in edges(mesh, omega) if f not in lag]


def _acyclic(n, cedges):
    """Kahn's algorithm on the cluster graph: True when every node is removed."""
    indeg = np.zeros(n, dtype=np.int64)
    succ = [[] for _ in range(n)]
    for a, b in cedges:
        succ[a].append(b)
        indeg[b] += 1
    stack = [v for v in range(n) if indeg[v] == 0]
    seen = 0
    while stack:
        v = stack.pop()
        seen += 1
        for w in succ[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                stack.append(w)
    return seen == n


def _cluster_edges(cluster_of, act):
    return {(cluster_of[u], cluster_of[v]) for u, v in act if cluster_of[u] != cluster_of[v]}


def _interval_clusters(order, ptr, size, within_levels):
    """cluster id of every cell: intervals of `size` positions of the order,
    restarted at every level boundary when within_levels (the work units)."""
    n = len(order)
    pos_cluster = np.empty(n, dtype=np.int64)
    if within_levels:
        cid = 0
        for l in range(len(ptr) - 1):
            a, b = ptr[l], ptr[l + 1]
            k = np.arange(b - a)
            pos_cluster[a:b] = cid + k // size
            cid += (b - a + size - 1) // size
    else:
        pos_cluster[:] = np.arange(n) // size
    cluster_of = np.empty(n, dtype=np.int64)
    cluster_of[order] = pos_cluster
    return cluster_of, int(pos_cluster.max()) + 1


def test_interval_clusters_of_the_sweep_order_give_acyclic_cluster_graphs():
    dirs, _ = oracle.product_quadrature(6, 6)
    checked_cyclic = 0
    for mesh in (hex_grid(6, 0.3, 3), kuhn_tets(4, 0.2, 2)):
        o = oracle.build_dags(mesh, dirs)
        for m in ODD:
            lag = o.lagged(m)
            checked_cyclic += len(lag) > 0
            act = _active_edges(mesh, dirs[m], lag[:, 0] if len(lag) else [])
            order, ptr = o.order(m)
            # the order itself is topological for the active edges
            pos = np.empty(len(order), dtype=np.int64)
            pos[order] = np.arange(len(order))
            assert all(pos[u] < pos[v] for u, v in act)
            for size in (1, 3, 16, 32, 64):
                for within in (True, False):
                    cl, nc = _interval_clusters(order, ptr, size, within)
                    assert _acyclic(nc, _cluster_edges(cl, act)), (m, size, within)
    assert checked_cyclic > 0  # the meshes do have lagged faces in these directions


def test_breaking_the_order_breaks_the_theorem():
    # a planted mistake: clusters of alternate positions (not intervals) on a
    # graph with long dependency chains give a cyclic cluster graph
    dirs, _ = oracle.product_quadrature(6, 6)
    mesh = hex_grid(6, 0.3, 3)
    o = oracle.build_dags(mesh, dirs)
    lag = o.lagged(0)
    act = _active_edges(mesh, dirs[0], lag[:, 0] if len(lag) else [])
    order, _ = o.order(0)
    cl = np.empty(len(order), dtype=np.int64)
    cl[order] = np.arange(len(order)) % 2  # two clusters interleaved along the order
    assert not _acyclic(2, _cluster_edges(cl, act))


def test_spatial_patches_of_a_jittered_grid_can_be_cyclic():
    n, p = 8, 4
    mesh = hex_grid(n, 0.3, 5)
    dirs, _ = oracle.product_quadrature(6, 6)
    o = oracle.build_dags(mesh, dirs)
    ids = np.arange(n ** 3)
    i, j, k = ids % n, (ids // n) % n, ids // (n * n)
    patch = (i // p) + (n // p) * ((j // p) + (n // p) * (k // p))
    cyclic = 0
    for m in range(len(dirs)):
        lag = o.lagged(m)
        act = _active_edges(mesh, dirs[m], lag[:, 0] if len(lag) else [])
        cyclic += not _acyclic(int(patch.max()) + 1, _cluster_edges(patch, act))
    assert cyclic > 0
