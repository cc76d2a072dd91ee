"""Seeded mesh generators: jittered hexahedral grids, Kuhn tetrahedra, small hand meshes.

Every generator returns a dict with the arrays that define a mesh for the sweep:

* ``n_cells`` N, ``n_faces`` F
* ``face_cells`` int64 [F, 2]: (cell0, cell1); cell1 = -1 marks a boundary face
* ``normals`` float64 [F, 3]: unit normal, pointing from cell0 into cell1
  (outward from cell0 on a boundary face)
* ``areas`` float64 [F]
* ``volumes`` float64 [N]
* ``centroids`` float64 [N, 3] (mean of the cell's nodes; used to paint materials)

The face id is the row index.  These are plain geometric inputs; the sweep
method (directions, upwind classification, dependency graph, solve) is not
here.
"""

from __future__ import annotations

import itertools

import numpy as np


def _finish(face_cells, avec, n_cells, cell_vol_terms, centroids):
    areas = np.sqrt(np.einsum("fi,fi->f", avec, avec))
    if np.any(areas <= 0):
        raise ValueError("degenerate face with zero area")
    normals = avec / areas[:, None]
    return {
        "n_cells": int(n_cells),
        "n_faces": int(face_cells.shape[0]),
        "face_cells": np.ascontiguousarray(face_cells, dtype=np.int64),
        "normals": np.ascontiguousarray(normals, dtype=np.float64),
        "areas": np.ascontiguousarray(areas, dtype=np.float64),
        "volumes": np.ascontiguousarray(cell_vol_terms, dtype=np.float64),
        "centroids": np.ascontiguousarray(centroids, dtype=np.float64),
    }


def _jittered_nodes(shape, lengths, jitter, rng):
    nx, ny, nz = shape
    lx, ly, lz = lengths
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    # nodes[k, j, i, :] so that a flat index is i + (nx+1)*(j + (ny+1)*k)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    nodes = np.stack([X, Y, Z], axis=-1)
    if jitter > 0.0:
        h = np.array([lx / nx, ly / ny, lz / nz])
        d = rng.uniform(-1.0, 1.0, size=nodes.shape) * (jitter * h)
        interior = np.zeros(nodes.shape[:3], dtype=bool)
        interior[1:-1, 1:-1, 1:-1] = True
        # boundary nodes stay fixed so the domain stays the box
        nodes = nodes + d * interior[..., None]
    return nodes


def _quad_avec(p0, p1, p2, p3):
    """Vector area of the bilinear surface spanning the loop p0-p1-p2-p3.

    Half the cross product of the diagonals; exact for any surface bounded by
    the four straight edges, so the six faces of a hexahedron sum to zero.
    """
    return 0.5 * np.cross(p2 - p0, p3 - p1)


def hex_grid(n=None, jitter=0.0, seed=0, shape=None, lengths=(1.0, 1.0, 1.0)):
    """Hexahedral grid on a box, interior nodes jittered by +-jitter*h per axis.

    Cell (i, j, k) has id ``i + nx*(j + ny*k)``.  Face ids: interior x-faces,
    then interior y-faces, then interior z-faces (each with i fastest, then j,
    then k), then boundary faces in the order x-, x+, y-, y+, z-, z+ (each
    with the in-plane index of smallest stride fastest).  Cell volumes are
    (1/3) sum_f xbar_f . A_f over the outward vector areas, so that the cell
    volumes of the box sum to its volume.
    """
    if shape is None:
        shape = (n, n, n)
    nx, ny, nz = (int(s) for s in shape)
    rng = np.random.default_rng(seed)
    P = _jittered_nodes((nx, ny, nz), lengths, jitter, rng)  # [nz+1, ny+1, nx+1, 3]

    def cid(i, j, k):
        return i + nx * (j + ny * k)

    fc_list, av_list, xb_list = [], [], []

    # interior x-faces at node plane i = 1..nx-1
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(1, nx), indexing="ij")
    k, j, i = k.ravel(), j.ravel(), i.ravel()
    p0, p1, p2, p3 = P[k, j, i], P[k, j + 1, i], P[k + 1, j + 1, i], P[k + 1, j, i]
    fc_list.append(np.stack([cid(i - 1, j, k), cid(i, j, k)], 1))
    av_list.append(_quad_avec(p0, p1, p2, p3))
    xb_list.append(0.25 * (p0 + p1 + p2 + p3))
    # interior y-faces at node plane j = 1..ny-1
    k, j, i = np.meshgrid(np.arange(nz), np.arange(1, ny), np.arange(nx), indexing="ij")
    k, j, i = k.ravel(), j.ravel(), i.ravel()
    p0, p1, p2, p3 = P[k, j, i], P[k + 1, j, i], P[k + 1, j, i + 1], P[k, j, i + 1]
    fc_list.append(np.stack([cid(i, j - 1, k), cid(i, j, k)], 1))
    av_list.append(_quad_avec(p0, p1, p2, p3))
    xb_list.append(0.25 * (p0 + p1 + p2 + p3))
    # interior z-faces at node plane k = 1..nz-1
    k, j, i = np.meshgrid(np.arange(1, nz), np.arange(ny), np.arange(nx), indexing="ij")
    k, j, i = k.ravel(), j.ravel(), i.ravel()
    p0, p1, p2, p3 = P[k, j, i], P[k, j, i + 1], P[k, j + 1, i + 1], P[k, j + 1, i]
    fc_list.append(np.stack([cid(i, j, k - 1), cid(i, j, k)], 1))
    av_list.append(_quad_avec(p0, p1, p2, p3))
    xb_list.append(0.25 * (p0 + p1 + p2 + p3))

    # boundary faces: x- and x+
    for plane, cell_i, sgn in ((0, 0, -1.0), (nx, nx - 1, 1.0)):
        k, j = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
        k, j = k.ravel(), j.ravel()
        i = np.full_like(j, plane)
        p0, p1, p2, p3 = P[k, j, i], P[k, j + 1, i], P[k + 1, j + 1, i], P[k + 1, j, i]
        fc_list.append(np.stack([cid(np.full_like(j, cell_i), j, k), -np.ones_like(j)], 1))
        av_list.append(sgn * _quad_avec(p0, p1, p2, p3))
        xb_list.append(0.25 * (p0 + p1 + p2 + p3))
    for plane, cell_j, sgn in ((0, 0, -1.0), (ny, ny - 1, 1.0)):
        k, i = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        k, i = k.ravel(), i.ravel()
        j = np.full_like(i, plane)
        p0, p1, p2, p3 = P[k, j, i], P[k + 1, j, i], P[k + 1, j, i + 1], P[k, j, i + 1]
        fc_list.append(np.stack([cid(i, np.full_like(i, cell_j), k), -np.ones_like(i)], 1))
        av_list.append(sgn * _quad_avec(p0, p1, p2, p3))
        xb_list.append(0.25 * (p0 + p1 + p2 + p3))
    for plane, cell_k, sgn in ((0, 0, -1.0), (nz, nz - 1, 1.0)):
        j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        j, i = j.ravel(), i.ravel()
        k = np.full_like(i, plane)
        p0, p1, p2, p3 = P[k, j, i], P[k, j, i + 1], P[k, j + 1, i + 1], P[k, j + 1, i]
        fc_list.append(np.stack([cid(i, j, np.full_like(i, cell_k)), -np.ones_like(i)], 1))
        av_list.append(sgn * _quad_avec(p0, p1, p2, p3))
        xb_list.append(0.25 * (p0 + p1 + p2 + p3))

    face_cells = np.concatenate(fc_list).astype(np.int64)
    avec = np.concatenate(av_list)
    xbar = np.concatenate(xb_list)
    n_cells = nx * ny * nz

    t = np.einsum("fi,fi->f", xbar, avec) / 3.0
    vol = np.bincount(face_cells[:, 0], weights=t, minlength=n_cells)
    inner = face_cells[:, 1] >= 0
    vol -= np.bincount(face_cells[inner, 1], weights=t[inner], minlength=n_cells)
    if np.any(vol <= 0):
        raise ValueError("inverted hexahedron: jitter too large")

    cen = np.zeros((n_cells, 3))
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                cen += P[dk:dk + nz, dj:dj + ny, di:di + nx].reshape(-1, 3)
    cen /= 8.0
    return _finish(face_cells, avec, n_cells, vol, cen)


_KUHN_PERMS = list(itertools.permutations(range(3)))


def kuhn_tets(n=None, jitter=0.0, seed=0, shape=None):
    """Jittered hexahedral grid, each hexahedron split into 6 Kuhn tetrahedra.

    The split follows the diagonal from the hexahedron's corner (0,0,0) to
    (1,1,1): for the p-th permutation (itertools order) of the axes, the tet
    walks v000 -> +e[p0] -> +e[p1] -> v111.  Tet id = 6*hex_id + p.  Local face
    q of a tet is the triangle opposite its vertex q.  Face ids follow the
    first occurrence when scanning (tet id, q) in increasing order; the tet of
    the first occurrence is cell0, the other one (if any) cell1.
    """
    if shape is None:
        shape = (n, n, n)
    nx, ny, nz = (int(s) for s in shape)
    rng = np.random.default_rng(seed)
    P = _jittered_nodes((nx, ny, nz), (1.0, 1.0, 1.0), jitter, rng).reshape(-1, 3)

    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k, j, i = k.ravel(), j.ravel(), i.ravel()
    n_hex = nx * ny * nz
    corner = np.empty((n_hex, 8), dtype=np.int64)
    for b in range(8):
        corner[:, b] = nid(i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1))
    tets = np.empty((n_hex, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_KUHN_PERMS):
        b1 = 1 << perm[0]
        b2 = b1 | (1 << perm[1])
        tets[:, p, 0] = corner[:, 0]
        tets[:, p, 1] = corner[:, b1]
        tets[:, p, 2] = corner[:, b2]
        tets[:, p, 3] = corner[:, 7]
    tets = tets.reshape(-1, 4)
    n_cells = tets.shape[0]

    x = P[tets]  # [T, 4, 3]
    det = np.einsum("ti,ti->t", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])
    # reference orientation from the unjittered split
    ref_sign = np.array([np.sign(np.linalg.det(np.array(
        [[1.0 if a == perm[0] else 0.0 for a in range(3)],
         [1.0 if a in perm[:2] else 0.0 for a in range(3)],
         [1.0, 1.0, 1.0]]))) for perm in _KUHN_PERMS])
    if np.any(det * np.tile(ref_sign, n_hex) <= 0):
        raise ValueError("inverted tetrahedron: jitter too large")

    # faces: local face q is opposite vertex q
    opp = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tri = tets[:, opp]  # [T, 4, 3]
    key_nodes = np.sort(tri, axis=2).reshape(-1, 3)
    nn = np.int64(P.shape[0])
    key = (key_nodes[:, 0] * nn + key_nodes[:, 1]) * nn + key_nodes[:, 2]
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    # face ids in first-occurrence order
    order = np.argsort(first, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    fid_of_slot = rank[inv]  # face id of each (tet, q) slot
    n_faces = uniq.size
    slot = np.arange(key.size)
    face_cells = -np.ones((n_faces, 2), dtype=np.int64)
    first_slot = first[order]  # slot of first occurrence per face id
    face_cells[:, 0] = first_slot // 4
    is_second = slot != first[inv]
    face_cells[fid_of_slot[is_second], 1] = slot[is_second] // 4
    # vector area of each face from its first occurrence, oriented away
    # from the opposite vertex of cell0
    t0 = first_slot // 4
    q0 = first_slot % 4
    a = P[tets[t0, opp[q0, 0]]]
    b = P[tets[t0, opp[q0, 1]]]
    c = P[tets[t0, opp[q0, 2]]]
    avec = 0.5 * np.cross(b - a, c - a)
    xopp = P[tets[t0, q0]]
    flip = np.einsum("fi,fi->f", avec, xopp - a) > 0
    avec[flip] *= -1.0
    xbar = (a + b + c) / 3.0

    t = np.einsum("fi,fi->f", xbar, avec) / 3.0
    vol = np.bincount(face_cells[:, 0], weights=t, minlength=n_cells)
    inner = face_cells[:, 1] >= 0
    vol -= np.bincount(face_cells[inner, 1], weights=t[inner], minlength=n_cells)
    if np.any(vol <= 0):
        raise ValueError("non-positive tetrahedron volume")
    cen = x.mean(axis=1)
    return _finish(face_cells, avec, n_cells, vol, cen)


def column_mesh(n_cells, length=1.0, width=1.0):
    """Unjittered n x 1 x 1 column of hexahedra along x (a 1D slab of cells)."""
    return hex_grid(shape=(n_cells, 1, 1), lengths=(length, width, width))


def pinwheel_mesh():
    """Four polyhedral cells whose dependency graph for Omega = +-z is cyclic.

    Interior faces (id: cell0 -> cell1), normals tilted around +z so that
    Omega = (0,0,1) sees flow from cell0 to cell1 on every one of them:
      f0: 0 -> 1,  f1: 1 -> 2,  f2: 2 -> 0,  f3: 2 -> 3,  f4: 3 -> 1.
    The graph holds the cycles 0-1-2-0 and 1-2-3-1 (one strongly connected
    component {0,1,2,3}).  Each cell is closed by one boundary face (ids 5..8)
    whose vector area is minus the sum of its other outward vector areas.
    The cells are abstract closed polyhedra (a valid input for the sweep),
    not a conforming geometric tiling.
    """
    inner = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 1)]
    tilt = np.array([
        [0.30, -0.10, 1.0],
        [-0.20, 0.25, 1.0],
        [0.15, 0.35, 1.0],
        [-0.40, -0.05, 1.0],
        [0.05, -0.30, 1.0],
    ])
    area_in = np.array([1.0, 0.8, 1.2, 0.9, 1.1])
    avec_in = tilt / np.linalg.norm(tilt, axis=1)[:, None] * area_in[:, None]
    n_cells = 4
    net = np.zeros((n_cells, 3))
    for f, (c0, c1) in enumerate(inner):
        net[c0] += avec_in[f]
        net[c1] -= avec_in[f]
    avec_b = -net
    face_cells = np.array(inner + [(c, -1) for c in range(n_cells)], dtype=np.int64)
    avec = np.concatenate([avec_in, avec_b])
    vol = np.array([1.0, 1.5, 0.75, 1.25])
    cen = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    return _finish(face_cells, avec, n_cells, vol, cen)
