"""Independent brute-force restatements used to pin the oracle on tiny inputs.

These use different algorithms from the oracle (reachability matrices instead
of Kahn + Tarjan, fixed-point relaxation instead of a topological pass, dense
LAPACK solves instead of ordered substitution) so that a mistake in either
shows up as a mismatch.
"""

import numpy as np


def face_dots(mesh, omega):
    n = mesh["normals"]
    return ((n[:, 0] * omega[0]) + (n[:, 1] * omega[1])) + (n[:, 2] * omega[2])


def edges(mesh, omega):
    """Active dependency edges (face, upwind, downwind) for one direction."""
    fc = mesh["face_cells"]
    d = face_dots(mesh, omega)
    out = []
    for f in range(mesh["n_faces"]):
        c0, c1 = fc[f]
        if c1 < 0 or d[f] == 0.0:
            continue
        out.append((f, c0, c1) if d[f] > 0 else (f, c1, c0))
    return out


def closure(n, edge_list):
    """Boolean reachability by paths of length >= 1 (repeated squaring)."""
    A = np.zeros((n, n), dtype=np.int64)
    for _, u, v in edge_list:
        A[u, v] = 1
    R = A.copy()
    while True:
        R2 = np.minimum(R + (R @ R > 0).astype(np.int64), 1)
        if np.array_equal(R2, R):
            return R.astype(bool)
        R = R2


def lag_rule(n, edge_list):
    """Apply the cycle rule by brute force; returns sorted lagged (face, up, down)."""
    active = list(edge_list)
    lagged = []
    while True:
        R = closure(n, active)
        on_cycle = np.diag(R)
        if not on_cycle.any():
            break
        same = R & R.T
        seen = np.zeros(n, dtype=bool)
        new = []
        for v in range(n):
            if seen[v] or not on_cycle[v]:
                continue
            comp = np.flatnonzero(same[v])
            comp = np.union1d(comp, [v])
            seen[comp] = True
            inside = [e for e in active if e[1] in comp and e[2] in comp]
            new.append(min(inside))
        for e in new:
            active.remove(e)
            lagged.append(e)
    return sorted(lagged), active


def relaxed_levels(n, edge_list):
    """Longest-path levels by fixed-point relaxation (Bellman-Ford style)."""
    lev = np.zeros(n, dtype=np.int64)
    for _ in range(n + 1):
        changed = False
        for _, u, v in edge_list:
            if lev[u] + 1 > lev[v]:
                lev[v] = lev[u] + 1
                changed = True
        if not changed:
            return lev
    raise AssertionError("relaxation did not settle: graph has a cycle")


def bface_index(mesh):
    fc = mesh["face_cells"]
    idx = -np.ones(mesh["n_faces"], dtype=np.int64)
    b = np.flatnonzero(fc[:, 1] < 0)
    idx[b] = np.arange(b.size)
    return idx


def transport_matrix(mesh, omega, sigma_t):
    """Step-scheme matrix of one direction with every face coupled implicitly.

    Row c: (sigma_t V + sum_out mu a) psi_c - sum_in |mu a| psi_up = S V + inflow
    terms; returns (A, B) where B maps boundary inflow values to the right-hand
    side (B[c, b] = |mu a| for an incoming boundary face b of c).
    """
    N = mesh["n_cells"]
    fc = mesh["face_cells"]
    d = face_dots(mesh, omega)
    a = mesh["areas"]
    bidx = bface_index(mesh)
    nb = int((fc[:, 1] < 0).sum())
    A = np.diag(sigma_t * mesh["volumes"]).astype(float)
    B = np.zeros((N, nb))
    for f in range(mesh["n_faces"]):
        c0, c1 = fc[f]
        for c, sgn in ((c0, 1.0), (c1, -1.0)):
            if c < 0:
                continue
            mu = sgn * d[f]
            if mu > 0:
                A[c, c] += mu * a[f]
            elif mu < 0:
                if c1 < 0:
                    B[c, bidx[f]] += -mu * a[f]
                else:
                    u = c1 if c == c0 else c0
                    A[c, u] -= -mu * a[f]
    return A, B


def si_fixed_point(mesh, dirs, weights, sigma_t, c_ratio, q, inflow=None):
    """Converged scalar flux of source iteration as one dense linear solve.

    phi = sum_m w_m A_m^{-1} (V (c sigma_t phi + q) / (4 pi) + B_m inflow)
    """
    N = mesh["n_cells"]
    V = mesh["volumes"]
    K = np.zeros((N, N))
    f = np.zeros(N)
    for m in range(dirs.shape[0]):
        A, B = transport_matrix(mesh, dirs[m], sigma_t)
        Ainv = np.linalg.inv(A)
        K += weights[m] * Ainv @ np.diag(V * c_ratio * sigma_t / (4 * np.pi))
        rhs = V * q / (4 * np.pi)
        if inflow is not None:
            rhs = rhs + B @ inflow
        f += weights[m] * Ainv @ rhs
    return np.linalg.solve(np.eye(N) - K, f)


def mg_fixed_point(mesh, dirs, weights, sigma_t, sigma_s, q, inflow=None):
    """Converged multigroup scalar flux as one dense block solve.

    phi_g = sum_m w_m A_{m,g}^{-1} (V (sum_h sigma_s[h, g] phi_h + q_g) / (4 pi)
                                     + B_m inflow_g)
    with A_{m,g} the step-scheme matrix of direction m for sigma_t[g].
    """
    N = mesh["n_cells"]
    G = sigma_t.shape[0]
    V = mesh["volumes"]
    K = np.zeros((G * N, G * N))
    f = np.zeros(G * N)
    for g in range(G):
        for m in range(dirs.shape[0]):
            A, B = transport_matrix(mesh, dirs[m], sigma_t[g])
            Ainv = np.linalg.inv(A)
            for h in range(G):
                K[g * N:(g + 1) * N, h * N:(h + 1) * N] += (
                    weights[m] * Ainv @ np.diag(V * sigma_s[h, g] / (4 * np.pi)))
            rhs = V * q[g] / (4 * np.pi)
            if inflow is not None:
                rhs = rhs + B @ inflow[g]
            f[g * N:(g + 1) * N] += weights[m] * Ainv @ rhs
    return np.linalg.solve(np.eye(G * N) - K, f).reshape(G, N)
