"""Pins of the oracle's sweep and source iteration against closed forms,
invariants and dense linear solves."""

import math

import numpy as np
import pytest

import oracle
from inputs import column_mesh, hex_grid, kuhn_tets, pinwheel_mesh
from _bruteforce import si_fixed_point, transport_matrix


@pytest.mark.parametrize("mu", [1.0, 0.37, 0.05])
def test_1d_upwind_recurrence(mu):
    # N x 1 x 1 column, direction (mu, 0, 0): side faces carry no flux, and the
    # step scheme reduces to psi_i = (q dx + mu psi_{i-1}) / (sigma dx + mu).
    n = 40
    mesh = column_mesh(n, length=2.0, width=1.0)
    rng = np.random.default_rng(5)
    sig = rng.uniform(0.2, 3.0, n)
    q = rng.uniform(0.0, 2.0, n)
    psi_in = 0.7
    dx = 2.0 / n
    for sgn in (1.0, -1.0):
        g = oracle.build_dags(mesh, np.array([[sgn * mu, 0.0, 0.0]]))
        nb = g.n_bfaces
        inflow = np.full((1, nb), psi_in)
        phi, psi, _ = g.sweep(sig, q[None], np.array([1.0]), inflow=inflow, want_psi=True)
        ref = np.empty(n)
        prev = psi_in
        cells = range(n) if sgn > 0 else range(n - 1, -1, -1)
        for i in cells:
            prev = (q[i] * dx + mu * prev) / (sig[i] * dx + mu)
            ref[i] = prev
        assert np.max(np.abs(psi[0, 0] - ref) / np.abs(ref)) < 1e-13
        assert np.allclose(phi[0], psi[0, 0], rtol=0, atol=0)
        # levels are the cell positions along the sweep
        lev = g.levels(0)
        assert np.array_equal(lev, np.arange(n) if sgn > 0 else np.arange(n)[::-1])


@pytest.mark.parametrize("mesh_fn", [lambda: hex_grid(6, 0.3, 11), lambda: kuhn_tets(4, 0.2, 2)])
def test_uniform_solution_invariant(mesh_fn):
    # S = k sigma_t with isotropic inflow k gives psi = k in every cell and
    # direction on any closed-cell mesh (sum of outward vector areas is zero).
    mesh = mesh_fn()
    dirs, w = oracle.product_quadrature(6, 6)
    g = oracle.build_dags(mesh, dirs)
    rng = np.random.default_rng(1)
    sig = rng.lognormal(0.0, 1.0, mesh["n_cells"])
    k = np.array([1.0, 2.5])
    src = k[:, None] * sig[None, :]
    inflow = np.repeat(k[:, None], g.n_bfaces, axis=1)
    lag = np.repeat(k[:, None], g.n_lag_total, axis=1)
    phi, psi, lag_out = g.sweep(sig, src, w, inflow=inflow, psi_lag=lag, want_psi=True)
    for r in range(2):
        assert np.max(np.abs(psi[r] - k[r])) < 1e-13 * k[r]
        assert np.max(np.abs(phi[r] - 4 * math.pi * k[r])) < 1e-12 * k[r]
        if lag_out.size:
            assert np.max(np.abs(lag_out[r] - k[r])) < 1e-13 * k[r]


def test_single_sweep_equals_dense_solve_on_acyclic_mesh():
    mesh = kuhn_tets(2, 0.2, 4)
    dirs, w = oracle.product_quadrature(1, 3)
    g = oracle.build_dags(mesh, dirs)
    assert g.n_lag_total == 0
    rng = np.random.default_rng(2)
    N = mesh["n_cells"]
    sig = rng.uniform(0.5, 2.0, N)
    src = rng.uniform(0.0, 1.0, (2, N))
    inflow = rng.uniform(0.0, 1.0, (2, g.n_bfaces))
    phi, psi, _ = g.sweep(sig, src, w, inflow=inflow, want_psi=True)
    for m in range(dirs.shape[0]):
        A, B = transport_matrix(mesh, dirs[m], sig)
        for r in range(2):
            ref = np.linalg.solve(A, src[r] * mesh["volumes"] + B @ inflow[r])
            assert np.max(np.abs(psi[r, m] - ref) / np.abs(ref)) < 1e-12
    ref_phi = np.einsum("m,rmn->rn", w, psi)
    assert np.max(np.abs(phi - ref_phi)) < 1e-13 * np.abs(ref_phi).max()


def test_lagged_sweep_equals_dense_solve_with_lag_moved_to_rhs():
    # On the cyclic pinwheel, one sweep with given lagged values solves the
    # system whose lagged couplings are taken from psi_lag (right-hand side).
    mesh = pinwheel_mesh()
    dirs = np.array([[0.0, 0.0, 1.0], [0.1, -0.2, -0.97]])
    w = np.array([0.6, 0.4])
    g = oracle.build_dags(mesh, dirs)
    assert g.n_lag_total >= 2
    N = 4
    rng = np.random.default_rng(3)
    sig = rng.uniform(0.5, 2.0, N)
    src = rng.uniform(0.0, 1.0, (1, N))
    lag_in = rng.uniform(0.0, 1.0, (1, g.n_lag_total))
    inflow = rng.uniform(0.0, 1.0, (1, g.n_bfaces))
    phi, psi, lag_out = g.sweep(sig, src, w, inflow=inflow, psi_lag=lag_in, want_psi=True)
    j = 0
    for m in range(2):
        A, B = transport_matrix(mesh, dirs[m], sig)
        rhs = src[0] * mesh["volumes"] + B @ inflow[0]
        from _bruteforce import face_dots
        d = face_dots(mesh, dirs[m])
        for f, u, v in g.lagged(m).tolist():
            coef = abs(d[f]) * mesh["areas"][f]
            A[v, u] += coef  # remove the implicit coupling
            rhs[v] += coef * lag_in[0, j]
            j += 1
        ref = np.linalg.solve(A, rhs)
        assert np.max(np.abs(psi[0, m] - ref) / np.abs(ref)) < 1e-13
    # lagged values are replaced by this sweep's upwind psi
    j = 0
    for m in range(2):
        for f, u, v in g.lagged(m).tolist():
            assert lag_out[0, j] == psi[0, m, u]
            j += 1


@pytest.mark.parametrize("mesh_fn,cval", [(lambda: hex_grid(3, 0.3, 7), 0.5),
                                          (lambda: pinwheel_mesh(), 0.7),
                                          (lambda: kuhn_tets(2, 0.25, 1), 0.9)])
def test_source_iteration_matches_dense_fixed_point(mesh_fn, cval):
    mesh = mesh_fn()
    dirs, w = oracle.product_quadrature(1, 3)
    if mesh["n_cells"] == 4:
        # pinwheel: directions near +-z so that the cycles are present
        dirs = np.concatenate([dirs, [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]]])
        w = np.concatenate([w * 0.9, [0.2 * math.pi, 0.2 * math.pi]])
    g = oracle.build_dags(mesh, dirs)
    N = mesh["n_cells"]
    rng = np.random.default_rng(4)
    sig = rng.uniform(0.5, 2.0, N)
    c = np.full(N, cval)
    q = rng.uniform(0.0, 1.0, (1, N))
    inflow = rng.uniform(0.0, 0.2, (1, g.n_bfaces))
    tol = 1e-13
    phi, it, res, conv, hist = g.source_iterate(sig, c, q, w, tol, 5000, inflow=inflow)
    assert conv and res < tol
    ref = si_fixed_point(mesh, dirs, w, sig, c, q[0], inflow=inflow[0])
    err = np.max(np.abs(phi[0] - ref)) / np.max(np.abs(ref))
    assert err < 50 * tol * cval / (1 - cval) + 1e-13
    if mesh["n_cells"] == 4:
        assert g.n_lag_total > 0


@pytest.mark.parametrize("mesh_fn", [lambda: hex_grid(5, 0.3, 11), lambda: kuhn_tets(3, 0.2, 8)])
def test_source_iteration_infinite_medium_analogue(mesh_fn):
    # q = Phi sigma_t (1 - c) with isotropic inflow Phi / (4 pi): the fixed
    # point is phi = Phi everywhere (psi = Phi / (4 pi)).
    mesh = mesh_fn()
    dirs, w = oracle.product_quadrature(2, 3)
    g = oracle.build_dags(mesh, dirs)
    N = mesh["n_cells"]
    rng = np.random.default_rng(9)
    sig = rng.lognormal(0.0, 1.0, N)
    c = rng.uniform(0.0, 0.8, N)
    Phi = 3.0
    q = (Phi * sig * (1 - c))[None]
    inflow = np.full((1, g.n_bfaces), Phi / (4 * math.pi))
    phi, it, res, conv, hist = g.source_iterate(sig, c, q, w, 1e-13, 5000, inflow=inflow)
    assert conv
    assert np.max(np.abs(phi - Phi)) < 1e-11 * Phi


def test_source_iteration_reports_not_converged():
    mesh = hex_grid(3, 0.2, 1)
    dirs, w = oracle.product_quadrature(1, 3)
    g = oracle.build_dags(mesh, dirs)
    N = mesh["n_cells"]
    phi, it, res, conv, hist = g.source_iterate(np.ones(N), np.full(N, 0.9), np.ones((1, N)), w,
                                                1e-14, 3)
    assert not conv and it == 3 and res > 1e-14
    assert np.all(np.diff(hist) < 0)  # contraction from phi = 0
