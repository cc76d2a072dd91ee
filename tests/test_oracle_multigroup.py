"""Pins of the oracle's multigroup source iteration (energy groups riding the
right-hand-side dimension of a sweep): reduction to one group, uncoupled
groups, an infinite-medium fixed point with upscatter, and a dense block
solve on a cyclic mesh."""

import math

import numpy as np
import pytest

import oracle
from inputs import hex_grid, kuhn_tets, multigroup_materials, pinwheel_mesh
from _bruteforce import mg_fixed_point


def _dags(mesh, quad=(1, 3)):
    dirs, w = oracle.product_quadrature(*quad)
    return oracle.build_dags(mesh, dirs), dirs, w


def test_one_group_is_single_group_source_iteration():
    mesh = hex_grid(4, 0.3, 5)
    g, dirs, w = _dags(mesh)
    N = mesh["n_cells"]
    rng = np.random.default_rng(31)
    sig = rng.uniform(0.5, 2.0, N)
    c = rng.uniform(0.2, 0.8, N)
    q = rng.uniform(0.0, 1.0, (1, N))
    inflow = rng.uniform(0.0, 0.3, (1, g.n_bfaces))
    ref, it_ref, _, conv_ref, _ = g.source_iterate(sig, c, q, w, 1e-12, 500, inflow=inflow)
    phi, it, _, conv, _ = g.multigroup_source_iterate(sig[None], (c * sig)[None, None], q, w, 1e-12, 500,
                                                       inflow=inflow)
    assert conv and conv_ref
    assert abs(it - it_ref) <= 1
    assert np.max(np.abs(phi - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_uncoupled_groups_are_independent_solves():
    mesh = kuhn_tets(3, 0.2, 6)
    g, dirs, w = _dags(mesh)
    N, G = mesh["n_cells"], 3
    sig, ss = multigroup_materials(N, G, seed=7)
    ss = ss * np.eye(G)[:, :, None]  # self-scattering only
    q = np.random.default_rng(32).uniform(0.0, 1.0, (G, N))
    phi, it, _, conv, _ = g.multigroup_source_iterate(sig, ss, q, w, 1e-12, 1000)
    assert conv
    for k in range(G):
        ref, _, _, ok, _ = g.source_iterate(sig[k], ss[k, k] / sig[k], q[k:k + 1], w, 1e-12, 1000)
        assert ok
        assert np.max(np.abs(phi[k] - ref[0])) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("mesh_fn", [lambda: hex_grid(4, 0.3, 12), lambda: kuhn_tets(3, 0.2, 9)])
def test_infinite_medium_fixed_point_with_upscatter(mesh_fn):
    # With isotropic inflow Phi_g / (4 pi) and q_g = sigma_t,g Phi_g - sum_h
    # sigma_s[h, g] Phi_h the fixed point is phi_g = Phi_g in every cell; the
    # scattering matrix is not symmetric and has upscatter, so a transposed
    # matrix (rate into h read as rate out of h) misses it.
    mesh = mesh_fn()
    g, dirs, w = _dags(mesh, (2, 3))
    N, G = mesh["n_cells"], 4
    sig, ss = multigroup_materials(N, G, seed=13, upscatter=0.2)
    Phi = np.array([1.0, 2.5, 0.7, 4.0])
    q = sig * Phi[:, None] - np.einsum("hgn,h->gn", ss, Phi)  # may be negative: the problem is linear
    inflow = np.repeat(Phi[:, None] / (4 * math.pi), g.n_bfaces, axis=1)
    phi, it, _, conv, _ = g.multigroup_source_iterate(sig, ss, q, w, 1e-13, 5000, inflow=inflow)
    assert conv
    assert np.max(np.abs(phi - Phi[:, None])) < 1e-10 * Phi.max()
    # the planted mistake: the transposed scattering matrix has another fixed point
    phi_t, _, _, conv_t, _ = g.multigroup_source_iterate(sig, ss.transpose(1, 0, 2), q, w, 1e-13, 5000,
                                                         inflow=inflow)
    assert conv_t and np.max(np.abs(phi_t - Phi[:, None])) > 1e-3


@pytest.mark.parametrize("mesh_fn", [lambda: hex_grid(3, 0.3, 7), lambda: pinwheel_mesh()])
def test_converged_multigroup_equals_dense_block_solve(mesh_fn):
    mesh = mesh_fn()
    dirs, w = oracle.product_quadrature(1, 3)
    if mesh["n_cells"] == 4:
        # pinwheel: directions near +-z so that the cycles (lagged faces) are present
        dirs = np.concatenate([dirs, [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]]])
        w = np.concatenate([w * 0.9, [0.2 * math.pi, 0.2 * math.pi]])
    g = oracle.build_dags(mesh, dirs)
    N, G = mesh["n_cells"], 3
    sig, ss = multigroup_materials(N, G, seed=17, upscatter=0.1)
    rng = np.random.default_rng(33)
    q = rng.uniform(0.0, 1.0, (G, N))
    inflow = rng.uniform(0.0, 0.2, (G, g.n_bfaces))
    tol = 1e-13
    phi, it, res, conv, hist = g.multigroup_source_iterate(sig, ss, q, w, tol, 5000, inflow=inflow)
    assert conv and res < tol
    ref = mg_fixed_point(mesh, dirs, w, sig, ss, q, inflow=inflow)
    # the largest scattering ratio (0.8) bounds the contraction of the iteration
    assert np.max(np.abs(phi - ref)) / np.max(np.abs(ref)) < 50 * tol * 0.8 / 0.2 + 1e-13
    if mesh["n_cells"] == 4:
        assert g.n_lag_total > 0
    assert np.all(np.diff(hist[:5]) < 0)  # contraction from phi = 0


def test_multigroup_materials_are_seeded_and_subcritical_per_group():
    sig, ss = multigroup_materials(500, 4, seed=3, upscatter=0.1)
    sig2, ss2 = multigroup_materials(500, 4, seed=3, upscatter=0.1)
    assert np.array_equal(sig, sig2) and np.array_equal(ss, ss2)
    assert sig.shape == (4, 500) and ss.shape == (4, 4, 500)
    assert np.all(sig > 0) and np.all(ss >= 0)
    out = ss.sum(axis=1)  # all scattering out of each group
    assert np.all(out < sig) and np.all(out >= 0.3 * sig - 1e-12)
    # mostly downscatter: each group sends less to the groups above it than to itself and below
    for g in range(4):
        assert np.all(ss[g, :g].sum(axis=0) < ss[g, g:].sum(axis=0))
