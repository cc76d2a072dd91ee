"""Seeded synthetic workloads shaped like the paper's benchmark problems.

The paper measures on the Kobayashi cube (structured, one group, scattering,
hundreds of directions) and on unstructured tetrahedral ball/reactor meshes
(S4, several groups).  Those inputs are not available; these generators
stand in for them with the shapes, sizes and value distributions below.

Seeds: mesh seed = workload number, material seed = 100 + workload number,
source seed for right-hand side r = 1000 * workload number + r.

Each workload dict holds the mesh arrays (see ``inputs.meshes``), the
material arrays ``sigma_t`` [N], ``c_ratio`` [N] (scattering ratio
sigma_s / sigma_t), the isotropic source ``q`` [R, N], and the product
quadrature shape ``(n_polar, n_azim)`` (the direction set itself is computed
by whoever runs the sweep).
"""

from __future__ import annotations


import numpy as np

from .meshes import hex_grid, kuhn_tets


def lognormal_blocks_sigma(centroids, rng, n_blocks=8, mu=0.0, s=1.0):
    """Piecewise-constant cross section over axis-aligned blocks.

    A background value and one value per block are drawn from
    lognormal(mu, s); each block has uniform random corners in the unit cube
    and is painted in order (a later block overwrites an earlier one); a cell
    belongs to a block when its centroid lies inside it.
    """
    n = centroids.shape[0]
    sig = np.full(n, rng.lognormal(mu, s))
    for _ in range(n_blocks):
        a = rng.uniform(0.0, 1.0, 3)
        b = rng.uniform(0.0, 1.0, 3)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        inside = np.all((centroids >= lo) & (centroids <= hi), axis=1)
        sig[inside] = rng.lognormal(mu, s)
    return sig


def _rhs(n_cells, n_rhs, wl_id):
    q = np.empty((n_rhs, n_cells))
    for r in range(n_rhs):
        q[r] = np.random.default_rng(1000 * wl_id + r).uniform(0.0, 1.0, n_cells)
    return q


WORKLOADS = {
    1: dict(name="hex16_fp64_si", kind="hex", n=16, jitter=0.15, quad=(3, 4), n_rhs=1,
            precision="f64", tol=1e-8),
    2: dict(name="tet48_fp32", kind="tet", n=48, jitter=0.20, quad=(4, 4), n_rhs=1,
            precision="f32", tol=1e-6),
    3: dict(name="hex128_fp32_r8", kind="hex", n=128, jitter=0.15, quad=(6, 6), n_rhs=8,
            precision="f32", tol=1e-6),
}


def make_workload(wl_id, n=None, n_rhs=None):
    """Build workload ``wl_id`` (1, 2 or 3); ``n`` / ``n_rhs`` override the size.

    1: hex n^3 (16), jitter +-0.15h, 3x4 quadrature (96 directions),
       sigma_t ~ U[0.5, 2], c = 0.5, q ~ U[0, 1], vacuum, FP64, tol 1e-8.
    2: tets 6 n^3 (n = 48), jitter +-0.2h, 4x4 quadrature (128 directions),
       sigma_t lognormal(0, 1) over 8 random blocks, c ~ U[0, 0.9], q ~ U[0, 1].
    3: hex n^3 (128), jitter +-0.15h, 6x6 quadrature (288 directions),
       sigma_t lognormal(0, 1) per cell, c = 0.8, 8 right-hand sides q ~ U[0, 1].
    """
    spec = dict(WORKLOADS[wl_id])
    if n is not None:
        spec["n"] = int(n)
    if n_rhs is not None:
        spec["n_rhs"] = int(n_rhs)
    if spec["kind"] == "hex":
        mesh = hex_grid(spec["n"], jitter=spec["jitter"], seed=wl_id)
    else:
        mesh = kuhn_tets(spec["n"], jitter=spec["jitter"], seed=wl_id)
    N = mesh["n_cells"]
    mrng = np.random.default_rng(100 + wl_id)
    if wl_id == 1:
        sigma_t = mrng.uniform(0.5, 2.0, N)
        c_ratio = np.full(N, 0.5)
    elif wl_id == 2:
        sigma_t = lognormal_blocks_sigma(mesh["centroids"], mrng)
        c_ratio = mrng.uniform(0.0, 0.9, N)
    else:
        sigma_t = mrng.lognormal(0.0, 1.0, N)
        c_ratio = np.full(N, 0.8)
    q = _rhs(N, spec["n_rhs"], wl_id)
    out = dict(mesh)
    out.update(spec=spec, sigma_t=sigma_t, c_ratio=c_ratio, q=q)
    return out


# product sets used by the batched and served workloads:
# directions 8*Np*Na in {24, 48, 96, 128, 288}
QUAD_BY_NDIRS = {24: (1, 3), 48: (2, 3), 96: (3, 4), 128: (4, 4), 288: (6, 6)}


def batch_problem_specs(n_problems=256, seed=4, ndirs_choices=(24, 96, 288),
                        lo=8, hi=40):
    """Sizes of a batch of independent tetrahedral problems.

    Hexahedron-equivalent edge n = round(lo * (hi/lo)**u), u ~ U[0, 1]
    (log-uniform between lo^3 and hi^3 hexahedra, 6 tets each); direction
    count drawn uniformly from ``ndirs_choices``.
    """
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, n_problems)
    ns = np.rint(lo * (hi / lo) ** u).astype(int)
    nd = rng.choice(np.array(ndirs_choices), n_problems)
    return [dict(n=int(a), ndirs=int(b), quad=QUAD_BY_NDIRS[int(b)], seed=10000 + i)
            for i, (a, b) in enumerate(zip(ns, nd))]


def make_batch_problem(spec):
    """One tetrahedral problem of a batch: materials drawn as in workload 1."""
    mesh = kuhn_tets(spec["n"], jitter=0.2, seed=spec["seed"])
    N = mesh["n_cells"]
    rng = np.random.default_rng(spec["seed"] + 1)
    out = dict(mesh)
    out.update(spec=dict(spec), sigma_t=rng.uniform(0.5, 2.0, N), c_ratio=np.full(N, 0.5),
               q=rng.uniform(0.0, 1.0, (1, N)))
    return out


def multigroup_materials(n_cells, n_groups=4, seed=0, upscatter=0.05):
    """Seeded multigroup cross sections of the shape of the paper's JSNT-U
    runs (4 energy groups): sigma_t [G, N] lognormal per group, growing with
    the group index (slower particles collide more), and an isotropic
    scattering matrix sigma_s [G, G, N] whose entry [g_from, g_to] is the
    rate from group g_from into group g_to.  Each group scatters a fraction
    0.3-0.8 of sigma_t, mostly into itself and the groups below it
    (downscatter), a fraction ``upscatter`` of it into the groups above; the
    outgoing scattering of a group stays below its sigma_t, so every group is
    subcritical on its own."""
    rng = np.random.default_rng(seed)
    G, N = n_groups, n_cells
    sigma_t = rng.lognormal(0.0, 0.5, (G, N)) * (1.0 + 0.5 * np.arange(G))[:, None]
    frac = rng.uniform(0.3, 0.8, (G, N))  # scattering fraction of each group
    shares = np.zeros((G, G, N))
    for g in range(G):
        for h in range(G):
            if h >= g:
                shares[g, h] = rng.uniform(0.5, 1.0, N) * (2.0 if h == g else 1.0)
            else:
                shares[g, h] = upscatter * rng.uniform(0.5, 1.0, N)
    shares /= shares.sum(axis=1, keepdims=True)
    sigma_s = shares * (frac * sigma_t)[:, None, :]
    return sigma_t, sigma_s


def tets_edge_for_cells(n_cells_target):
    """Edge n of a 6 n^3 Kuhn mesh closest to a target cell count."""
    return max(1, int(round((n_cells_target / 6.0) ** (1.0 / 3.0))))


__all__ = ["WORKLOADS", "make_workload", "lognormal_blocks_sigma", "batch_problem_specs",
           "make_batch_problem", "multigroup_materials", "tets_edge_for_cells", "QUAD_BY_NDIRS"]
