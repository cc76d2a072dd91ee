"""The serving loop on the GPU: continuously batched requests give each
request the same result as solving it alone, within the memory budget."""

import numpy as np
import pytest

import oracle
from inputs import hex_grid, kuhn_tets
from _gpu import J

pytestmark = pytest.mark.gpu

CATALOG = {
    "tet4_24": (lambda: kuhn_tets(4, 0.2, 31), (1, 3)),
    "tet6_128": (lambda: kuhn_tets(6, 0.2, 32), (4, 4)),
    "hex8_48": (lambda: hex_grid(8, 0.3, 33), (2, 3)),  # cyclic: lagged faces
    "tet24_128": (lambda: kuhn_tets(24, 0.2, 34), (4, 4)),  # 82,944 cells: the per-(direction, cell) term dominates
}
STREAM_KEYS = ["hex8_48", "tet4_24", "tet6_128"]
_cache = {}


def catalog(key):
    if key not in _cache:
        make, quad = CATALOG[key]
        dirs, w = oracle.product_quadrature(*quad)
        _cache[key] = (make(), dirs, w)
    return _cache[key]


def inputs_for(key, seed):
    N = catalog(key)[0]["n_cells"]
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 2.0, N), np.full(N, 0.5), rng.uniform(0.0, 1.0, (1, N))


@pytest.mark.parametrize("lanes", [(3e6, 3e7), (1e4, 1e5)], ids=["one_lane", "three_lanes_with_solo"])
def test_served_results_equal_alone_within_budget(lanes):
    # with bounds (1e4, 1e5) the three stream meshes fall in three lanes, the
    # largest (tet6, 128 directions) in the solo lane
    import torch
    from paper_1803_09876_gb300.serve import GpuBackend, Server, poisson_stream, run_one_at_a_time, summarize

    J()
    reqs = poisson_stream(14, 400.0, STREAM_KEYS, inputs_for, seed=5000)
    be = GpuBackend(catalog, dtype=torch.float32, tol=1e-6, max_iters=500, lanes=lanes)
    budget = 256 << 20
    srv = Server(be, budget, sweeps_per_step=1)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    out = srv.run(reqs)
    torch.cuda.synchronize()
    assert srv.peak_used <= budget
    assert torch.cuda.max_memory_allocated() - base <= budget
    # requests overlapped on the device
    ev = srv.events
    most = 0
    live = 0
    for _, kind, _ in sorted(ev, key=lambda e: e[0]):
        live += 1 if kind == "admit" else -1
        most = max(most, live)
    assert most >= 2
    # each result equals the request solved alone (same kernels, same arithmetic)
    alone = run_one_at_a_time(GpuBackend(catalog, dtype=torch.float32, tol=1e-6, max_iters=500),
                              [r.__class__(rid=r.rid, arrival=0.0, mesh_key=r.mesh_key, sigma_t=r.sigma_t,
                                           c_ratio=r.c_ratio, q=r.q) for r in reqs])
    by_id = {r.rid: r for r in alone}
    for r in out:
        a = by_id[r.rid]
        assert r.iters == a.iters and r.resid == a.resid
        assert np.array_equal(r.phi, a.phi)
    s = summarize(out, lambda r: r.iters * catalog(r.mesh_key)[0]["n_cells"] * len(catalog(r.mesh_key)[1]))
    assert s["p50_s"] <= s["p99_s"]


def test_mesh_memory_estimate_bounds_the_build_peak():
    import torch
    from paper_1803_09876_gb300.serve import GpuBackend

    J()
    be = GpuBackend(catalog, dtype=torch.float32)
    for key in CATALOG:
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        g, nbytes = be.build_mesh(key)
        torch.cuda.synchronize()
        peak = torch.cuda.max_memory_allocated() - base
        built = nbytes - be.resident_extra_bytes(key)  # the reservation for state of the first solve
        assert 0 < built <= peak <= be.mesh_bytes_estimate(key), (key, built, peak, be.mesh_bytes_estimate(key))
        del g


def test_solo_lane_state_stays_within_the_mesh_reservation():
    # a solo-lane request leaves its sweep state (psi, the face stream) on the
    # mesh's handle; the reservation made with the mesh covers it
    import torch
    from paper_1803_09876_gb300.serve import GpuBackend, Request

    J()
    be = GpuBackend(catalog, dtype=torch.float32, tol=1e-6, max_iters=50, lanes=(1e4, 1e5))
    key = "tet24_128"
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    g, nbytes = be.build_mesh(key)
    assert be.lane_of(g) == be.solo_lane
    sig, c, q = inputs_for(key, 7)
    r = Request(rid=0, arrival=0.0, mesh_key=key, sigma_t=sig, c_ratio=c, q=q)
    for _ in range(2):
        be.solve_alone(g, r)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() - base <= nbytes
    assert be.request_bytes(g, r) < be.resident_extra_bytes(key)
