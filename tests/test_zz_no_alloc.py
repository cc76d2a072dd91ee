"""The allocation-free source iteration against the regular one.

jsweep_source_iterate_noalloc exists for callers that cannot allocate device
memory while they run (a host application that owns the device's memory
budget, or a loop that cannot afford the device-wide synchronisation of
cudaMalloc/cudaFree).  These checks call both entry points through the C ABI on
the same inputs, twice in a row.  Both run the same per-cell solve, emission,
phi reduction and residual kernels, so they must agree bit for bit (same
iteration count, same residual, same phi); each result is also checked against
the FP64 oracle's converged solution within the parity tolerance of its
precision.  The checks also require that the calls make no allocation through
the installed (torch) allocator and that a problem larger than the fixed
scratch array is refused.  This file is collected last so that a run stopping
at its first failure has run everything else first.
"""

import numpy as np
import pytest

import oracle
from inputs import hex_grid, make_workload
from _gpu import J, TOL_F32, TOL_F64, build, rel_err, tensor

pytestmark = pytest.mark.gpu


def _alloc_count(torch):
    return torch.cuda.memory_stats().get("allocation.all.allocated", 0)


def _compare(mesh, dirs, w, sig, c, q, dtype, tol, rel_tol, inflow=None):
    import torch
    js = J()
    g = build(mesh, dirs, w)
    args = (tensor(sig, dtype), tensor(c, dtype), tensor(q, dtype))
    infl = None if inflow is None else tensor(inflow, dtype)
    R, N = q.shape
    ref_phi, _, _, conv, _ = oracle.build_dags(mesh, dirs).source_iterate(
        sig, c, q, w, tol, 2000, inflow=inflow, nthreads=oracle.max_threads())
    assert conv
    outs = []
    for _ in range(2):
        phi, it, res, ok = js.jsweep_source_iterate(g, *args, inflow=infl, tol=tol, max_iters=2000)
        assert ok
        outs.append((phi.cpu().numpy(), it, res))
    phi_na = torch.empty((R, N), dtype=dtype, device="cuda")
    torch.cuda.synchronize()
    before = _alloc_count(torch)
    na = []
    for _ in range(2):
        phi, it, res, ok = js.jsweep_source_iterate_noalloc(g, *args, phi_na, inflow=infl, tol=tol,
                                                             max_iters=2000)
        assert ok and res < tol
        na.append((phi.cpu().numpy(), it, res))
    torch.cuda.synchronize()
    assert _alloc_count(torch) == before  # nothing was allocated through the installed allocator
    for (ref, it_ref, res_ref), (got, it_got, res_got) in zip(outs, na):
        assert it_got == it_ref and res_got == res_ref
        assert np.array_equal(got, ref)  # same kernels: the same bits
        assert rel_err(got, ref_phi) < rel_tol  # and the oracle's fixed point
    return g


def test_noalloc_matches_regular_fp64_workload1():
    wl = make_workload(1)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    import torch
    _compare(wl, dirs, w, wl["sigma_t"], wl["c_ratio"], wl["q"], torch.float64, 1e-8, TOL_F64)


def test_noalloc_matches_regular_fp32_cyclic_eight_rhs_with_inflow():
    import torch
    mesh = hex_grid(6, 0.3, 3)
    dirs, w = oracle.product_quadrature(6, 6)
    N = mesh["n_cells"]
    rng = np.random.default_rng(21)
    sig = rng.lognormal(0.0, 1.0, N)
    c = np.full(N, 0.7)
    q = rng.uniform(0.0, 1.0, (8, N))
    g0 = oracle.build_dags(mesh, dirs)
    assert g0.n_lag_total > 0
    inflow = rng.uniform(0.0, 0.3, (8, g0.n_bfaces))
    _compare(mesh, dirs, w, sig, c, q, torch.float32, 1e-6, TOL_F32, inflow=inflow)


def test_noalloc_refuses_problems_larger_than_its_array():
    import torch
    js = J()
    mesh = hex_grid(24, 0.1, 1)  # 13,824 cells x 288 directions x 8 rhs x 4 B = 127 MB of psi
    dirs, w = oracle.product_quadrature(6, 6)
    g = build(mesh, dirs, w)
    N = mesh["n_cells"]
    q = torch.ones((8, N), dtype=torch.float32, device="cuda")
    one = torch.ones(N, dtype=torch.float32, device="cuda")
    phi = torch.empty((8, N), dtype=torch.float32, device="cuda")
    with pytest.raises(js.JsweepError) as e:
        js.jsweep_source_iterate_noalloc(g, one, one * 0.5, q, phi)
    assert e.value.code == js.JSWEEP_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
