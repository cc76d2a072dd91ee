"""Failures made on the host: an allocator that refuses memory.  The library
must report JSWEEP_ERR_OOM, leave nothing half-built behind, and keep working
once memory is available again.  No GPU fault is involved."""

import numpy as np
import pytest

import oracle
from inputs import hex_grid
from _gpu import J, TOL_F64, build, rel_err, tensor

pytestmark = pytest.mark.gpu


def _refusing_allocator(js, limit):
    import torch

    def _alloc(nbytes, stream, ctx):
        if nbytes > limit:
            return None  # refused: the library must report JSWEEP_ERR_OOM
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      torch.cuda.current_stream()))

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    js.set_allocator(js._ALLOC_FN(_alloc), js._FREE_FN(_free))  # kept alive by the binding


def test_allocator_refusal_reports_oom_and_recovers():
    import torch
    js = J()
    mesh = hex_grid(16, 0.15, 1)  # 4,096 cells x 288 directions: the graph arrays exceed 1 MiB
    dirs, w = oracle.product_quadrature(6, 6)
    _refusing_allocator(js, 1 << 20)
    try:
        with pytest.raises(js.JsweepError) as e:
            build(mesh, dirs, w)
        assert e.value.code == js.JSWEEP_ERR_OOM
    finally:
        js.use_torch_allocator()
    # the same build succeeds once memory is available, and sweeps correctly
    g = build(mesh, dirs, w)
    N = mesh["n_cells"]
    rng = np.random.default_rng(8)
    sig, src = rng.uniform(0.5, 2.0, N), rng.uniform(0.0, 1.0, (1, N))
    phi = js.jsweep_sweep(g, tensor(sig, torch.float64), tensor(src, torch.float64))
    ref = oracle.build_dags(mesh, dirs).sweep(sig, src, w)[0]
    assert rel_err(phi.cpu().numpy(), ref) < TOL_F64


def test_batch_add_refused_adds_nothing():
    import torch
    js = J()
    mesh = hex_grid(8, 0.15, 2)
    dirs, w = oracle.product_quadrature(6, 6)
    g = build(mesh, dirs, w)
    N = mesh["n_cells"]
    args = [torch.ones(N, dtype=torch.float32, device="cuda"), torch.full((N,), 0.5, device="cuda"),
            torch.ones((1, N), dtype=torch.float32, device="cuda")]
    b = js.Batch(torch.float32, 1)
    phi = torch.empty((1, N), dtype=torch.float32, device="cuda")
    _refusing_allocator(js, 64 << 10)  # psi of this problem is 590 KB
    try:
        with pytest.raises(js.JsweepError) as e:
            b.add(g, *args, phi_out=phi, tol=1e-6)
        assert e.value.code == js.JSWEEP_ERR_OOM
        assert len(b) == 0
    finally:
        js.use_torch_allocator()
    pid = b.add(g, *args, phi_out=phi, tol=1e-6)
    b.source_iterate()
    ref, it, _, _ = js.jsweep_source_iterate(g, *args, tol=1e-6)
    assert b.query(pid)[1] == it
    assert torch.equal(b.phi(pid), ref)
