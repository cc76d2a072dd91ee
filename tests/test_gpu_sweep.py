"""GPU sweeps and source iteration against the FP64 oracle."""

import math

import numpy as np
import pytest

import oracle
from inputs import column_mesh, hex_grid, kuhn_tets, make_workload, pinwheel_mesh
from _gpu import J, TOL_F32, TOL_F64, build, rel_err, set_opts, tensor

pytestmark = pytest.mark.gpu

MODES = [dict(sweep_mode=1), dict(sweep_mode=2), dict(sweep_mode=2, priority=1, cluster_cells=7),
         dict(sweep_mode=2, priority=2, cluster_cells=1), dict(sweep_mode=1, cluster_cells=5),
         dict(sweep_mode=2, priority=3), dict(sweep_mode=2, priority=3, cluster_cells=3),
         dict(sweep_mode=2, priority=4), dict(sweep_mode=2, priority=4, cluster_cells=3),
         dict(sweep_mode=3), dict(sweep_mode=3, patch_cells=64), dict(sweep_mode=1, tail_units=64),
         dict(sweep_mode=1, no_sweep_order_psi=1)]


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("opts", MODES, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
@pytest.mark.parametrize("R", [1, 3, 8])
def test_fp64_two_sweeps_with_lag(opts, R):
    # cyclic jittered hex mesh: the second sweep uses the first sweep's lagged values
    torch = _torch()
    mesh = hex_grid(6, 0.3, 3)
    dirs, w = oracle.product_quadrature(6, 6)
    g = build(mesh, dirs, w, **opts)
    o = oracle.build_dags(mesh, dirs)
    assert o.n_lag_total > 0
    N, M = mesh["n_cells"], len(dirs)
    rng = np.random.default_rng(10 + R)
    sig = rng.lognormal(0.0, 1.0, N)
    lag = None
    for it in range(2):
        src = rng.uniform(0.0, 1.0, (R, N))
        inflow = rng.uniform(0.0, 1.0, (R, o.n_bfaces))
        phi_ref, psi_ref, lag = o.sweep(sig, src, w, inflow=inflow, psi_lag=lag, want_psi=True)
        psi_gpu = torch.empty((R, M, N), dtype=torch.float64, device="cuda")
        phi_gpu = J().jsweep_sweep(g, tensor(sig, torch.float64), tensor(src, torch.float64),
                                   inflow=tensor(inflow, torch.float64), psi_out=psi_gpu)
        assert rel_err(phi_gpu.cpu().numpy(), phi_ref) < TOL_F64
        assert rel_err(psi_gpu.cpu().numpy().reshape(R, -1), psi_ref.reshape(R, -1)) < TOL_F64


@pytest.mark.parametrize("opts", MODES[:3] + MODES[5:], ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_fp32_sweep_tets_and_hex(opts):
    torch = _torch()
    for mesh, quad in ((kuhn_tets(8, 0.2, 2), (4, 4)), (hex_grid(10, 0.15, 5), (6, 6))):
        dirs, w = oracle.product_quadrature(*quad)
        g = build(mesh, dirs, w, **opts)
        o = oracle.build_dags(mesh, dirs)
        N = mesh["n_cells"]
        rng = np.random.default_rng(3)
        sig = rng.lognormal(0.0, 1.0, N)
        src = rng.uniform(0.0, 1.0, (8, N))
        phi_ref, _, lag = o.sweep(sig, src, w)
        phi_gpu = J().jsweep_sweep(g, tensor(sig, torch.float32), tensor(src, torch.float32))
        assert rel_err(phi_gpu.cpu().numpy(), phi_ref) < TOL_F32
        # second sweep (lagged values from the first)
        phi_ref2, _, _ = o.sweep(sig, src, w, psi_lag=lag)
        phi_gpu2 = J().jsweep_sweep(g, tensor(sig, torch.float32), tensor(src, torch.float32))
        assert rel_err(phi_gpu2.cpu().numpy(), phi_ref2) < TOL_F32


def test_workload1_source_iteration_fp64_full_size():
    torch = _torch()
    wl = make_workload(1)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    o = oracle.build_dags(wl, dirs)
    phi_ref, it_ref, res_ref, conv, _ = o.source_iterate(wl["sigma_t"], wl["c_ratio"], wl["q"], w, 1e-8, 1000)
    assert conv
    for opts in (dict(sweep_mode=1), dict(sweep_mode=2)):
        g = build(wl, dirs, w, **opts)
        phi, it, res, ok = J().jsweep_source_iterate(
            g, tensor(wl["sigma_t"], torch.float64), tensor(wl["c_ratio"], torch.float64),
            tensor(wl["q"], torch.float64), tol=1e-8, max_iters=1000)
        assert ok and it == it_ref
        assert abs(res - res_ref) <= 1e-6 * res_ref
        assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F64


def test_cyclic_source_iteration_fp64_converges_to_oracle():
    torch = _torch()
    mesh = hex_grid(5, 0.3, 11)
    dirs, w = oracle.product_quadrature(6, 6)
    o = oracle.build_dags(mesh, dirs)
    assert o.n_lag_total > 0
    N = mesh["n_cells"]
    rng = np.random.default_rng(8)
    sig = rng.uniform(0.5, 2.0, N)
    c = np.full(N, 0.6)
    q = rng.uniform(0.0, 1.0, (2, N))
    inflow = rng.uniform(0.0, 0.5, (2, o.n_bfaces))
    phi_ref, it_ref, _, conv, _ = o.source_iterate(sig, c, q, w, 1e-10, 500, inflow=inflow)
    g = build(mesh, dirs, w, sweep_mode=2, priority=1)
    phi, it, res, ok = J().jsweep_source_iterate(
        g, tensor(sig, torch.float64), tensor(c, torch.float64), tensor(q, torch.float64),
        inflow=tensor(inflow, torch.float64), tol=1e-10, max_iters=500)
    assert ok and it == it_ref
    assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F64


def test_fp32_source_iteration_fixed_and_converged():
    torch = _torch()
    mesh = kuhn_tets(10, 0.2, 2)
    dirs, w = oracle.product_quadrature(4, 4)
    o = oracle.build_dags(mesh, dirs)
    N = mesh["n_cells"]
    rng = np.random.default_rng(2)
    sig = rng.lognormal(0.0, 1.0, N)
    c = rng.uniform(0.0, 0.9, N)
    q = rng.uniform(0.0, 1.0, (1, N))
    g = build(mesh, dirs, w)
    args = (tensor(sig, torch.float32), tensor(c, torch.float32), tensor(q, torch.float32))
    # same fixed number of iterations from phi = 0
    phi_ref, _, _, _, _ = o.source_iterate(sig, c, q, w, 0.0, 5)
    phi, it, _, ok = J().jsweep_source_iterate(g, *args, tol=0.0, max_iters=5, allow_not_converged=True)
    assert not ok and it == 5
    assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F32
    # converged solutions (tol 1e-6)
    phi_ref, _, _, conv, _ = o.source_iterate(sig, c, q, w, 1e-6, 1000)
    phi, it, res, ok = J().jsweep_source_iterate(g, *args, tol=1e-6, max_iters=1000)
    assert ok and conv and res < 1e-6
    assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F32


def test_workload3_downscaled_fp32_eight_rhs_si():
    torch = _torch()
    wl = make_workload(3, n=24)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    o = oracle.build_dags(wl, dirs)
    assert o.n_lag_total > 0
    phi_ref, _, _, _, _ = o.source_iterate(wl["sigma_t"], wl["c_ratio"], wl["q"], w, 0.0, 3, nthreads=oracle.max_threads())
    for opts in (dict(sweep_mode=1), dict(sweep_mode=2, priority=2)):
        g = build(wl, dirs, w, **opts)
        phi, it, _, _ = J().jsweep_source_iterate(
            g, tensor(wl["sigma_t"], torch.float32), tensor(wl["c_ratio"], torch.float32),
            tensor(wl["q"], torch.float32), tol=0.0, max_iters=3, allow_not_converged=True)
        assert it == 3
        assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F32


def test_column_closed_form_fp64():
    torch = _torch()
    n, mu = 64, 0.37
    mesh = column_mesh(n, length=2.0)
    g = build(mesh, np.array([[mu, 0.0, 0.0]]), np.array([1.0]))
    rng = np.random.default_rng(5)
    sig = rng.uniform(0.2, 3.0, n)
    q = rng.uniform(0.0, 2.0, n)
    nb = g.mesh.n_bfaces
    inflow = np.full((1, nb), 0.7)
    phi = J().jsweep_sweep(g, tensor(sig, torch.float64), tensor(q[None], torch.float64),
                           inflow=tensor(inflow, torch.float64)).cpu().numpy()[0]
    dx = 2.0 / n
    prev, ref = 0.7, np.empty(n)
    for i in range(n):
        prev = (q[i] * dx + mu * prev) / (sig[i] * dx + mu)
        ref[i] = prev
    assert np.max(np.abs(phi - ref) / ref) < 1e-13


def test_uniform_solution_invariant_fp32_and_fp64():
    # S = k sigma_t with inflow k gives psi = k (acyclic tet mesh: no lagged values)
    torch = _torch()
    mesh = kuhn_tets(7, 0.2, 4)
    dirs, w = oracle.product_quadrature(4, 4)
    assert oracle.build_dags(mesh, dirs).n_lag_total == 0
    g = build(mesh, dirs, w, sweep_mode=2)
    N, M = mesh["n_cells"], len(dirs)
    sig = np.random.default_rng(1).lognormal(0.0, 1.0, N)
    k = 1.75
    for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
        psi = torch.empty((1, M, N), dtype=dt, device="cuda")
        phi = J().jsweep_sweep(g, tensor(sig, dt), tensor(k * sig[None], dt),
                               inflow=tensor(np.full((1, g.mesh.n_bfaces), k), dt), psi_out=psi)
        assert torch.max(torch.abs(psi.double() - k)).item() < tol * k
        assert np.max(np.abs(phi.cpu().numpy() / (4 * math.pi) - k)) < 10 * tol * k


def test_single_cell_and_unjittered_grid():
    torch = _torch()
    for mesh in (hex_grid(1, 0.0, 0), hex_grid(4, 0.0, 0)):
        dirs, w = oracle.product_quadrature(2, 3)
        g = build(mesh, dirs, w)
        o = oracle.build_dags(mesh, dirs)
        N = mesh["n_cells"]
        src = np.random.default_rng(0).uniform(0, 1, (2, N))
        sig = np.ones(N)
        phi_ref, _, _ = o.sweep(sig, src, w)
        phi = J().jsweep_sweep(g, tensor(sig, torch.float64), tensor(src, torch.float64))
        assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F64


def test_workload2_full_size_fp32_sweep_and_two_iterations():
    torch = _torch()
    wl = make_workload(2)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    o = oracle.build_dags(wl, dirs)
    nt = oracle.max_threads()
    phi_ref, _, _, _, _ = o.source_iterate(wl["sigma_t"], wl["c_ratio"], wl["q"], w, 0.0, 2, nthreads=nt)
    g = build(wl, dirs, w)
    phi, it, _, _ = J().jsweep_source_iterate(
        g, tensor(wl["sigma_t"], torch.float32), tensor(wl["c_ratio"], torch.float32),
        tensor(wl["q"], torch.float32), tol=0.0, max_iters=2, allow_not_converged=True)
    assert it == 2
    assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F32


def _bench_options(**override):
    """jsweep_options fields of the benchmark's default line (bench.py)."""
    import bench
    opts = bench.sweep_options(bench.parse([]))
    opts.update(override)
    return opts


def _oracle_phi_all_directions(wl, dirs, w, src, chunk=36):
    """phi of one oracle sweep over every direction, built and swept chunk by
    chunk of directions (bounded host memory); FP64 sums."""
    nt = oracle.max_threads()
    phi = None
    for m0 in range(0, len(dirs), chunk):
        o = oracle.build_dags(wl, dirs[m0:m0 + chunk])
        p, _, _ = o.sweep(wl["sigma_t"], src, w[m0:m0 + chunk], nthreads=nt)
        phi = p if phi is None else phi + p
        del o
    return phi


def test_workload3_full_size_benchmark_configuration_against_oracle():
    # 128^3, 288 directions, 8 right-hand sides, FP32, with the options the
    # benchmark times (bench.sweep_options of its default arguments): the full
    # phi of one sweep against the oracle's phi over all 288 directions, and
    # psi of sampled directions against the oracle's psi.  This reaches what
    # only the full size reaches: 64-bit psi and face-record offsets, grid
    # sizes, 1,859 schedule slots.  The persistent queue-driven schedule must
    # give the same bits.
    torch = _torch()
    wl = make_workload(3)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    g = build(wl, dirs, w, **_bench_options())
    N, M, R = wl["n_cells"], len(dirs), 8
    src = wl["q"] / (4 * math.pi)
    psi = torch.empty((R, M, N), dtype=torch.float32, device="cuda")
    sig_t, src_t = tensor(wl["sigma_t"], torch.float32), tensor(src, torch.float32)
    phi = J().jsweep_sweep(g, sig_t, src_t, psi_out=psi)
    sample = [0, 37, 100, 143, 200, 287]
    psi_s = psi[:, sample, :].cpu().numpy()
    del psi
    phi_np = phi.cpu().numpy()
    # the same sweep again (lagged values back to zero) on the persistent schedule
    g.reset_lag()
    set_opts(g, **_bench_options(sweep_mode=2))
    phi_q = J().jsweep_sweep(g, sig_t, src_t)
    same_bits = torch.equal(phi_q.cpu(), phi.cpu())
    del g
    torch.cuda.empty_cache()
    o = oracle.build_dags(wl, dirs[sample])
    _, psi_ref, _ = o.sweep(wl["sigma_t"], src, w[sample], want_psi=True, nthreads=oracle.max_threads())
    for i in range(len(sample)):
        assert rel_err(psi_s[:, i, :], psi_ref[:, i, :]) < TOL_F32
    del o, psi_ref
    phi_ref = _oracle_phi_all_directions(wl, dirs, w, src)
    assert rel_err(phi_np, phi_ref) < TOL_F32
    assert same_bits


def test_workload3_downscaled_converged_fp32_source_iteration():
    # workload 3 at 32^3 (c = 0.8, 8 right-hand sides, 288 directions): FP32
    # source iteration converged to 1e-6 against the oracle converged to the
    # same tolerance (the truncation error tol c / (1 - c) = 4e-6 stays inside
    # the FP32 tolerance), with the benchmark's options and the persistent one
    torch = _torch()
    wl = make_workload(3, n=32)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    o = oracle.build_dags(wl, dirs)
    assert o.n_lag_total > 0
    phi_ref, it_ref, _, conv, _ = o.source_iterate(wl["sigma_t"], wl["c_ratio"], wl["q"], w, 1e-6, 1000,
                                                   nthreads=oracle.max_threads())
    assert conv
    args = (tensor(wl["sigma_t"], torch.float32), tensor(wl["c_ratio"], torch.float32),
            tensor(wl["q"], torch.float32))
    outs = []
    for opts in (_bench_options(), _bench_options(sweep_mode=2)):
        g = build(wl, dirs, w, **opts)
        phi, it, res, ok = J().jsweep_source_iterate(g, *args, tol=1e-6, max_iters=1000)
        assert ok and res < 1e-6 and abs(it - it_ref) <= 2
        assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F32
        outs.append(phi.cpu())
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("mode", [2, 3], ids=["persistent", "patch_programs"])
def test_bounded_wait_times_out_and_context_survives(mode):
    torch = _torch()
    js = J()
    mesh = hex_grid(6, 0.15, 1)
    dirs, w = oracle.product_quadrature(1, 3)
    g = build(mesh, dirs, w, sweep_mode=mode, debug_block_waits=1, spin_timeout_s=0.05, patch_cells=32)
    N = mesh["n_cells"]
    sig = tensor(np.ones(N), torch.float32)
    src = tensor(np.ones((1, N)), torch.float32)
    with pytest.raises(js.JsweepError) as e:
        js.jsweep_sweep(g, sig, src)
    assert e.value.code == js.JSWEEP_ERR_DEVICE_TIMEOUT
    # the context is still usable
    set_opts(g, sweep_mode=mode, patch_cells=32)
    o = oracle.build_dags(mesh, dirs)
    phi_ref, _, _ = o.sweep(np.ones(N), np.ones((1, N)), w)
    phi = js.jsweep_sweep(g, sig, src)
    assert rel_err(phi.cpu().numpy(), phi_ref) < TOL_F32


def test_invalid_inputs_are_rejected():
    torch = _torch()
    js = J()
    mesh = hex_grid(3, 0.1, 1)
    bad = dict(mesh)
    bad["normals"] = mesh["normals"].copy()
    bad["normals"][5] = [0.0, 0.0, 1.0]  # breaks closure of two cells
    with pytest.raises(js.JsweepError) as e:
        js.mesh_from_dict(bad)
    assert e.value.code == js.JSWEEP_ERR_MESH_INVALID and "not closed" in str(e.value)
    bad = dict(mesh)
    bad["face_cells"] = mesh["face_cells"].copy()
    bad["face_cells"][0] = [3, 3]
    with pytest.raises(js.JsweepError) as e:
        js.mesh_from_dict(bad)
    assert e.value.code == js.JSWEEP_ERR_MESH_INVALID
    bad = dict(mesh)
    bad["volumes"] = -mesh["volumes"]
    with pytest.raises(js.JsweepError):
        js.mesh_from_dict(bad)
    dirs, w = oracle.product_quadrature(1, 3)
    g = build(mesh, dirs, w)
    N = mesh["n_cells"]
    with pytest.raises(js.JsweepError) as e:
        js.jsweep_sweep(g, tensor(np.ones(N), torch.float64), tensor(np.ones((9, N)), torch.float64))
    assert e.value.code == js.JSWEEP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        js.jsweep_sweep(g, tensor(np.ones(N), torch.float32), tensor(np.ones((1, N)), torch.float64))
    with pytest.raises(js.JsweepError):
        js.jsweep_quadrature_create(np.zeros((2, 3)), np.ones(2))


@pytest.mark.parametrize("patch_cells", [32, 200, 512])
def test_patch_programs_source_iteration_fp32_matches_oracle(patch_cells):
    # patch programs on a cyclic hex mesh and on tets, through source iteration
    torch = _torch()
    js = J()
    for mesh, quad in ((hex_grid(10, 0.3, 7), (6, 6)), (kuhn_tets(7, 0.2, 3), (4, 4))):
        dirs, w = oracle.product_quadrature(*quad)
        g = build(mesh, dirs, w, sweep_mode=3, patch_cells=patch_cells)
        N = mesh["n_cells"]
        rng = np.random.default_rng(patch_cells)
        sig, c, q = rng.uniform(0.5, 2.0, N), np.full(N, 0.6), rng.uniform(0.0, 1.0, (2, N))
        o = oracle.build_dags(mesh, dirs)
        ref = o.source_iterate(sig, c, q, w, tol=1e-10, max_iters=2000)[0]
        phi, it, res, ok = js.jsweep_source_iterate(g, tensor(sig, torch.float32), tensor(c, torch.float32),
                                                    tensor(q, torch.float32), tol=1e-6, max_iters=500)
        assert ok
        assert rel_err(phi.cpu().numpy(), ref) < 5 * TOL_F32


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_face_stream_and_every_schedule_give_the_same_bits(prec):
    # each cell-direction is solved by the same operations in every kernel (the
    # face coefficients Omega.A and the upwind sums are explicitly rounded), so
    # the precomputed face stream, the geometry reads and the data-driven and
    # patch-program schedules agree bit for bit, lagged faces included
    torch = _torch()
    dt = torch.float32 if prec == "f32" else torch.float64
    for mesh, quad, R in ((hex_grid(6, 0.3, 3), (6, 6), 1), (kuhn_tets(6, 0.2, 4), (4, 4), 3),
                          (column_mesh(40), (4, 4), 8), (pinwheel_mesh(), (6, 6), 2)):
        dirs, w = oracle.product_quadrature(*quad)
        N = mesh["n_cells"]
        rng = np.random.default_rng(21)
        sig = rng.lognormal(0.0, 1.0, N)
        srcs = [rng.uniform(0.0, 1.0, (R, N)) for _ in range(2)]
        outs = []
        for opts in (dict(sweep_mode=1), dict(sweep_mode=1, no_face_stream=1),
                     dict(sweep_mode=1, no_sweep_order_psi=1),
                     dict(sweep_mode=1, tail_units=1 << 30), dict(sweep_mode=1, tail_units=40),
                     dict(sweep_mode=1, tail_units=40, no_sweep_order_psi=1),
                     dict(sweep_mode=2), dict(sweep_mode=2, priority=3), dict(sweep_mode=2, priority=4),
                     dict(sweep_mode=3, patch_cells=64)):
            g = build(mesh, dirs, w, **opts)
            outs.append([J().jsweep_sweep(g, tensor(sig, dt), tensor(s, dt)).cpu() for s in srcs])
        for o in outs[1:]:
            for a, b in zip(outs[0], o):
                assert torch.equal(a, b)


def test_face_stream_refused_falls_back_to_geometry_reads():
    import torch
    js = J()
    mesh = kuhn_tets(6, 0.2, 4)
    dirs, w = oracle.product_quadrature(4, 4)
    N, M = mesh["n_cells"], len(dirs)
    # FP32 tetrahedra: four Omega.A values and four neighbour ids, 32 bytes per
    # record; the library rounds allocations up to 256 bytes
    stream_bytes = (N * M * 32 + 255) // 256 * 256
    g = build(mesh, dirs, w)
    rng = np.random.default_rng(22)
    sig, src = rng.uniform(0.5, 2.0, N), rng.uniform(0.0, 1.0, (1, N))
    ref = J().jsweep_sweep(build(mesh, dirs, w, no_face_stream=1), tensor(sig, torch.float32),
                           tensor(src, torch.float32)).cpu()

    def _alloc(nbytes, stream, ctx):
        if nbytes == stream_bytes:
            return None
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      torch.cuda.current_stream()))

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    js.set_allocator(js._ALLOC_FN(_alloc), js._FREE_FN(_free))
    try:
        phi = js.jsweep_sweep(g, tensor(sig, torch.float32), tensor(src, torch.float32)).cpu()
    finally:
        js.use_torch_allocator()
    assert torch.equal(phi, ref)
