"""Batched source iteration (jsweep_batch_*) against the single-problem path
and the FP64 oracle.

A problem's per-cell solves and its phi reduction are the same device
functions in a batch as alone, and the residual is a max (order-free), so a
problem's phi and iteration count in a batch must be bit-identical to
jsweep_source_iterate on it alone; the oracle check bounds both.
"""

import numpy as np
import pytest

import oracle
from inputs import hex_grid, kuhn_tets, make_batch_problem
from _gpu import J, TOL_F32, TOL_F64, build, rel_err, tensor

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _problems():
    """Uneven problems: tets and hexes, 24..288 directions, a cyclic mesh with
    lagged faces, one with inflow, and two problems on one shared handle."""
    rng = np.random.default_rng(77)
    out = []
    specs = [(kuhn_tets(5, 0.2, 11), (1, 3), False), (hex_grid(6, 0.3, 3), (6, 6), True),
             (kuhn_tets(3, 0.2, 12), (3, 4), False), (hex_grid(9, 0.15, 4), (2, 3), False),
             (kuhn_tets(7, 0.2, 13), (4, 4), False)]
    for mesh, quad, with_inflow in specs:
        dirs, w = oracle.product_quadrature(*quad)
        N = mesh["n_cells"]
        out.append(dict(mesh=mesh, dirs=dirs, w=w, sig=rng.uniform(0.5, 2.0, N), c=np.full(N, 0.5),
                        q=rng.uniform(0.0, 1.0, (1, N)), inflow=with_inflow))
    # a second problem on the first problem's mesh and directions (shared handle)
    p0 = out[0]
    N0 = p0["mesh"]["n_cells"]
    out.append(dict(p0, sig=rng.uniform(0.5, 2.0, N0), q=rng.uniform(0.0, 1.0, (1, N0)), share=0))
    return out


def _setup(dtype, nrhs=1, **opt):
    torch = _torch()
    js = J()
    probs = _problems()
    handles = []
    for i, p in enumerate(probs):
        if "share" in p:
            handles.append(handles[p["share"]])
        else:
            handles.append(build(p["mesh"], p["dirs"], p["w"]))
    data = []
    for p, g in zip(probs, handles):
        N = p["mesh"]["n_cells"]
        q = np.repeat(p["q"], nrhs, axis=0) * (1.0 + np.arange(nrhs))[:, None]
        infl = None
        if p["inflow"]:
            nb = g.mesh.n_bfaces
            infl = tensor(np.random.default_rng(5).uniform(0.0, 0.5, (nrhs, nb)), dtype)
        data.append(dict(g=g, sig=tensor(p["sig"], dtype), c=tensor(p["c"], dtype), q=tensor(q, dtype),
                         inflow=infl, q_np=q, p=p, N=N))
    return js, data


def _solo(js, d, tol, max_iters=500, allow=False):
    phi, it, res, ok = js.jsweep_source_iterate(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=tol,
                                                max_iters=max_iters, allow_not_converged=allow)
    return phi.cpu().numpy().copy(), it, res


@pytest.mark.parametrize("mode", [1, 2], ids=["level_sync", "persistent"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_equals_solo_bitwise(prec, mode):
    torch = _torch()
    dtype = torch.float64 if prec == "f64" else torch.float32
    tol = 1e-8 if prec == "f64" else 1e-6
    js, data = _setup(dtype)
    b = js.Batch(dtype, 1, js.jsweep_options_default(angles_per_warp=1, sweep_mode=mode))
    ids = [b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=tol, max_iters=500) for d in data]
    its, res = b.source_iterate()
    for k, (pid, d) in enumerate(zip(ids, data)):
        ref, it_ref, res_ref = _solo(js, d, tol)
        got = b.phi(pid).cpu().numpy()
        assert its[k] == it_ref
        assert res[k] == res_ref
        assert np.array_equal(got, ref), f"problem {k}: max diff {np.max(np.abs(got - ref))}"
        assert b.query(pid) == (js.JSWEEP_PROBLEM_CONVERGED, it_ref, res_ref)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_of_one_cell_shape_reads_face_streams_bitwise(prec):
    # all problems on tetrahedra: the level-synchronous batch reads every
    # handle's face-coefficient stream (with upwind positions and sweep-order
    # psi by default, with cell ids when that copy is off); with the stream off
    # it reads the cell geometry; all give the single-problem bits
    torch = _torch()
    dtype = torch.float64 if prec == "f64" else torch.float32
    tol = 1e-8 if prec == "f64" else 1e-6
    js = J()
    rng = np.random.default_rng(78)
    data = []
    for n, quad in ((5, (1, 3)), (3, (3, 4)), (7, (4, 4)), (6, (2, 2))):
        mesh = kuhn_tets(n, 0.2, 20 + n)
        dirs, w = oracle.product_quadrature(*quad)
        N = mesh["n_cells"]
        data.append(dict(g=build(mesh, dirs, w), sig=tensor(rng.uniform(0.5, 2.0, N), dtype),
                         c=tensor(np.full(N, 0.5), dtype), q=tensor(rng.uniform(0.0, 1.0, (2, N)), dtype),
                         inflow=None, N=N))
    solo = [js.jsweep_source_iterate(d["g"], d["sig"], d["c"], d["q"], tol=tol, max_iters=500) for d in data]
    for no_stream, no_seq in ((0, 0), (0, 1), (1, 0)):
        b = js.Batch(dtype, 2, js.jsweep_options_default(sweep_mode=1, no_face_stream=no_stream,
                                                         no_sweep_order_psi=no_seq))
        ids = [b.add(d["g"], d["sig"], d["c"], d["q"], tol=tol, max_iters=500) for d in data]
        its, _ = b.source_iterate()
        for k, pid in enumerate(ids):
            assert its[k] == solo[k][1]
            assert torch.equal(b.phi(pid), solo[k][0])


@pytest.mark.parametrize("mode,apw,cells,order", [(2, 2, 16, 1), (2, 4, 8, 0), (1, 4, 8, 1), (1, 2, 16, 0),
                                                  (2, 1, 5, 1)])
def test_batch_angles_per_warp_fp32_against_oracle(mode, apw, cells, order):
    torch = _torch()
    js, data = _setup(torch.float32, nrhs=2)
    b = js.Batch(torch.float32, 2, js.jsweep_options_default(angles_per_warp=apw, cluster_cells=cells,
                                                              unit_order=order, sweep_mode=mode))
    ids = [b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=1e-6) for d in data]
    b.source_iterate()
    for pid, d in zip(ids, data):
        p = d["p"]
        o = oracle.build_dags(p["mesh"], p["dirs"])
        infl = None if d["inflow"] is None else d["inflow"].double().cpu().numpy()
        ref = o.source_iterate(p["sig"], p["c"], d["q_np"], p["w"], inflow=infl, tol=1e-10,
                               max_iters=2000)[0]
        assert rel_err(b.phi(pid).cpu().numpy(), ref) < TOL_F32 * 5  # converged to 1e-6 vs 1e-10


def test_batch_fp64_eight_rhs_against_oracle():
    torch = _torch()
    js, data = _setup(torch.float64, nrhs=8)
    b = js.Batch(torch.float64, 8)
    ids = [b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=1e-12, max_iters=2000)
           for d in data[:3]]
    its, _ = b.source_iterate()
    for k, (pid, d) in enumerate(zip(ids, data[:3])):
        p = d["p"]
        o = oracle.build_dags(p["mesh"], p["dirs"])
        infl = None if d["inflow"] is None else d["inflow"].cpu().numpy()
        ref, it_ref = o.source_iterate(p["sig"], p["c"], d["q_np"], p["w"], inflow=infl, tol=1e-12,
                                       max_iters=2000)[:2]
        assert its[k] == it_ref
        assert rel_err(b.phi(pid).cpu().numpy(), ref) < TOL_F64


@pytest.mark.parametrize("mode", [1, 2], ids=["level_sync", "persistent"])
def test_continuous_batching_add_remove_between_steps(mode):
    # problems join while others iterate and leave when done; every result
    # equals the problem solved alone
    torch = _torch()
    js, data = _setup(torch.float32)
    refs = [_solo(js, d, 1e-6) for d in data]
    b = js.Batch(torch.float32, 1, js.jsweep_options_default(sweep_mode=mode))
    live = {}
    pending = list(range(len(data)))
    done = {}
    rounds = 0
    while pending or live:
        if pending:  # admit one new problem per step
            k = pending.pop(0)
            d = data[k]
            live[b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=1e-6)] = k
        b.step(2)
        for pid in list(live):
            st, it, res = b.query(pid)
            if st != js.JSWEEP_PROBLEM_ACTIVE:
                assert st == js.JSWEEP_PROBLEM_CONVERGED
                done[live[pid]] = (b.phi(pid).cpu().numpy().copy(), it, res)
                b.remove(pid)
                del live[pid]
        rounds += 1
        assert rounds < 1000
    assert len(b) == 0
    for k, (ref, it_ref, res_ref) in enumerate(refs):
        got, it, res = done[k]
        assert it == it_ref and res == res_ref
        assert np.array_equal(got, ref)


def test_remove_active_problem_and_reuse():
    torch = _torch()
    js, data = _setup(torch.float32)
    b = js.Batch(torch.float32, 1)
    a = b.add(data[1]["g"], data[1]["sig"], data[1]["c"], data[1]["q"], inflow=data[1]["inflow"], tol=1e-6)
    c = b.add(data[4]["g"], data[4]["sig"], data[4]["c"], data[4]["q"], tol=1e-6)
    assert b.step(1) == 2
    b.remove(a)  # still active
    while b.step(3):
        pass
    ref, it_ref, _ = _solo(js, data[4], 1e-6)
    assert b.query(c)[1] == it_ref
    assert np.array_equal(b.phi(c).cpu().numpy(), ref)
    with pytest.raises(js.JsweepError) as e:
        b.query(a)
    assert e.value.code == js.JSWEEP_ERR_INVALID_ARG


def test_max_iters_state_and_output():
    torch = _torch()
    js, data = _setup(torch.float64)
    d = data[1]
    b = js.Batch(torch.float64, 1)
    pid = b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=0.0, max_iters=4)
    its, res = b.source_iterate(allow_not_converged=True)
    ref, it_ref, res_ref = _solo(js, d, 0.0, max_iters=4, allow=True)
    assert its[0] == 4 == it_ref and res[0] == res_ref
    assert b.query(pid)[0] == js.JSWEEP_PROBLEM_MAX_ITERS
    assert np.array_equal(b.phi(pid).cpu().numpy(), ref)
    with pytest.raises(js.JsweepError) as e:
        b.source_iterate()
    assert e.value.code == js.JSWEEP_ERR_NOT_CONVERGED


def test_autotune_keeps_results():
    torch = _torch()
    js, data = _setup(torch.float32)
    b = js.Batch(torch.float32, 1)
    ids = [b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=1e-6) for d in data]
    ms = b.autotune()
    assert ms > 0.0
    b.source_iterate()
    sweep_ms, iter_ms, launches = b.stats()
    assert 0.0 < sweep_ms <= iter_ms and launches > 0
    for pid, d in zip(ids, data):
        ref, it_ref, _ = _solo(js, d, 1e-6)
        assert np.array_equal(b.phi(pid).cpu().numpy(), ref)


def test_handle_outlives_destroy_while_in_batch():
    torch = _torch()
    js = J()
    p = make_batch_problem(dict(n=4, ndirs=24, quad=(1, 3), seed=123))
    dirs, w = oracle.product_quadrature(1, 3)
    g = build(p, dirs, w)
    args = (tensor(p["sigma_t"], torch.float32), tensor(p["c_ratio"], torch.float32), tensor(p["q"], torch.float32))
    ref, it_ref, _, _ = js.jsweep_source_iterate(g, *args, tol=1e-6)
    ref = ref.cpu().numpy().copy()
    b = js.Batch(torch.float32, 1)
    pid = b.add(g, *args, tol=1e-6)
    # drop the caller's reference: the batch problem keeps the handle alive
    js.lib().jsweep_dags_destroy(g._h)
    g._h = None
    b.source_iterate()
    assert np.array_equal(b.phi(pid).cpu().numpy(), ref)
    b.remove(pid)


def test_problem_bytes_match_allocation():
    # count the bytes the library requests through its allocator while adding
    # a problem (torch's own statistics also count cached-block slack)
    import ctypes
    torch = _torch()
    js, data = _setup(torch.float32, nrhs=8)
    d = data[1]
    b = js.Batch(torch.float32, 8)
    want = b.problem_bytes(d["g"], has_inflow=True)
    phi_out = torch.empty((8, d["N"]), dtype=torch.float32, device="cuda")
    requested = []

    def _alloc(nbytes, stream, ctx):
        requested.append(int(nbytes))
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      torch.cuda.current_stream()))

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    js.set_allocator(js._ALLOC_FN(_alloc), js._FREE_FN(_free))  # kept alive by the binding
    try:
        pid = b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], phi_out=phi_out, tol=1e-6)
        b.remove(pid)
    finally:
        js.use_torch_allocator()
    # psi and its sweep-order copy (a level-synchronous batch), flags, source records, lagged
    # values, two phi buffers, inflow
    assert len(requested) == 8
    assert want <= sum(requested) <= want + 8 * 255  # each request rounded up to 256 bytes


def test_batch_timeout_reports_error_and_recovers():
    torch = _torch()
    js, data = _setup(torch.float32)
    d = data[1]  # hex grid, several layers per direction: the waits run out
    b = js.Batch(torch.float32, 1, js.jsweep_options_default(debug_block_waits=1, spin_timeout_s=0.05,
                                                              sweep_mode=2))
    b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=1e-6)
    with pytest.raises(js.JsweepError) as e:
        b.step(1)
    assert e.value.code == js.JSWEEP_ERR_DEVICE_TIMEOUT
    # the context is still usable
    ref, it_ref, _ = _solo(js, d, 1e-6)
    assert it_ref > 1 and np.isfinite(ref).all()


def test_launch_and_poll_two_batches_on_two_streams():
    # one host thread keeps two batches busy at once; each result equals the
    # problem solved alone
    torch = _torch()
    js, data = _setup(torch.float32)
    refs = [_solo(js, d, 1e-6) for d in data]
    lanes = [js.Batch(torch.float32, 1), js.Batch(torch.float32, 1)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ids = []
    for k, d in enumerate(data):
        b = lanes[k % 2]
        ids.append((k % 2, b.add(d["g"], d["sig"], d["c"], d["q"], inflow=d["inflow"], tol=1e-6)))
    active = [sum(1 for lane, _ in ids if lane == i) for i in range(2)]
    pending = [False, False]
    rounds = 0
    while any(active) or any(pending):
        for i, b in enumerate(lanes):
            if active[i] and not pending[i]:
                b.launch(1, stream=streams[i])
                pending[i] = True
        for i, b in enumerate(lanes):
            if pending[i]:
                done, n = b.poll()
                if done:
                    pending[i] = False
                    active[i] = n
        rounds += 1
        assert rounds < 10_000_000
    for (lane, pid), (ref, it_ref, res_ref) in zip(ids, refs):
        st, it, res = lanes[lane].query(pid)
        assert st == js.JSWEEP_PROBLEM_CONVERGED and it == it_ref and res == res_ref
        assert np.array_equal(lanes[lane].phi(pid).cpu().numpy(), ref)
    with pytest.raises(js.JsweepError):
        lanes[0].launch(0)
