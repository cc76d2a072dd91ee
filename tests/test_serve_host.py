"""Host logic of the serving loop (admission by memory budget, resident-mesh
LRU, continuous batching, latency bookkeeping) with a fake device backend and
a virtual clock: no GPU."""

import numpy as np
import pytest

from paper_1803_09876_gb300.serve import (Request, Server, face_record_bytes, handle_resident_bytes, percentile,
                                          poisson_stream, run_one_at_a_time, summarize)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


class FakeBackend:
    """Mesh `key` is an int: its graph takes 100*key bytes, a request on it 10*key.
    A request converges after `q[0, 0]` sweeps; a step costs 1 ms per sweep."""

    def __init__(self, clock, budget):
        self.clock = clock
        self.budget = budget
        self.allocated = 0
        self.peak = 0
        self.resident = {}
        self.probs = {}
        self.next_pid = 0
        self.builds = []
        self.released = []

    def _alloc(self, n):
        self.allocated += n
        self.peak = max(self.peak, self.allocated)
        assert self.allocated <= self.budget, "budget exceeded"

    def mesh_bytes_estimate(self, key):
        return 100 * key

    def request_bytes_estimate(self, key):
        return 10 * key

    def build_mesh(self, key):
        self._alloc(100 * key)
        self.builds.append(key)
        h = ("mesh", key)
        self.resident[h] = 100 * key
        return h, 100 * key

    def release_mesh(self, h):
        self.allocated -= self.resident.pop(h)
        self.released.append(h[1])

    def request_bytes(self, h, req):
        return 10 * h[1]

    def add(self, h, req):
        assert h in self.resident
        self._alloc(10 * h[1])
        pid = self.next_pid
        self.next_pid += 1
        self.probs[pid] = dict(h=h, req=req, it=0, target=int(req.q[0, 0]))
        return pid

    def step(self, k):
        self.clock.t += 1e-3 * k
        for p in self.probs.values():
            p["it"] = min(p["target"], p["it"] + k)

    def finished(self, pid):
        p = self.probs[pid]
        return p["it"] >= p["target"]

    def result(self, pid):
        p = self.probs[pid]
        return np.full(3, float(p["req"].rid)), p["it"], 0.0

    def remove(self, pid):
        p = self.probs.pop(pid)
        self.allocated -= 10 * p["h"][1]

    def solve_alone(self, h, req):
        n = int(req.q[0, 0])
        self.clock.t += 1e-3 * n
        return np.full(3, float(req.rid)), n, 0.0


def _req(rid, t, key, iters):
    return Request(rid=rid, arrival=t, mesh_key=key, sigma_t=np.ones(3), c_ratio=np.ones(3),
                   q=np.full((1, 3), float(iters)))


def test_all_requests_served_with_their_results():
    clk = Clock()
    be = FakeBackend(clk, budget=10_000)
    reqs = [_req(i, 0.002 * i, 1 + i % 3, 5 + i) for i in range(12)]
    out = Server(be, 10_000, clock=clk, sleep=clk.sleep).run(reqs)
    for r in out:
        assert r.iters == 5 + r.rid
        assert np.all(r.phi == r.rid)
        assert r.latency >= 0 and r.done >= r.admitted >= r.arrival
    assert be.allocated == sum(be.resident.values())  # only resident meshes remain


def test_budget_is_never_exceeded_and_lru_eviction_spares_meshes_in_use():
    clk = Clock()
    budget = 2 * 100 * 3 + 3 * 10 * 3  # two size-3 meshes and three requests on them
    be = FakeBackend(clk, budget=budget)
    # three meshes of size 3 cycle; each request is long enough to overlap the next arrival
    reqs = [Request(rid=i, arrival=0.004 * i, mesh_key=(3, i % 3), sigma_t=np.ones(3), c_ratio=np.ones(3),
                    q=np.full((1, 3), 6.0)) for i in range(9)]

    class KeyedBackend(FakeBackend):
        def mesh_bytes_estimate(self, key):
            return 100 * key[0]

        def request_bytes_estimate(self, key):
            return 10 * key[0]

        def build_mesh(self, key):
            self._alloc(100 * key[0])
            self.builds.append(key)
            h = ("mesh", key)
            self.resident[h] = 100 * key[0]
            return h, 100 * key[0]

        def release_mesh(self, h):
            # a mesh is never evicted while a request on it is admitted and unfinished
            assert all(p["h"] != h for p in self.probs.values())
            self.allocated -= self.resident.pop(h)
            self.released.append(h[1])

        def request_bytes(self, h, req):
            return 10 * h[1][0]

        def add(self, h, req):
            self._alloc(10 * h[1][0])
            pid = self.next_pid
            self.next_pid += 1
            self.probs[pid] = dict(h=h, req=req, it=0, target=int(req.q[0, 0]), size=10 * h[1][0])
            return pid

        def remove(self, pid):
            self.allocated -= self.probs.pop(pid)["size"]

    be = KeyedBackend(clk, budget=budget)
    srv = Server(be, budget, clock=clk, sleep=clk.sleep)
    out = srv.run(reqs)
    assert all(r.iters == 6 for r in out)
    assert be.peak <= budget and srv.peak_used <= budget
    assert len(be.released) >= 1  # a third mesh forced an eviction
    assert len(be.builds) > 3  # an evicted mesh was rebuilt when requested again


def test_continuous_batching_admits_while_others_iterate():
    clk = Clock()
    be = FakeBackend(clk, budget=10_000)
    reqs = [_req(0, 0.0, 1, 50), _req(1, 0.005, 2, 5)]
    srv = Server(be, 10_000, clock=clk, sleep=clk.sleep)
    out = srv.run(reqs)
    ev = [(k, rid) for _, k, rid in srv.events]
    # request 1 is admitted and finishes while request 0 is still iterating
    assert ev.index(("admit", 1)) < ev.index(("done", 0))
    assert ev.index(("done", 1)) < ev.index(("done", 0))
    assert out[1].latency < out[0].latency


def test_admission_is_first_come_first_served():
    clk = Clock()
    budget = 100 * 2 + 10 * 2 + 5  # one request on mesh 2 at a time; mesh 1 only once mesh 2 is evicted
    be = FakeBackend(clk, budget=budget)
    reqs = [_req(0, 0.0, 2, 20), _req(1, 0.001, 2, 20), _req(2, 0.002, 1, 1)]
    srv = Server(be, budget, clock=clk, sleep=clk.sleep)
    srv.run(reqs)
    admits = [rid for _, k, rid in srv.events if k == "admit"]
    assert admits == [0, 1, 2]
    # request 1 waits for request 0's memory; request 2 (small, but behind it) waits for request 1
    t = {rid: tm for tm, k, rid in srv.events if k == "admit"}
    done = {rid: tm for tm, k, rid in srv.events if k == "done"}
    assert t[1] >= done[0] and t[2] >= done[1]
    assert be.released == [2]


def test_request_larger_than_budget_is_rejected():
    clk = Clock()
    be = FakeBackend(clk, budget=50)
    with pytest.raises(ValueError):
        Server(be, 50, clock=clk, sleep=clk.sleep).run([_req(0, 0.0, 1, 3)])


def test_one_at_a_time_is_serial_and_in_arrival_order():
    clk = Clock()
    be = FakeBackend(clk, budget=10_000)
    reqs = [_req(i, 0.0, 1, 10) for i in range(4)]
    out = run_one_at_a_time(be, reqs, clock=clk, sleep=clk.sleep)
    done = [r.done for r in out]
    assert done == sorted(done)
    assert np.allclose(np.diff(done), 0.010)
    s = summarize(out, lambda r: 1.0)
    assert s["requests"] == 4 and s["p50_s"] <= s["p99_s"] <= s["max_s"]


def test_percentile_and_poisson_stream_are_deterministic():
    assert percentile([1, 2, 3, 4], 50) == 2.5
    assert percentile([5], 99) == 5
    mk = lambda key, seed: (np.ones(2), np.ones(2), np.ones((1, 2)) * seed)  # noqa: E731
    a = poisson_stream(20, 10.0, ["a", "b"], mk, seed=5000)
    b = poisson_stream(20, 10.0, ["a", "b"], mk, seed=5000)
    assert [(r.arrival, r.mesh_key) for r in a] == [(r.arrival, r.mesh_key) for r in b]
    assert a[0].arrival == 0.0 and all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))
    # mean gap close to 1 / rate
    gaps = np.diff([r.arrival for r in poisson_stream(4000, 10.0, ["a"], mk, seed=1)])
    assert abs(gaps.mean() - 0.1) < 0.01


def test_cancelled_requests_free_their_memory_and_others_finish():
    clk = Clock()
    be = FakeBackend(clk, budget=10_000)
    reqs = [_req(0, 0.0, 2, 40), _req(1, 0.0, 1, 10), _req(2, 0.001, 3, 10), _req(3, 0.05, 1, 5)]
    srv = Server(be, 10_000, clock=clk, sleep=clk.sleep)
    # request 0 is cancelled while it iterates, request 3 just after it is admitted
    out = srv.run(reqs, cancels=[(0.005, 0), (0.0505, 3)])
    by = {r.rid: r for r in out}
    assert by[0].cancelled and by[0].phi is None and by[0].done is None
    assert not by[1].cancelled and by[1].iters == 10
    assert not by[2].cancelled and by[2].iters == 10
    assert len(be.probs) == 0 and srv.reserved == 0
    assert be.allocated == sum(be.resident.values())
    kinds = [(k, rid) for _, k, rid in srv.events]
    assert ("cancel", 0) in kinds and ("done", 0) not in kinds
    assert by[3].cancelled and ("cancel", 3) in kinds
    s = summarize(out, lambda r: 1.0)
    assert s["requests"] == 2 and s["cancelled"] == 2


def test_lane_caps_let_other_lanes_pass_and_keep_order_within_a_lane():
    clk = Clock()

    class LaneBackend(FakeBackend):
        # lane = mesh key; lane 2 runs one request at a time
        def can_admit(self, h):
            return h[1] != 2 or sum(1 for p in self.probs.values() if p["h"][1] == 2 and p["it"] < p["target"]) < 1

    be = LaneBackend(clk, budget=10_000)
    reqs = [_req(0, 0.0, 2, 30), _req(1, 0.0, 2, 30), _req(2, 0.0, 1, 5), _req(3, 0.0, 2, 30)]
    srv = Server(be, 10_000, clock=clk, sleep=clk.sleep)
    srv.run(reqs)
    admit = {rid: t for t, k, rid in srv.events if k == "admit"}
    done = {rid: t for t, k, rid in srv.events if k == "done"}
    # the small request passes the queued large ones; large ones run one at a time, in order
    assert admit[2] == admit[0]
    assert admit[1] >= done[0] and admit[3] >= done[1]
    order = [rid for _, k, rid in srv.events if k == "admit" and rid != 2]
    assert order == [0, 1, 3]


def test_face_record_sizes_and_handle_reservation():
    # records: Omega.A per face slot and an int32 neighbour id, padded to 16 bytes
    assert [face_record_bytes(f, 4) for f in (4, 5, 6, 7)] == [32, 48, 48, 64]
    assert [face_record_bytes(f, 8) for f in (4, 6, 7)] == [48, 80, 96]
    N, F, M, Fb = 1000, 2200, 48, 300
    batched = handle_resident_bytes(N, F, M, Fb, 4, 4, 1, solo=False)
    assert batched == (2 + 32) * M * N  # unit table and FP32 tet stream
    solo = handle_resident_bytes(N, F, M, Fb, 4, 4, 1, solo=True)
    # plus psi and its sweep-order copy (R = 1), source records (2 values) and two phi rows, inflow and
    # lagged psi, scratch
    assert solo - batched == 2 * M * N * 4 + N * (2 + 2) * 4 + (Fb + F) * 4 + (M + 8) * 8 + (1 << 20)
    # 3 rhs are padded to 4 for psi and the source records (8 values), phi keeps 3 rows
    s3 = handle_resident_bytes(N, F, M, Fb, 6, 8, 3, solo=True)
    assert s3 - handle_resident_bytes(N, F, M, Fb, 6, 8, 3, solo=False) == (
        2 * M * N * 4 * 8 + N * (8 + 6) * 8 + (Fb + F) * 4 * 8 + (M + 8) * 8 + (1 << 20))
