"""Serving loop: source-iteration requests on resident meshes, continuously batched.

Requests (a mesh from a catalog plus per-request materials and sources)
arrive over time.  The server

* keeps meshes and their dependency graphs resident on the device (built on
  first use, evicted least-recently-used when memory is needed and no active
  request uses them),
* admits waiting requests in arrival order whenever their memory (graph if
  not resident, the batch workspaces, the input and output arrays) fits the
  device-memory budget,
* advances every admitted request together, one batched launch per source
  iteration (jsweep_batch_step), so requests that arrive while others iterate
  join the next iteration (continuous batching),
* delivers each result to host memory when its request converges and frees
  its memory at once.

It reports per-request latency (arrival to result on the host), p50 / p99,
and throughput.  ``run_one_at_a_time`` serves the same stream with the plain
single-problem path (jsweep_source_iterate, one request after the other) as
the comparison.

The device work goes through a backend object (``GpuBackend`` for the real
library); the scheduling logic itself is host code and is tested with a fake
backend on the CPU.
"""

from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Any, Callable

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float               # seconds after the start of the stream
    mesh_key: Any                # key of the mesh in the catalog
    sigma_t: np.ndarray          # [N]
    c_ratio: np.ndarray          # [N]
    q: np.ndarray                # [R, N]
    # filled by the server
    admitted: float | None = None
    done: float | None = None
    iters: int | None = None
    resid: float | None = None
    phi: np.ndarray | None = None
    cancelled: bool = False

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class ResidentMeshes:
    """Meshes and graphs on the device, least recently used first."""

    def __init__(self):
        self.items = collections.OrderedDict()  # key -> (handle, bytes)
        self.in_use = collections.Counter()

    def get(self, key):
        if key in self.items:
            self.items.move_to_end(key)
            return self.items[key][0]
        return None

    def put(self, key, handle, nbytes):
        self.items[key] = (handle, int(nbytes))
        self.items.move_to_end(key)

    def bytes(self):
        return sum(b for _, b in self.items.values())

    def evictable(self):
        return [k for k in self.items if self.in_use[k] == 0]

    def evict(self, key):
        handle, nbytes = self.items.pop(key)
        return handle, nbytes


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * p / 100.0
    lo, hi = int(np.floor(k)), int(np.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


class Server:
    """Continuous-batching server over a backend (see ``GpuBackend``)."""

    def __init__(self, backend, budget_bytes: float, sweeps_per_step: int = 1,
                 clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep):
        self.be = backend
        self.budget = float(budget_bytes)
        self.k = int(sweeps_per_step)
        self.clock = clock
        self.sleep = sleep
        self.meshes = ResidentMeshes()
        self.active = {}          # pid -> (request, reserved bytes)
        self.reserved = 0.0       # bytes held by admitted requests
        self.peak_used = 0.0
        self.events = []          # (time, kind, rid)
        self.steps = 0

    def warm(self, keys):
        """Build and keep resident the meshes of `keys` (as far as the budget allows)."""
        for key in keys:
            if self.meshes.get(key) is None and self._make_room(self.be.mesh_bytes_estimate(key)):
                handle, nbytes = self.be.build_mesh(key)
                self.meshes.put(key, handle, nbytes)
        return self.meshes

    # memory held now: resident graphs + admitted requests
    def used(self):
        return self.meshes.bytes() + self.reserved

    def _make_room(self, need):
        """Evict unused resident meshes (LRU first) until `need` more bytes fit."""
        while self.used() + need > self.budget:
            cand = self.meshes.evictable()
            if not cand:
                return False
            handle, _ = self.meshes.evict(cand[0])
            self.be.release_mesh(handle)
        return True

    def _try_admit(self, req, now):
        """True if admitted; "memory" if it does not fit the budget now; "lane"
        if its lane already runs as many requests as it may."""
        key = req.mesh_key
        handle = self.meshes.get(key)
        mesh_need = 0 if handle is not None else self.be.mesh_bytes_estimate(key)
        if handle is None:
            if not self._make_room(mesh_need + self.be.request_bytes_estimate(key)):
                return "memory"
            handle, nbytes = self.be.build_mesh(key)
            self.meshes.put(key, handle, nbytes)
        if hasattr(self.be, "can_admit") and not self.be.can_admit(handle):
            return "lane"
        need = self.be.request_bytes(handle, req)
        self.meshes.in_use[key] += 1  # pin the mesh while making room for the request
        ok = self._make_room(need)
        if not ok:
            self.meshes.in_use[key] -= 1
            return "memory"
        pid = self.be.add(handle, req)
        self.active[pid] = (req, need)
        self.reserved += need
        self.peak_used = max(self.peak_used, self.used())
        req.admitted = now
        self.events.append((now, "admit", req.rid))
        return True

    def _finish(self, pid, now):
        req, need = self.active.pop(pid)
        req.phi, req.iters, req.resid = self.be.result(pid)
        self.be.remove(pid)
        self.reserved -= need
        self.meshes.in_use[req.mesh_key] -= 1
        req.done = self.clock() - self._t0
        self.events.append((req.done, "done", req.rid))

    def _cancel(self, rid, waiting, now):
        """Drop request `rid`: out of the queue if it waits, out of the batch
        (memory freed at once) if it iterates; a finished request is kept."""
        for r in list(waiting):
            if r.rid == rid:
                waiting.remove(r)
                r.cancelled = True
                self.events.append((now, "cancel", rid))
                return
        for pid, (req, need) in list(self.active.items()):
            if req.rid == rid:
                self.be.remove(pid)
                del self.active[pid]
                self.reserved -= need
                self.meshes.in_use[req.mesh_key] -= 1
                req.cancelled = True
                self.events.append((now, "cancel", rid))
                return

    def run(self, requests, cancels=()):
        """Serve `requests` (sorted by arrival) in real time; returns them
        filled.  `cancels` lists (time, request id): the client gives up on
        that request at that time."""
        cancels = sorted(cancels)
        nc = 0
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            need = self.be.mesh_bytes_estimate(r.mesh_key) + self.be.request_bytes_estimate(r.mesh_key)
            if need > self.budget:
                raise ValueError(f"request {r.rid} needs {need:.3g} bytes, more than the budget {self.budget:.3g}")
        nxt = 0
        waiting = collections.deque()
        self._t0 = self.clock()
        while nxt < len(reqs) or waiting or self.active:
            now = self.clock() - self._t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                waiting.append(reqs[nxt])
                nxt += 1
            while nc < len(cancels) and cancels[nc][0] <= now:
                self._cancel(cancels[nc][1], waiting, now)
                nc += 1
            # admission in arrival order: a request whose lane is full lets later
            # requests of other lanes pass; one that does not fit in memory stops
            # the scan (so a large request is not starved by small ones)
            for req in list(waiting):
                res = self._try_admit(req, now)
                if res is True:
                    waiting.remove(req)
                elif res == "memory":
                    if not self.active:
                        raise RuntimeError(f"request {req.rid} does not fit the budget even when idle")
                    break
            if self.active:
                if hasattr(self.be, "pump"):
                    self.be.pump(self.k)  # returns once some lane has finished an iteration
                else:
                    self.be.step(self.k)
                self.steps += 1
                now = self.clock() - self._t0
                for pid in list(self.active):
                    if self.be.finished(pid):
                        self._finish(pid, now)
            elif nxt < len(reqs):
                self.sleep(max(0.0, reqs[nxt].arrival - (self.clock() - self._t0)))
        return reqs


def run_one_at_a_time(backend, requests, clock=time.perf_counter, sleep=time.sleep, budget_bytes=None,
                      meshes=None):
    """The comparison: the plain single-problem GPU path, one request after the
    other in arrival order (meshes stay resident as in the server; `meshes`
    may hand over the server's resident set)."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    meshes = meshes if meshes is not None else ResidentMeshes()
    t0 = clock()
    for r in reqs:
        now = clock() - t0
        if r.arrival > now:
            sleep(r.arrival - now)
        handle = meshes.get(r.mesh_key)
        if handle is None:
            need = backend.mesh_bytes_estimate(r.mesh_key) + backend.request_bytes_estimate(r.mesh_key)
            while budget_bytes is not None and meshes.items and meshes.bytes() + need > budget_bytes:
                h, _ = meshes.evict(next(iter(meshes.items)))
                backend.release_mesh(h)
            handle, nbytes = backend.build_mesh(r.mesh_key)
            meshes.put(r.mesh_key, handle, nbytes)
        r.admitted = clock() - t0
        r.phi, r.iters, r.resid = backend.solve_alone(handle, r)
        r.done = clock() - t0
    return reqs


def summarize(reqs, cell_dir_updates: Callable[[Request], float]):
    """Latency percentiles and throughput over the requests that finished."""
    done = [r for r in reqs if r.done is not None]
    lat = [r.latency for r in done]
    t_end = max(r.done for r in done)
    t_start = min(r.arrival for r in reqs)
    work = sum(cell_dir_updates(r) for r in done)
    return {"requests": len(done), "cancelled": sum(r.cancelled for r in reqs),
            "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
            "mean_s": float(np.mean(lat)), "max_s": max(lat), "makespan_s": t_end - t_start,
            "requests_per_s": len(reqs) / (t_end - t_start),
            "cell_angle_updates_per_s": work / (t_end - t_start)}


def face_record_bytes(faces_per_cell: int, elem_bytes: int) -> int:
    """Bytes of one face-coefficient record of a handle's stream: Omega.A of
    every face slot (4 slots up to 4 faces, 6 up to 6, else 7) and the slot's
    neighbour id (int32), padded to 16 bytes."""
    slots = 4 if faces_per_cell <= 4 else 6 if faces_per_cell <= 6 else 7
    return -(-(slots * elem_bytes + slots * 4) // 16) * 16


def handle_resident_bytes(n_cells: int, n_faces: int, n_dirs: int, n_bfaces: int, faces_per_cell: int,
                          elem_bytes: int, nrhs: int, solo: bool) -> int:
    """Device bytes a handle allocates at its first solve and keeps while it
    lives: its own unit table (one 16-byte unit per 8 or more (direction,
    cell) pairs, 2 bytes per pair), its face-coefficient stream (one record
    per pair), and, when its requests run through jsweep_source_iterate (the
    solo lane), that call's sweep state: psi and its copy in sweep order,
    source records, phi ping-pong, inflow and lagged psi, the residual and
    counter scratch and 1 MiB of slack."""
    N, F, M = n_cells, n_faces, n_dirs
    extra = (2 + face_record_bytes(faces_per_cell, elem_bytes)) * M * N
    if solo:
        R = 1 if nrhs <= 1 else 2 if nrhs <= 2 else 4 if nrhs <= 4 else 8
        RS = 2 * R if R >= 4 else (4 if R == 2 else 2)
        extra += (2 * M * N * R * elem_bytes + N * (RS + 2 * nrhs) * elem_bytes
                  + (max(n_bfaces, 1) + F) * R * elem_bytes + (M + 8) * 8 + (1 << 20))
    return extra


class GpuBackend:
    """The library's C ABI: graphs from jsweep_build_dags, requests in jsweep
    batches, the comparison through jsweep_source_iterate.

    Requests are split by work per iteration (cells x directions) into lanes,
    one batch and one CUDA stream per lane (``lanes`` gives the upper bounds
    of all lanes but the last).  A small request then iterates at the pace of
    the small requests, not of the largest mesh in the mix; the lanes run
    concurrently on the device (jsweep_batch_launch / jsweep_batch_poll).
    ``lane_caps`` bounds how many requests a lane runs at once.
    """

    def __init__(self, catalog: Callable[[Any], tuple], dtype=None, nrhs=1, tol=1e-6, max_iters=1000,
                 options=None, batch_options=None, lanes=(3e6, 3e7), lane_caps=(None, 8, 1), solo_last_lane=True):
        import torch

        from . import jsweep as J
        self.J = J
        self.torch = torch
        self.catalog = catalog  # key -> (mesh dict, dirs, weights)
        self.dtype = dtype or torch.float32
        self.nrhs = nrhs
        self.tol = tol
        self.max_iters = max_iters
        self.options = options
        self.bounds = list(lanes)
        n = len(self.bounds) + 1
        # requests a lane runs at once (None: no limit): small requests gain most
        # from sharing iterations; large ones keep the device to themselves and
        # finish in arrival order instead of all finishing late together
        self.caps = list(lane_caps) + [None] * max(0, n - len(lane_caps))
        # the largest requests gain nothing from sharing iterations: the last lane
        # runs them through jsweep_source_iterate on its own stream, in a worker
        # thread (the C calls release the interpreter), beside the batched lanes
        self.solo_lane = n - 1 if solo_last_lane else None
        self.solo_jobs = {}
        self._solo_next = 0
        self.batches = [J.Batch(self.dtype, nrhs, batch_options) for _ in range(n)]
        self.streams = [torch.cuda.Stream() for _ in range(n)]
        self.active = [0] * n      # unfinished problems per lane
        self.pending = [False] * n
        self.inputs = {}
        self._est = {}
        self.builds = 0

    @property
    def batch(self):  # the first lane (kept for single-lane use)
        return self.batches[0]

    def can_admit(self, handle):
        lane = self.lane_of(handle)
        return self.caps[lane] is None or self.active[lane] < self.caps[lane]

    def _lane_of_work(self, work):
        for i, b in enumerate(self.bounds):
            if work < b:
                return i
        return len(self.bounds)

    def lane_of(self, handle):
        return self._lane_of_work(handle.n_cells * handle.n_dirs)

    # sizes
    def _shape(self, key):
        if key not in self._est:
            mesh, dirs, _ = self.catalog(key)
            fc = np.asarray(mesh["face_cells"]).ravel()
            fs = int(np.bincount(fc[fc >= 0]).max()) if fc.size else 1
            self._est[key] = (mesh["n_cells"], mesh["n_faces"], len(dirs), mesh.get("n_bfaces", 0), fs)
        return self._est[key]

    def _rhs_padded(self):
        return 1 if self.nrhs <= 1 else 2 if self.nrhs <= 2 else 4 if self.nrhs <= 4 else 8

    def resident_extra_bytes(self, key):
        """Device bytes a mesh's handle allocates at its first solve and keeps
        until it is released, reserved with the mesh (handle_resident_bytes)."""
        N, F, M, Fb, FS = self._shape(key)
        es = 8 if self.dtype == self.torch.float64 else 4
        solo = self.solo_lane is not None and self._lane_of_work(N * M) == self.solo_lane
        return handle_resident_bytes(N, F, M, Fb, FS, es, self.nrhs, solo)

    def mesh_bytes_estimate(self, key):
        """Device bytes of a mesh and its graphs while they are being built
        (an upper bound of the peak): the per-(direction, cell) arrays of the
        graph build (levels, orders, masks, peel and cycle-search state, sort
        buffers; 92 bytes per pair measured on a 82,944-tet, 128-direction
        mesh, 16.5 bytes of which stay resident) and the per-cell and
        per-face mesh arrays."""
        N, F, M, _, _ = self._shape(key)
        return 104 * M * N + 256 * N + 64 * F + (64 << 20) + self.resident_extra_bytes(key)

    def request_bytes_estimate(self, key):
        """Batch workspaces (psi and its sweep-order copy, epoch flags, source
        records, phi), inputs and output, and the request's share of the
        merged unit table (at most one 20-byte unit per 8 (direction, cell)
        pairs, plus the handle's own table)."""
        N, F, M, _, _ = self._shape(key)
        es = 8 if self.dtype == self.torch.float64 else 4
        R = self._rhs_padded()
        return M * N * (2 * R * es + 4 + 5) + N * (2 * R + 3 * self.nrhs + 4) * es + F * R * es + (1 << 20)

    def build_mesh(self, key):
        torch = self.torch
        mesh, dirs, w = self.catalog(key)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        m = self.J.mesh_from_dict(mesh)
        qd = self.J.jsweep_quadrature_create(dirs, w)
        g = self.J.jsweep_build_dags(m, qd, self.options)
        torch.cuda.synchronize()
        self.builds += 1
        return g, torch.cuda.memory_allocated() - before + self.resident_extra_bytes(key)

    def release_mesh(self, handle):
        del handle  # the handle's destructor releases it (batch problems hold their own reference)

    def request_bytes(self, handle, req):
        es = 8 if self.dtype == self.torch.float64 else 4
        io = (2 * handle.n_cells + 2 * req.q.size) * es  # sigma_t, c, q, phi_out
        lane = self.lane_of(handle)
        if lane == self.solo_lane:
            return io  # the sweep state stays on the handle, reserved with the mesh
        tables = 3 * handle.n_dirs * handle.n_cells  # the request's share of the merged unit table
        return self.batches[lane].problem_bytes(handle) + io + tables

    def _tensors(self, req):
        t = self.torch
        dev = "cuda"
        sig = t.as_tensor(np.ascontiguousarray(req.sigma_t), dtype=self.dtype).pin_memory().to(dev, non_blocking=True)
        c = t.as_tensor(np.ascontiguousarray(req.c_ratio), dtype=self.dtype).pin_memory().to(dev, non_blocking=True)
        q = t.as_tensor(np.ascontiguousarray(req.q), dtype=self.dtype).pin_memory().to(dev, non_blocking=True)
        return sig, c, q

    def _solo_run(self, job, handle, req, stream):
        torch = self.torch
        try:
            with torch.cuda.stream(stream):
                sig, c, q = self._tensors(req)
                phi, it, res, ok = self.J.jsweep_source_iterate(handle, sig, c, q, tol=self.tol,
                                                                max_iters=self.max_iters, stream=stream,
                                                                allow_not_converged=True)
                job["result"] = (phi.cpu().numpy(), it, res)
        except Exception as e:  # reported by result()
            job["error"] = e
        job["done"] = True

    def add(self, handle, req):
        lane = self.lane_of(handle)
        if lane == self.solo_lane:
            pid = ("solo", self._solo_next)
            self._solo_next += 1
            job = {"done": False, "result": None, "error": None, "stream": self.streams[lane]}
            job["thread"] = threading.Thread(target=self._solo_run, args=(job, handle, req, self.streams[lane]),
                                             daemon=True)
            self.solo_jobs[pid] = job
            self.inputs[pid] = req
            self.active[lane] += 1
            job["thread"].start()
            return pid
        sig, c, q = self._tensors(req)
        pid = (lane, self.batches[lane].add(handle, sig, c, q, tol=self.tol, max_iters=self.max_iters))
        self.inputs[pid] = req
        self.active[lane] += 1
        return pid

    def step(self, k):
        for lane in range(len(self.batches)):
            if self.active[lane] and lane != self.solo_lane:
                self.active[lane] = self.batches[lane].step(k, stream=self.streams[lane])

    def pump(self, k, spin_s=20e-6):
        """Keep every lane with unfinished problems busy; return once at least
        one lane has finished its queued iterations."""
        while True:
            for lane, b in enumerate(self.batches):
                if lane != self.solo_lane and self.active[lane] and not self.pending[lane]:
                    b.launch(k, stream=self.streams[lane])
                    self.pending[lane] = True
            progressed = False
            for lane, b in enumerate(self.batches):
                if self.pending[lane]:
                    done, n = b.poll()
                    if done:
                        self.pending[lane] = False
                        self.active[lane] = n
                        progressed = True
            if any(j["done"] and not j.get("seen") for j in self.solo_jobs.values()):
                for j in self.solo_jobs.values():
                    j["seen"] = j["done"]
                progressed = True
            if progressed or not (any(self.pending) or self.solo_jobs):
                return
            time.sleep(spin_s)

    def finished(self, pid):
        if pid in self.solo_jobs:
            return self.solo_jobs[pid]["done"]
        lane, i = pid
        return self.batches[lane].query(i)[0] != self.J.JSWEEP_PROBLEM_ACTIVE

    def result(self, pid):
        if pid in self.solo_jobs:
            job = self.solo_jobs[pid]
            job["thread"].join()
            if job["error"] is not None:
                raise job["error"]
            return job["result"]
        lane, i = pid
        st, it, res = self.batches[lane].query(i)
        phi = self.batches[lane].phi(i).cpu().numpy()  # written by the lane's finished iteration
        return phi, it, res

    def remove(self, pid):
        if pid in self.solo_jobs:
            job = self.solo_jobs.pop(pid)
            job["thread"].join()  # a cancelled solve runs to its end; its result is dropped
            self.active[self.solo_lane] -= 1
            self.inputs.pop(pid, None)
            return
        lane, i = pid
        if self.pending[lane]:
            done, n = self.batches[lane].poll(wait=True)
            self.pending[lane] = False
            self.active[lane] = n
        was_active = self.batches[lane].query(i)[0] == self.J.JSWEEP_PROBLEM_ACTIVE
        self.batches[lane].remove(i)
        if was_active:
            self.active[lane] = max(0, self.active[lane] - 1)
        self.inputs.pop(pid, None)

    def solve_alone(self, handle, req):
        sig, c, q = self._tensors(req)
        phi, it, res, ok = self.J.jsweep_source_iterate(handle, sig, c, q, tol=self.tol, max_iters=self.max_iters,
                                                        allow_not_converged=True)
        return phi.cpu().numpy(), it, res


def poisson_stream(n_requests, rate_per_s, catalog_keys, make_inputs, seed=5000):
    """Seeded Poisson arrivals; each request draws a catalog mesh uniformly and
    its inputs from make_inputs(key, request seed)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    keys = rng.integers(0, len(catalog_keys), n_requests)
    out = []
    for i in range(n_requests):
        key = catalog_keys[int(keys[i])]
        sig, c, q = make_inputs(key, seed * 1000 + i)
        out.append(Request(rid=i, arrival=float(t[i]), mesh_key=key, sigma_t=sig, c_ratio=c, q=q))
    return out


__all__ = ["Request", "Server", "GpuBackend", "run_one_at_a_time", "summarize", "poisson_stream", "percentile",
           "ResidentMeshes"]
