"""FP64 CPU oracle of the S_n sweep path (TEST INFRASTRUCTURE ONLY).

The oracle is the plain, slow, obviously correct reference the GPU library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the library never does, and the
oracle never imports the library.  Its arithmetic lives in
``jsweep_oracle.c`` (plain C, FP64, compiled with ``-ffp-contract=off``) and
``quadrature.py``; this module only builds and wraps it.

Parity pins (tests/test_oracle_*.py) tie it to the paper and to mathematics:
the 1D upwind recurrence, the uniform-solution invariant, a dense linear
solve of the discrete system, brute-force levels, a hand-worked cyclic mesh,
quadrature moments, and for the multigroup iteration its one-group and
uncoupled limits, an infinite-medium fixed point and a dense block solve.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .quadrature import product_quadrature  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jsweep_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libjsweep_oracle.so")
_lock = threading.Lock()
_lib = None

OD_OK, OD_NOT_CONVERGED = 0, 1

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.od_build_dags.restype = _p
            lib.od_build_dags.argtypes = [_i64, _i64, _p, _p, _p, _p, _i64, _p, _p]
            lib.od_free.argtypes = [_p]
            for name in ("od_nlevels", "od_nlag"):
                getattr(lib, name).restype = _i64
                getattr(lib, name).argtypes = [_p, _i64]
            for name in ("od_nlag_total", "od_n_bfaces"):
                getattr(lib, name).restype = _i64
                getattr(lib, name).argtypes = [_p]
            lib.od_levels.argtypes = [_p, _i64, _p]
            lib.od_order.argtypes = [_p, _i64, _p, _p]
            lib.od_lagged.argtypes = [_p, _i64, _p]
            lib.od_sweep.restype = ctypes.c_int
            lib.od_sweep.argtypes = [_p, _i64, _p, _p, _p, _p, _p, _p, _p, _p, _i64, ctypes.c_int]
            lib.od_source_iterate.restype = ctypes.c_int
            lib.od_source_iterate.argtypes = [_p, _i64, _p, _p, _p, _p, _p, ctypes.c_double, _i64,
                                              _p, _p, _p, _p, ctypes.c_int]
            lib.od_source_iterate_mg.restype = ctypes.c_int
            lib.od_source_iterate_mg.argtypes = [_p, _i64, _p, _p, _p, _p, _p, ctypes.c_double, _i64,
                                                 _p, _p, _p, _p, ctypes.c_int]
            lib.od_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(_load().od_max_threads())


class OracleDags:
    """Per-direction dependency graphs of one mesh (levels, order, lagged faces)."""

    def __init__(self, mesh, dirs):
        lib = _load()
        self._lib = lib
        self.n_cells = int(mesh["n_cells"])
        self.n_faces = int(mesh["n_faces"])
        self.dirs = _f64(dirs).reshape(-1, 3)
        self.n_dirs = self.dirs.shape[0]
        self._keep = [np.ascontiguousarray(mesh["face_cells"], dtype=np.int64),
                      _f64(mesh["normals"]), _f64(mesh["areas"]), _f64(mesh["volumes"]), self.dirs]
        st = ctypes.c_int(0)
        h = lib.od_build_dags(self.n_cells, self.n_faces, *[_ptr(a) for a in self._keep[:4]],
                              self.n_dirs, _ptr(self.dirs), ctypes.byref(st))
        if not h:
            raise RuntimeError(f"oracle dag build failed (status {st.value})")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.od_free(self._h)
            self._h = None

    @property
    def n_bfaces(self) -> int:
        return int(self._lib.od_n_bfaces(self._h))

    @property
    def n_lag_total(self) -> int:
        return int(self._lib.od_nlag_total(self._h))

    def nlevels(self, m: int) -> int:
        return int(self._lib.od_nlevels(self._h, m))

    def levels(self, m: int) -> np.ndarray:
        out = np.empty(self.n_cells, dtype=np.int32)
        self._lib.od_levels(self._h, m, _ptr(out))
        return out

    def order(self, m: int):
        order = np.empty(self.n_cells, dtype=np.int32)
        ptr = np.empty(self.nlevels(m) + 1, dtype=np.int32)
        self._lib.od_order(self._h, m, _ptr(order), _ptr(ptr))
        return order, ptr

    def lagged(self, m: int) -> np.ndarray:
        n = int(self._lib.od_nlag(self._h, m))
        out = np.empty((n, 3), dtype=np.int64)
        if n:
            self._lib.od_lagged(self._h, m, _ptr(out))
        return out

    def sweep(self, sigma_t, src, weights, inflow=None, psi_lag=None, dir_list=None,
              want_psi=False, nthreads=1):
        """One sweep; returns (phi [R, N], psi [R, n_dirs_swept, N] or None, psi_lag)."""
        src = _f64(src)
        src = src.reshape(-1, self.n_cells)
        R = src.shape[0]
        sig = _f64(sigma_t)
        w = _f64(weights)
        inf = None if inflow is None else _f64(inflow).reshape(R, self.n_bfaces)
        T = self.n_lag_total
        lag = np.zeros((R, T)) if psi_lag is None else _f64(psi_lag).reshape(R, T).copy()
        dl = None if dir_list is None else np.ascontiguousarray(dir_list, dtype=np.int64)
        nl = self.n_dirs if dl is None else dl.size
        phi = np.empty((R, self.n_cells))
        psi = np.empty((R, nl, self.n_cells)) if want_psi else None
        rc = self._lib.od_sweep(self._h, R, _ptr(sig), _ptr(src), _ptr(inf), _ptr(w), _ptr(lag),
                                _ptr(phi), _ptr(psi), _ptr(dl), nl, int(nthreads))
        if rc != OD_OK:
            raise RuntimeError(f"oracle sweep failed ({rc})")
        return phi, psi, lag

    def source_iterate(self, sigma_t, c_ratio, q, weights, tol, max_iters, inflow=None,
                       nthreads=1):
        """Source iteration from phi = 0; returns (phi, iters, resid, converged, history)."""
        q = _f64(q).reshape(-1, self.n_cells)
        R = q.shape[0]
        inf = None if inflow is None else _f64(inflow).reshape(R, self.n_bfaces)
        phi = np.empty((R, self.n_cells))
        it = ctypes.c_int64(0)
        res = ctypes.c_double(0.0)
        hist = np.zeros(max(int(max_iters), 1))
        sig, cr, w = _f64(sigma_t), _f64(c_ratio), _f64(weights)
        rc = self._lib.od_source_iterate(self._h, R, _ptr(sig), _ptr(cr), _ptr(q), _ptr(inf),
                                         _ptr(w), float(tol), int(max_iters), _ptr(phi),
                                         ctypes.byref(it), ctypes.byref(res), _ptr(hist),
                                         int(nthreads))
        if rc not in (OD_OK, OD_NOT_CONVERGED):
            raise RuntimeError(f"oracle source iteration failed ({rc})")
        return phi, int(it.value), float(res.value), rc == OD_OK, hist[: it.value]


    def multigroup_source_iterate(self, sigma_t, sigma_s, q, weights, tol, max_iters, inflow=None,
                                  nthreads=1):
        """Multigroup source iteration from phi = 0 (the appendix's transport
        equation over energy groups, Alg. 1): every iteration forms each
        group's scattering source from the previous iterate of all groups,
        S_g = (sum_h sigma_s[h, g] phi_h + q_g) / (4 pi), sweeps each group with
        its own sigma_t, and stops when every group's relative max-norm change
        is below tol.  sigma_t [G, N]; sigma_s [G, G, N] with [h, g] the rate
        from group h into group g; q [G, N]; inflow [G, n_bfaces] or None.
        Returns (phi [G, N], iters, resid, converged, history)."""
        sig = _f64(sigma_t).reshape(-1, self.n_cells)
        G = sig.shape[0]
        ss = _f64(sigma_s).reshape(G, G, self.n_cells)
        q = _f64(q).reshape(G, self.n_cells)
        inf = None if inflow is None else _f64(inflow).reshape(G, self.n_bfaces)
        w = _f64(weights)
        phi = np.empty((G, self.n_cells))
        it = ctypes.c_int64(0)
        res = ctypes.c_double(0.0)
        hist = np.zeros(max(int(max_iters), 1))
        rc = self._lib.od_source_iterate_mg(self._h, G, _ptr(sig), _ptr(ss), _ptr(q), _ptr(inf), _ptr(w),
                                            float(tol), int(max_iters), _ptr(phi), ctypes.byref(it),
                                            ctypes.byref(res), _ptr(hist), int(nthreads))
        if rc not in (OD_OK, OD_NOT_CONVERGED):
            raise RuntimeError(f"oracle multigroup source iteration failed ({rc})")
        return phi, int(it.value), float(res.value), rc == OD_OK, hist[: it.value]


def build_dags(mesh, dirs) -> OracleDags:
    return OracleDags(mesh, dirs)
