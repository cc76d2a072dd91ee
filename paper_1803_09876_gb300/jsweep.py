"""Thin Python binding of the jsweep C ABI (``include/jsweep.h``).

Argument marshalling only: every step of the sweep path runs in the CUDA
library ``libjsweep.so``.  Host arrays are numpy arrays; device arrays are
CUDA torch tensors (their ``data_ptr()`` is passed through) and the stream is
torch's current stream.  PyTorch also provides the library's own device
memory (its caching allocator is installed with ``jsweep_set_allocator``).

There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""

from __future__ import annotations

import atexit
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjsweep.so")

JSWEEP_OK = 0
JSWEEP_ERR_INVALID_ARG = -1
JSWEEP_ERR_MESH_INVALID = -2
JSWEEP_ERR_OOM = -3
JSWEEP_ERR_NOT_CONVERGED = -4
JSWEEP_ERR_DEVICE_TIMEOUT = -5
JSWEEP_ERR_CUDA = -6
JSWEEP_ERR_UNIMPLEMENTED = -7
JSWEEP_ERR_CYCLE = -8

JSWEEP_F64 = 0
JSWEEP_F32 = 1

JSWEEP_MODE_AUTO = 0
JSWEEP_MODE_LEVEL_SYNC = 1
JSWEEP_MODE_PERSISTENT = 2
JSWEEP_MODE_PATCH = 3

JSWEEP_LAYERS_OCTANT = 0
JSWEEP_LAYERS_LEVEL = 1

JSWEEP_PRIO_LEVEL = 0
JSWEEP_PRIO_DEPTH = 1
JSWEEP_PRIO_OCTANT = 2
JSWEEP_PRIO_PATCH = 3
JSWEEP_PRIO_PATCH_SLBD = 4

# every symbol include/jsweep.h declares
EXPORTED = [
    "jsweep_options_default", "jsweep_last_error", "jsweep_version", "jsweep_set_allocator",
    "jsweep_mesh_create", "jsweep_mesh_destroy", "jsweep_mesh_info",
    "jsweep_quadrature_product", "jsweep_quadrature_create", "jsweep_quadrature_destroy",
    "jsweep_build_dags", "jsweep_dags_destroy", "jsweep_dags_info", "jsweep_dags_nlevels",
    "jsweep_dags_levels", "jsweep_dags_order", "jsweep_dags_schedule", "jsweep_dags_lagged", "jsweep_dags_reset_lag",
    "jsweep_dags_set_options", "jsweep_sweep", "jsweep_source_iterate", "jsweep_dags_timing",
    "jsweep_source_iterate_noalloc", "jsweep_source_iterate_mg", "jsweep_bounds_checked", "jsweep_bounds_error",
    "jsweep_batch_create", "jsweep_batch_problem_bytes", "jsweep_batch_add", "jsweep_batch_step",
    "jsweep_batch_launch", "jsweep_batch_poll",
    "jsweep_batch_query", "jsweep_batch_remove", "jsweep_batch_clear", "jsweep_batch_size",
    "jsweep_batch_source_iterate", "jsweep_batch_autotune", "jsweep_batch_stats", "jsweep_batch_options",
    "jsweep_batch_destroy",
]


class JsweepError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"jsweep error {code}: {msg}")
        self.code = code


class jsweep_options(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int),
        ("sweep_mode", ctypes.c_int),
        ("priority", ctypes.c_int),
        ("cluster_cells", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int),
        ("octant_stagger", ctypes.c_int),
        ("spin_timeout_s", ctypes.c_double),
        ("cycle_search_max", ctypes.c_int),
        ("debug_block_waits", ctypes.c_int),
        ("layering", ctypes.c_int),
        ("angles_per_warp", ctypes.c_int),
        ("unit_order", ctypes.c_int),
        ("patch_cells", ctypes.c_int),
        ("eager_search_max", ctypes.c_int),
        ("no_face_stream", ctypes.c_int),
        ("tail_units", ctypes.c_int),
        ("no_sweep_order_psi", ctypes.c_int),
    ]


class jsweep_timing(ctypes.Structure):
    _fields_ = [
        ("build_ms", ctypes.c_double),
        ("sweep_ms", ctypes.c_double),
        ("phi_ms", ctypes.c_double),
        ("sweep_launches", ctypes.c_int64),
        ("build_launches", ctypes.c_int64),
        ("call_launches", ctypes.c_int64),
        ("build_steps", ctypes.c_int64),
        ("build_stall_rounds", ctypes.c_int64),
        ("build_phase_ms", ctypes.c_double * 6),
        ("sweep_programs", ctypes.c_int64),
        ("sweep_requeues", ctypes.c_int64),
    ]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None
_callbacks = None
# Every allocator ever installed stays referenced: a device buffer is released
# through the free function of the allocator that produced it, which must
# therefore outlive the buffer (see jsweep_set_allocator).
_installed = []
_exiting = False


def _at_exit():
    # Handles still alive at interpreter exit are left to the process teardown:
    # releasing them would call back into Python (torch's allocator) while it
    # shuts down.
    global _exiting
    _exiting = True


atexit.register(_at_exit)


def _live():
    return _lib is not None and not _exiting


def load(path: str = LIB_PATH):
    """Load libjsweep.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_1803_09876_gb300.build.build() "
                              "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(path)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sig = {
            "jsweep_options_default": (I, [P]),
            "jsweep_last_error": (ctypes.c_char_p, []),
            "jsweep_version": (I, []),
            "jsweep_set_allocator": (I, [P, P, P]),
            "jsweep_mesh_create": (I, [I64, I64, P, P, P, P, P]),
            "jsweep_mesh_destroy": (I, [P]),
            "jsweep_mesh_info": (I, [P, P, P, P, P]),
            "jsweep_quadrature_product": (I, [I, I, P, P]),
            "jsweep_quadrature_create": (I, [I64, P, P, P]),
            "jsweep_quadrature_destroy": (I, [P]),
            "jsweep_build_dags": (I, [P, P, P, P, P]),
            "jsweep_dags_destroy": (I, [P]),
            "jsweep_dags_info": (I, [P, P, P, P]),
            "jsweep_dags_nlevels": (I, [P, I64, P]),
            "jsweep_dags_levels": (I, [P, I64, P]),
            "jsweep_dags_order": (I, [P, I64, P, P]),
            "jsweep_dags_schedule": (I, [P, I64, P, P, P]),
            "jsweep_dags_lagged": (I, [P, I64, P, P]),
            "jsweep_dags_reset_lag": (I, [P]),
            "jsweep_dags_set_options": (I, [P, P]),
            "jsweep_sweep": (I, [P, I, I, P, P, P, P, P, P]),
            "jsweep_source_iterate": (I, [P, I, I, P, P, P, P, ctypes.c_double, I, P, P, P, P]),
            "jsweep_dags_timing": (I, [P, P]),
            "jsweep_source_iterate_noalloc": (I, [P, I, I, P, P, P, P, ctypes.c_double, I, P, P, P, P]),
            "jsweep_source_iterate_mg": (I, [P, I, I, P, P, P, P, ctypes.c_double, I, P, P, P, P]),
            "jsweep_bounds_checked": (I, []),
            "jsweep_bounds_error": (I, [P]),
            "jsweep_batch_create": (I, [I, I, P, P]),
            "jsweep_batch_problem_bytes": (I, [P, P, I, P]),
            "jsweep_batch_add": (I, [P, P, P, P, P, P, P, ctypes.c_double, I, P, P]),
            "jsweep_batch_step": (I, [P, I, P, P]),
            "jsweep_batch_launch": (I, [P, I, P]),
            "jsweep_batch_poll": (I, [P, I, P, P]),
            "jsweep_batch_query": (I, [P, I64, P, P, P]),
            "jsweep_batch_remove": (I, [P, I64]),
            "jsweep_batch_clear": (I, [P]),
            "jsweep_batch_size": (I, [P, P]),
            "jsweep_batch_source_iterate": (I, [P, P, P, P]),
            "jsweep_batch_autotune": (I, [P, P, P]),
            "jsweep_batch_stats": (I, [P, P, P, P, P, P]),
            "jsweep_batch_options": (I, [P, P]),
            "jsweep_batch_destroy": (I, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def lib():
    return load()


def _check(code, what=""):
    if code != JSWEEP_OK:
        msg = lib().jsweep_last_error().decode(errors="replace")
        raise JsweepError(code, f"{what}: {msg}" if what else msg)
    return code


def use_torch_allocator():
    """Route the library's own device allocations through torch's caching allocator."""
    global _callbacks
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          torch.cuda.current_stream()))
        except Exception:  # out of memory: the library reports JSWEEP_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    cbs = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    set_allocator(*cbs)
    _callbacks = cbs


def set_allocator(alloc_cb, free_cb):
    """Install ctypes allocator callbacks (_ALLOC_FN, _FREE_FN); they are kept
    alive for the rest of the process."""
    _installed.append((alloc_cb, free_cb))
    _check(lib().jsweep_set_allocator(ctypes.cast(alloc_cb, ctypes.c_void_p),
                                      ctypes.cast(free_cb, ctypes.c_void_p), None), "set_allocator")


def jsweep_options_default(**overrides) -> jsweep_options:
    o = jsweep_options()
    _check(lib().jsweep_options_default(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def jsweep_version() -> int:
    return int(lib().jsweep_version())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype, n, what):
    """Device pointer of a contiguous CUDA tensor with exactly n elements."""
    if t is None:
        return None
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{what}: need a contiguous {dtype} tensor of {n} elements, "
                         f"got {t.dtype} {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """Handle of a mesh on the device (jsweep_mesh_create)."""

    def __init__(self, handle):
        self._h = handle
        n, f, b, fs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().jsweep_mesh_info(self._h, ctypes.byref(n), ctypes.byref(f), ctypes.byref(b), ctypes.byref(fs)))
        self.n_cells, self.n_faces, self.n_bfaces, self.max_faces = n.value, f.value, b.value, fs.value

    def __del__(self):
        if getattr(self, "_h", None) and _live():
            _lib.jsweep_mesh_destroy(self._h)
            self._h = None


class Quad:
    """Handle of a direction set (jsweep_quadrature_create)."""

    def __init__(self, handle, dirs, weights):
        self._h = handle
        self.dirs = dirs
        self.weights = weights
        self.n_dirs = dirs.shape[0]

    def __del__(self):
        if getattr(self, "_h", None) and _live():
            _lib.jsweep_quadrature_destroy(self._h)
            self._h = None


class Dags:
    """Per-direction dependency graphs resident on the device (jsweep_build_dags)."""

    def __init__(self, handle, mesh, quad):
        self._h = handle
        self.mesh = mesh
        self.quad = quad
        M, L, T = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().jsweep_dags_info(self._h, ctypes.byref(M), ctypes.byref(L), ctypes.byref(T)))
        self.n_dirs, self.max_levels, self.n_lag_total = M.value, L.value, T.value
        self.n_cells = mesh.n_cells

    def __del__(self):
        if getattr(self, "_h", None) and _live():
            _lib.jsweep_dags_destroy(self._h)
            self._h = None

    def nlevels(self, m: int) -> int:
        out = ctypes.c_int64()
        _check(lib().jsweep_dags_nlevels(self._h, int(m), ctypes.byref(out)))
        return out.value

    def levels(self, m: int) -> np.ndarray:
        out = np.empty(self.n_cells, dtype=np.int32)
        _check(lib().jsweep_dags_levels(self._h, int(m), _ptr(out)))
        return out

    def order(self, m: int):
        order = np.empty(self.n_cells, dtype=np.int32)
        ptr = np.empty(self.nlevels(m) + 1, dtype=np.int32)
        _check(lib().jsweep_dags_order(self._h, int(m), _ptr(order), _ptr(ptr)))
        return order, ptr

    def schedule(self, m: int):
        """(order [n_cells], layer_ptr [n_layers + 1]) of the layers the sweeps of direction m run."""
        n = ctypes.c_int64()
        _check(lib().jsweep_dags_schedule(self._h, int(m), ctypes.byref(n), None, None))
        order = np.empty(self.n_cells, dtype=np.int32)
        ptr = np.empty(n.value + 1, dtype=np.int32)
        _check(lib().jsweep_dags_schedule(self._h, int(m), ctypes.byref(n), _ptr(order), _ptr(ptr)))
        return order, ptr

    def lagged(self, m: int) -> np.ndarray:
        n = ctypes.c_int64()
        _check(lib().jsweep_dags_lagged(self._h, int(m), None, ctypes.byref(n)))
        rows = np.empty((n.value, 3), dtype=np.int64)
        if n.value:
            _check(lib().jsweep_dags_lagged(self._h, int(m), _ptr(rows), ctypes.byref(n)))
        return rows

    def reset_lag(self):
        _check(lib().jsweep_dags_reset_lag(self._h))

    def set_options(self, opt: jsweep_options):
        _check(lib().jsweep_dags_set_options(self._h, ctypes.byref(opt)))

    def timing(self) -> dict:
        t = jsweep_timing()
        _check(lib().jsweep_dags_timing(self._h, ctypes.byref(t)))
        return {"build_ms": t.build_ms, "sweep_ms": t.sweep_ms, "phi_ms": t.phi_ms,
                "sweep_launches": t.sweep_launches, "build_launches": t.build_launches,
                "call_launches": t.call_launches, "build_steps": t.build_steps,
                "build_stall_rounds": t.build_stall_rounds, "build_phase_ms": list(t.build_phase_ms),
                "sweep_programs": t.sweep_programs, "sweep_requeues": t.sweep_requeues}


def jsweep_mesh_create(n_cells, n_faces, face_cells, normals, areas, volumes) -> Mesh:
    fc = _np(face_cells, np.int64).reshape(-1, 2)
    nr = _np(normals, np.float64).reshape(-1, 3)
    ar = _np(areas, np.float64).ravel()
    vo = _np(volumes, np.float64).ravel()
    if fc.shape[0] != n_faces or nr.shape[0] != n_faces or ar.size != n_faces or vo.size != n_cells:
        raise ValueError("jsweep_mesh_create: array sizes do not match n_cells / n_faces")
    h = ctypes.c_void_p()
    _check(lib().jsweep_mesh_create(int(n_cells), int(n_faces), _ptr(fc), _ptr(nr), _ptr(ar), _ptr(vo),
                                    ctypes.byref(h)), "jsweep_mesh_create")
    return Mesh(h)


def mesh_from_dict(mesh: dict) -> Mesh:
    return jsweep_mesh_create(mesh["n_cells"], mesh["n_faces"], mesh["face_cells"], mesh["normals"],
                              mesh["areas"], mesh["volumes"])


def jsweep_quadrature_product(n_polar: int, n_azim: int):
    M = 8 * n_polar * n_azim
    d = np.empty((M, 3))
    w = np.empty(M)
    _check(lib().jsweep_quadrature_product(int(n_polar), int(n_azim), _ptr(d), _ptr(w)),
           "jsweep_quadrature_product")
    return d, w


def jsweep_quadrature_create(dirs, weights) -> Quad:
    d = _np(dirs, np.float64).reshape(-1, 3)
    w = _np(weights, np.float64).ravel()
    if w.size != d.shape[0]:
        raise ValueError("jsweep_quadrature_create: dirs and weights differ in length")
    h = ctypes.c_void_p()
    _check(lib().jsweep_quadrature_create(d.shape[0], _ptr(d), _ptr(w), ctypes.byref(h)),
           "jsweep_quadrature_create")
    return Quad(h, d, w)


def jsweep_build_dags(mesh: Mesh, quad: Quad, options: jsweep_options | None = None, stream=None) -> Dags:
    h = ctypes.c_void_p()
    _check(lib().jsweep_build_dags(mesh._h, quad._h, ctypes.byref(options) if options is not None else None,
                                   _stream(stream), ctypes.byref(h)), "jsweep_build_dags")
    return Dags(h, mesh, quad)


def _prec(dtype):
    import torch
    if dtype == torch.float64:
        return JSWEEP_F64
    if dtype == torch.float32:
        return JSWEEP_F32
    raise TypeError(f"unsupported dtype {dtype} (float64 or float32)")


def jsweep_sweep(dags: Dags, sigma_t, ang_source, inflow=None, phi_out=None, psi_out=None, stream=None):
    """One sweep of all directions; ang_source [R, N] (device).  Returns phi [R, N]."""
    import torch
    N, M, Fb = dags.n_cells, dags.n_dirs, dags.mesh.n_bfaces
    R = ang_source.shape[0] if ang_source.dim() == 2 else 1
    dt = ang_source.dtype
    prec = _prec(dt)
    if phi_out is None:
        phi_out = torch.empty((R, N), dtype=dt, device=ang_source.device)
    rc = lib().jsweep_sweep(dags._h, R, prec, _dptr(sigma_t, dt, N, "sigma_t"), _dptr(ang_source, dt, R * N, "ang_source"),
                            _dptr(inflow, dt, R * Fb, "inflow"), _dptr(phi_out, dt, R * N, "phi_out"),
                            _dptr(psi_out, dt, R * M * N, "psi_out"), _stream(stream))
    _check(rc, "jsweep_sweep")
    return phi_out


def jsweep_source_iterate(dags: Dags, sigma_t, c_ratio, q, inflow=None, tol=1e-8, max_iters=1000,
                          phi_out=None, stream=None, allow_not_converged=False):
    """Source iteration from phi = 0.  Returns (phi [R, N], iterations, residual, converged)."""
    import torch
    N, Fb = dags.n_cells, dags.mesh.n_bfaces
    R = q.shape[0] if q.dim() == 2 else 1
    dt = q.dtype
    prec = _prec(dt)
    if phi_out is None:
        phi_out = torch.empty((R, N), dtype=dt, device=q.device)
    it = ctypes.c_int()
    res = ctypes.c_double()
    rc = lib().jsweep_source_iterate(dags._h, R, prec, _dptr(sigma_t, dt, N, "sigma_t"), _dptr(c_ratio, dt, N, "c_ratio"),
                                     _dptr(q, dt, R * N, "q"), _dptr(inflow, dt, R * Fb, "inflow"), float(tol),
                                     int(max_iters), _dptr(phi_out, dt, R * N, "phi_out"), ctypes.byref(it),
                                     ctypes.byref(res), _stream(stream))
    if rc == JSWEEP_ERR_NOT_CONVERGED and allow_not_converged:
        return phi_out, it.value, res.value, False
    _check(rc, "jsweep_source_iterate")
    return phi_out, it.value, res.value, True


def jsweep_source_iterate_mg(dags: Dags, sigma_t, sigma_s, q, inflow=None, tol=1e-8, max_iters=1000,
                             phi_out=None, stream=None, allow_not_converged=False):
    """Multigroup source iteration from phi = 0: sigma_t [G, N], sigma_s [G, G, N]
    ([h, g]: rate from group h into group g), q [G, N], inflow [G, n_bfaces] or
    None.  Returns (phi [G, N], iterations, residual, converged)."""
    import torch
    N, Fb = dags.n_cells, dags.mesh.n_bfaces
    G = q.shape[0] if q.dim() == 2 else 1
    dt = q.dtype
    prec = _prec(dt)
    if phi_out is None:
        phi_out = torch.empty((G, N), dtype=dt, device=q.device)
    it = ctypes.c_int()
    res = ctypes.c_double()
    rc = lib().jsweep_source_iterate_mg(dags._h, G, prec, _dptr(sigma_t, dt, G * N, "sigma_t"),
                                        _dptr(sigma_s, dt, G * G * N, "sigma_s"), _dptr(q, dt, G * N, "q"),
                                        _dptr(inflow, dt, G * Fb, "inflow"), float(tol), int(max_iters),
                                        _dptr(phi_out, dt, G * N, "phi_out"), ctypes.byref(it), ctypes.byref(res),
                                        _stream(stream))
    if rc == JSWEEP_ERR_NOT_CONVERGED and allow_not_converged:
        return phi_out, it.value, res.value, False
    _check(rc, "jsweep_source_iterate_mg")
    return phi_out, it.value, res.value, True


def jsweep_bounds_checked() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(lib().jsweep_bounds_checked())


def jsweep_bounds_error() -> int:
    """The first out-of-range index recorded by a bounds-checked build on the
    current device ((code << 56) | index, 0 = none); clears it."""
    w = ctypes.c_uint64(0)
    _check(lib().jsweep_bounds_error(ctypes.byref(w)), "jsweep_bounds_error")
    return int(w.value)


JSWEEP_PROBLEM_ACTIVE = 0
JSWEEP_PROBLEM_CONVERGED = 1
JSWEEP_PROBLEM_MAX_ITERS = 2


class Batch:
    """Many independent source-iteration problems advanced by one data-driven
    launch per iteration (jsweep_batch_*).

    ``add`` takes a built :class:`Dags` and the problem's device tensors (kept
    referenced here until the problem is removed) and returns the problem id.
    ``step`` advances every active problem by up to ``n_sweeps`` iterations;
    a finished problem has its ``phi_out`` written when ``step`` returns.
    """

    def __init__(self, dtype, nrhs: int = 1, options: jsweep_options | None = None):
        self.dtype = dtype
        self.nrhs = int(nrhs)
        self._prec = _prec(dtype)
        h = ctypes.c_void_p()
        _check(lib().jsweep_batch_create(self._prec, self.nrhs, ctypes.byref(options) if options is not None else None,
                                         ctypes.byref(h)), "jsweep_batch_create")
        self._h = h
        self._keep = {}  # id -> (dags, tensors) referenced while the problem is in the batch

    def __del__(self):
        if getattr(self, "_h", None) and _live():
            _lib.jsweep_batch_destroy(self._h)
            self._h = None

    def problem_bytes(self, dags: Dags, has_inflow: bool = False) -> int:
        out = ctypes.c_int64()
        _check(lib().jsweep_batch_problem_bytes(self._h, dags._h, int(bool(has_inflow)), ctypes.byref(out)),
               "jsweep_batch_problem_bytes")
        return out.value

    def add(self, dags: Dags, sigma_t, c_ratio, q, inflow=None, phi_out=None, tol=1e-8, max_iters=1000,
            stream=None) -> int:
        import torch
        N, Fb, R, dt = dags.n_cells, dags.mesh.n_bfaces, self.nrhs, self.dtype
        if phi_out is None:
            phi_out = torch.empty((R, N), dtype=dt, device=q.device)
        pid = ctypes.c_int64()
        _check(lib().jsweep_batch_add(self._h, dags._h, _dptr(sigma_t, dt, N, "sigma_t"),
                                      _dptr(c_ratio, dt, N, "c_ratio"), _dptr(q, dt, R * N, "q"),
                                      _dptr(inflow, dt, R * Fb, "inflow"), _dptr(phi_out, dt, R * N, "phi_out"),
                                      float(tol), int(max_iters), ctypes.byref(pid), _stream(stream)),
               "jsweep_batch_add")
        self._keep[pid.value] = (dags, sigma_t, c_ratio, q, inflow, phi_out)
        return pid.value

    def phi(self, pid: int):
        return self._keep[pid][5]

    def step(self, n_sweeps: int = 1, stream=None) -> int:
        n = ctypes.c_int64()
        _check(lib().jsweep_batch_step(self._h, int(n_sweeps), ctypes.byref(n), _stream(stream)),
               "jsweep_batch_step")
        return n.value

    def launch(self, n_sweeps: int = 1, stream=None):
        """Queue up to n_sweeps iterations and return at once (see poll)."""
        _check(lib().jsweep_batch_launch(self._h, int(n_sweeps), _stream(stream)), "jsweep_batch_launch")

    def poll(self, wait: bool = False):
        """(finished, problems still iterating) of the last launch."""
        done, n = ctypes.c_int(), ctypes.c_int64()
        _check(lib().jsweep_batch_poll(self._h, int(bool(wait)), ctypes.byref(done), ctypes.byref(n)),
               "jsweep_batch_poll")
        return bool(done.value), n.value

    def query(self, pid: int):
        """(state, iterations, residual) of a problem."""
        st, it, res = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().jsweep_batch_query(self._h, int(pid), ctypes.byref(st), ctypes.byref(it), ctypes.byref(res)),
               "jsweep_batch_query")
        return st.value, it.value, res.value

    def remove(self, pid: int):
        _check(lib().jsweep_batch_remove(self._h, int(pid)), "jsweep_batch_remove")
        self._keep.pop(pid, None)

    def clear(self):
        _check(lib().jsweep_batch_clear(self._h), "jsweep_batch_clear")
        self._keep.clear()

    def __len__(self):
        n = ctypes.c_int64()
        _check(lib().jsweep_batch_size(self._h, ctypes.byref(n)), "jsweep_batch_size")
        return n.value

    def source_iterate(self, stream=None, allow_not_converged=False):
        """Restart every problem from phi = 0 and iterate all to the end.
        Returns (iterations, residuals) as arrays in increasing id."""
        n = len(self)
        it = np.zeros(max(n, 1), dtype=np.int32)
        res = np.zeros(max(n, 1), dtype=np.float64)
        rc = lib().jsweep_batch_source_iterate(self._h, _ptr(it), _ptr(res), _stream(stream))
        if not (rc == JSWEEP_ERR_NOT_CONVERGED and allow_not_converged):
            _check(rc, "jsweep_batch_source_iterate")
        return it[:n], res[:n]

    def autotune(self, stream=None) -> float:
        ms = ctypes.c_double()
        _check(lib().jsweep_batch_autotune(self._h, _stream(stream), ctypes.byref(ms)), "jsweep_batch_autotune")
        return ms.value

    def options(self) -> jsweep_options:
        o = jsweep_options()
        _check(lib().jsweep_batch_options(self._h, ctypes.byref(o)), "jsweep_batch_options")
        return o

    def stats(self):
        """(sweep launch ms, whole iteration ms) of the last batched iteration
        and the kernels launched by this batch so far."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(lib().jsweep_batch_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n), None, None),
               "jsweep_batch_stats")
        return a.value, b.value, n.value

    def setup_stats(self):
        """(host ms spent rebuilding tables and captured iterations, rebuilds) so far."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().jsweep_batch_stats(self._h, None, None, None, ctypes.byref(ms), ctypes.byref(n)),
               "jsweep_batch_stats")
        return ms.value, n.value


JSWEEP_NOALLOC_SCRATCH_BYTES = 64 << 20


def jsweep_source_iterate_noalloc(dags: Dags, sigma_t, c_ratio, q, phi_out, inflow=None, tol=1e-8,
                                  max_iters=1000, stream=None, allow_not_converged=False):
    """Source iteration that allocates no device memory (jsweep_source_iterate_noalloc).

    For callers that cannot allocate device memory while they run (a host
    application that owns the device's memory budget, or a loop that cannot
    afford cudaMalloc's device-wide synchronisation): all temporaries live in
    the library's fixed JSWEEP_NOALLOC_SCRATCH_BYTES device array.  The caller
    passes every input and the output ``phi_out`` [R, N]; nothing here
    allocates on the device.  Calls share that array, so calls that overlap on
    the GPU must be serialised.  Returns (phi_out, iterations, residual, converged).
    """
    N, Fb = dags.n_cells, dags.mesh.n_bfaces
    R = q.shape[0] if q.dim() == 2 else 1
    dt = q.dtype
    prec = _prec(dt)
    it = ctypes.c_int()
    res = ctypes.c_double()
    rc = lib().jsweep_source_iterate_noalloc(
        dags._h, R, prec, _dptr(sigma_t, dt, N, "sigma_t"), _dptr(c_ratio, dt, N, "c_ratio"),
        _dptr(q, dt, R * N, "q"), _dptr(inflow, dt, R * Fb, "inflow"), float(tol), int(max_iters),
        _dptr(phi_out, dt, R * N, "phi_out"), ctypes.byref(it), ctypes.byref(res), _stream(stream))
    if rc == JSWEEP_ERR_NOT_CONVERGED and allow_not_converged:
        return phi_out, it.value, res.value, False
    _check(rc, "jsweep_source_iterate_noalloc")
    return phi_out, it.value, res.value, True
