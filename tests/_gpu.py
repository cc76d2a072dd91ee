"""Helpers of the GPU parity tests: handles through the C ABI, tolerances."""

import numpy as np

# relative max-norm tolerances on phi (and psi): FP64 path, FP32 path
TOL_F64 = 1e-12
TOL_F32 = 2e-5

_allocator_set = False


def J():
    from paper_1803_09876_gb300 import build as libbuild
    from paper_1803_09876_gb300 import jsweep

    global _allocator_set
    libbuild.build()
    jsweep.load()
    if not _allocator_set:
        jsweep.use_torch_allocator()
        _allocator_set = True
    return jsweep


def build(mesh, dirs, w, **opt):
    js = J()
    m = js.mesh_from_dict(mesh)
    q = js.jsweep_quadrature_create(dirs, w)
    o = js.jsweep_options_default(**opt)
    return js.jsweep_build_dags(m, q, o)


def set_opts(dags, **opt):
    js = J()
    dags.set_options(js.jsweep_options_default(**opt))


def rel_err(a, b):
    """Per right-hand side: max |a - b| / max |b|; returns the worst."""
    a = np.asarray(a, dtype=np.float64).reshape(np.shape(b)[0] if np.ndim(b) > 1 else 1, -1)
    b = np.asarray(b, dtype=np.float64).reshape(a.shape)
    worst = 0.0
    for r in range(a.shape[0]):
        den = np.max(np.abs(b[r]))
        err = np.max(np.abs(a[r] - b[r]))
        worst = max(worst, err / den if den > 0 else err)
    return worst


def tensor(x, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")
