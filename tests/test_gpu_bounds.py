"""The bounds-checked build (JSWEEP_BOUNDS_CHECK) on tiny meshes: every sweep
schedule, batches, the allocation-free and multigroup iterations run with
every gather index checked, reach the oracle's fixed point, and record no
index out of range.  It runs in a child process, which loads
libjsweep_bounds.so instead of the normal library."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import math, sys
import numpy as np
import torch
ROOT = sys.argv[1]
sys.path[:0] = [ROOT, ROOT + "/tests"]
import oracle
from inputs import hex_grid, kuhn_tets, multigroup_materials, pinwheel_mesh
from paper_1803_09876_gb300 import build as libbuild
from paper_1803_09876_gb300 import jsweep as J

J.load(libbuild.build(bounds_check=True))
J.use_torch_allocator()
assert J.jsweep_bounds_checked()
f64 = torch.float64


def tensor(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=f64, device="cuda")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def clean(what):
    w = J.jsweep_bounds_error()
    assert w == 0, f"{what}: index out of range, code {w >> 56}, index {w & ((1 << 56) - 1)}"


def quad_for(mesh):
    dirs, w = oracle.product_quadrature(1, 3)
    if mesh["n_cells"] == 4:  # pinwheel: directions near +-z make its cycles appear
        dirs = np.concatenate([dirs, [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]]])
        w = np.concatenate([w * 0.9, [0.2 * math.pi, 0.2 * math.pi]])
    return dirs, w


cases = [("hex 2^3", hex_grid(2, 0.2, 1)), ("one tet cube", kuhn_tets(1, 0.2, 2)),
         ("cyclic hex 4^3", hex_grid(4, 0.3, 5)), ("pinwheel", pinwheel_mesh())]
for name, mesh in cases:
    dirs, w = quad_for(mesh)
    o = oracle.build_dags(mesh, dirs)
    N = mesh["n_cells"]
    rng = np.random.default_rng(5)
    sig, c = rng.uniform(0.5, 2.0, N), np.full(N, 0.5)
    q = rng.uniform(0.0, 1.0, (2, N))
    inflow = rng.uniform(0.0, 0.3, (2, o.n_bfaces))
    ref = o.source_iterate(sig, c, q, w, 1e-11, 1000, inflow=inflow)[0]
    quad = J.jsweep_quadrature_create(dirs, w)
    for opts in (dict(sweep_mode=1), dict(sweep_mode=1, no_face_stream=1), dict(sweep_mode=1, tail_units=1 << 30),
                 dict(sweep_mode=2)):
        g = J.jsweep_build_dags(J.mesh_from_dict(mesh), quad, J.jsweep_options_default(**opts))
        clean(f"{name} build")
        phi, it, res, ok = J.jsweep_source_iterate(g, tensor(sig), tensor(c), tensor(q), inflow=tensor(inflow),
                                                   tol=1e-11, max_iters=1000)
        assert ok and rel(phi.cpu().numpy(), ref) < 1e-8, (name, opts)
        clean(f"{name} {opts}")
    g = J.jsweep_build_dags(J.mesh_from_dict(mesh), quad)
    for mode in (1, 2):
        b = J.Batch(f64, 2, J.jsweep_options_default(sweep_mode=mode))
        pid = b.add(g, tensor(sig), tensor(c), tensor(q), inflow=tensor(inflow), tol=1e-11, max_iters=1000)
        b.source_iterate()
        assert rel(b.phi(pid).cpu().numpy(), ref) < 1e-8, (name, "batch", mode)
        clean(f"{name} batch mode {mode}")
    phi = torch.empty((2, N), dtype=f64, device="cuda")
    J.jsweep_source_iterate_noalloc(g, tensor(sig), tensor(c), tensor(q), phi, inflow=tensor(inflow), tol=1e-11,
                                    max_iters=1000)
    assert rel(phi.cpu().numpy(), ref) < 1e-8, (name, "noalloc")
    clean(f"{name} noalloc")
    sg, ss = multigroup_materials(N, 2, seed=9)
    mg_ref = o.multigroup_source_iterate(sg, ss, q, w, 1e-11, 1000, inflow=inflow)[0]
    phi_mg = J.jsweep_source_iterate_mg(g, tensor(sg), tensor(ss), tensor(q), inflow=tensor(inflow), tol=1e-11,
                                        max_iters=1000)[0]
    assert rel(phi_mg.cpu().numpy(), mg_ref) < 1e-8, (name, "multigroup")
    clean(f"{name} multigroup")
print("bounds-checked build: no index out of range")
'''


def test_bounds_checked_build_on_tiny_meshes():
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "no index out of range" in r.stdout
