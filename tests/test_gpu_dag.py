"""GPU dependency graphs against the oracle: levels, orders and lagged faces bit-exact."""

import json
import os

import numpy as np
import pytest

import oracle
from inputs import column_mesh, hex_grid, kuhn_tets, make_workload, pinwheel_mesh
from _gpu import build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def compare_all(mesh, dirs, w, dir_sample=None, **opt):
    g = build(mesh, dirs, w, **opt)
    sample = range(dirs.shape[0]) if dir_sample is None else dir_sample
    sub = dirs[list(sample)]
    o = oracle.build_dags(mesh, sub)
    n_lag = 0
    for i, m in enumerate(sample):
        assert g.nlevels(m) == o.nlevels(i), f"direction {m}"
        assert np.array_equal(g.levels(m), o.levels(i)), f"direction {m}"
        go, gp = g.order(m)
        oo, op = o.order(i)
        assert np.array_equal(go, oo), f"direction {m}"
        assert np.array_equal(gp, op), f"direction {m}"
        gl, ol = g.lagged(m), o.lagged(i)
        assert np.array_equal(gl, ol), f"direction {m}"
        n_lag += len(ol)
    return g, n_lag


def test_pinwheel_golden():
    gold = json.load(open(os.path.join(HERE, "golden", "pinwheel.json")))
    mesh = pinwheel_mesh()
    dirs = np.array([c["omega"] for c in gold["cases"]])
    g = build(mesh, dirs, np.ones(len(dirs)))
    for m, case in enumerate(gold["cases"]):
        assert g.lagged(m).tolist() == case["lagged"]
        assert g.levels(m).tolist() == case["levels"]
        order, ptr = g.order(m)
        assert order.tolist() == case["order"] and ptr.tolist() == case["level_ptr"]


@pytest.mark.parametrize("kind,n,jit,seed,quad", [
    ("hex", 4, 0.3, 7, (6, 6)),
    ("hex", 5, 0.3, 11, (6, 6)),
    ("hex", 6, 0.25, 3, (6, 6)),
    ("tet", 5, 0.2, 2, (4, 4)),
    ("hex", 1, 0.0, 0, (2, 3)),
])
def test_small_meshes_bit_exact(kind, n, jit, seed, quad):
    mesh = hex_grid(n, jit, seed) if kind == "hex" else kuhn_tets(n, jit, seed)
    dirs, w = oracle.product_quadrature(*quad)
    _, n_lag = compare_all(mesh, dirs, w)
    if kind == "hex" and jit >= 0.25:
        assert n_lag > 0


@pytest.mark.parametrize("n_dirs,seed", [(13, 1), (29, 2), (8, 3)])
def test_uneven_octants_bit_exact(n_dirs, seed):
    # the build groups each octant's directions into slots of 8 (padded when
    # cheap): random direction sets leave octants empty, short and uneven,
    # and a few axis-aligned directions sit on octant borders
    rng = np.random.default_rng(seed)
    dirs = rng.normal(size=(n_dirs, 3))
    dirs[:2] = [[1.0, 0.0, 0.0], [0.0, -1.0, 0.0]]
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    w = np.full(n_dirs, 4 * np.pi / n_dirs)
    for mesh in (hex_grid(6, 0.3, 5), kuhn_tets(4, 0.2, 6)):
        compare_all(mesh, dirs, w)
        compare_all(mesh, dirs, w, layering=1)


def test_workload1_full_size_bit_exact():
    wl = make_workload(1)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    compare_all(wl, dirs, w)


def test_many_cycles_several_tiles_bit_exact():
    # 32^3 hex, 288 directions: thousands of lagged faces, several sort tiles
    mesh = hex_grid(32, 0.15, 3)
    dirs, w = oracle.product_quadrature(6, 6)
    _, n_lag = compare_all(mesh, dirs, w)
    assert n_lag > 1000


def test_deep_graphs_and_partial_sort_tiles_bit_exact():
    # the level sort with two and three radix passes over segments that end in
    # a partial tile (4,096 keys per tile), and a lag list longer than a tile:
    # a long jittered slab (6,000 cells; 1,500-2,100 levels and ~9,000 lagged
    # faces over 48 directions; components of at most 19 cells) and a
    # 70,000-cell column (70,000 levels)
    slab = hex_grid(jitter=0.2, seed=9, shape=(300, 5, 4))
    dirs, w = oracle.product_quadrature(2, 3)
    g, n_lag = compare_all(slab, dirs, w)
    assert min(g.nlevels(m) for m in range(dirs.shape[0])) > 256 and n_lag > 4096
    col = column_mesh(70000)
    dirs = np.array([[1.0, 0.0, 0.0], [-0.6, 0.8, 0.0], [0.36, 0.48, 0.8]])
    g, _ = compare_all(col, dirs, np.full(3, 4 * np.pi / 3))
    assert all(g.nlevels(m) == 70000 for m in range(3))


def test_unstructured_tets_bit_exact():
    mesh = kuhn_tets(12, 0.2, 2)
    dirs, w = oracle.product_quadrature(4, 4)
    compare_all(mesh, dirs, w)


def test_unjittered_and_column():
    # exact zero fluxes (Omega . n == 0) carry no dependency on both sides
    mesh = hex_grid(6, 0.0, 0)
    dirs = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.0, 1.0]])
    compare_all(mesh, dirs, np.ones(4))
    col = column_mesh(50)
    compare_all(col, np.array([[0.3, 0.0, 0.0], [-1.0, 0.0, 0.0]]), np.ones(2))


def test_small_cluster_and_search_cap_options():
    mesh = hex_grid(5, 0.3, 11)
    dirs, w = oracle.product_quadrature(6, 6)
    compare_all(mesh, dirs, w, cluster_cells=3, cycle_search_max=32)


def test_cycle_search_cap_too_small_is_an_error():
    from paper_1803_09876_gb300 import jsweep as J
    mesh = hex_grid(5, 0.3, 11)
    dirs, w = oracle.product_quadrature(6, 6)
    with pytest.raises(J.JsweepError) as e:
        build(mesh, dirs, w, cycle_search_max=2)
    assert e.value.code == J.JSWEEP_ERR_CYCLE


def _sample_dirs(dirs, k_grazing=4, k_other=2):
    mu = np.abs(dirs[:, 2])
    graz = list(np.argsort(mu, kind="stable")[:: max(1, len(mu) // (4 * k_grazing))][:k_grazing])
    other = [len(dirs) // 3, (2 * len(dirs)) // 3 + 1][:k_other]
    return sorted(set(int(x) for x in graz + other))


def test_workload3_full_size_sampled_directions_bit_exact():
    # 128^3 jittered hexes, 288 directions: the whole build runs on the GPU;
    # sampled directions (grazing ones carry cycles) are checked bit-exact.
    wl = make_workload(3, n_rhs=1)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    sample = _sample_dirs(dirs)
    g, n_lag = compare_all(wl, dirs, w, dir_sample=sample)
    assert g.n_lag_total > 0


def test_workload2_full_size_sampled_directions_bit_exact():
    wl = make_workload(2)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    compare_all(wl, dirs, w, dir_sample=_sample_dirs(dirs, 3, 2))


@pytest.mark.parametrize("eager", [1, 8, 1024])
def test_eager_search_cap_does_not_change_the_graphs(eager):
    # eager cycle searches capped at 1..1024 cells (a build that cannot break a
    # cycle that way is repeated with the full cap): the graphs are the oracle's
    mesh = hex_grid(16, 0.3, 5)
    dirs, w = oracle.product_quadrature(6, 6)
    _, n_lag = compare_all(mesh, dirs, w, eager_search_max=eager, cycle_search_max=max(256, eager))
    assert n_lag > 100


@pytest.mark.parametrize("layering", [0, 1], ids=["octant_layers", "levels"])
def test_schedule_layers_follow_every_active_dependency(layering):
    # the paper's progress argument, checked on the layers the sweeps run: a
    # cell is scheduled after every active (not lagged) upwind cell
    from _bruteforce import edges
    for mesh, quad in ((hex_grid(5, 0.3, 11), (6, 6)), (kuhn_tets(4, 0.2, 8), (4, 4))):
        dirs, w = oracle.product_quadrature(*quad)
        g = build(mesh, dirs, w, layering=layering)
        N = mesh["n_cells"]
        for m in range(len(dirs)):
            order, ptr = g.schedule(m)
            assert np.array_equal(np.sort(order), np.arange(N))
            assert ptr[0] == 0 and ptr[-1] == N and np.all(np.diff(ptr) >= 0)  # octant layers may be empty
            if layering == 1:  # the level schedule is the level-major order
                lo, lp = g.order(m)
                assert np.array_equal(order, lo) and np.array_equal(ptr, lp)
            layer = np.empty(N, dtype=np.int64)
            for k in range(len(ptr) - 1):
                layer[order[ptr[k]:ptr[k + 1]]] = k
            lagged = {int(f) for f in g.lagged(m)[:, 0]}
            for f, u, v in edges(mesh, dirs[m]):
                if f not in lagged:
                    assert layer[u] < layer[v], (m, f, u, v)
