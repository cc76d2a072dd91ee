"""The benchmark's JSON line (reference arm, small case on the host cores):
one line on stdout with the keys and units the benchmark contract names."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", *extra], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_line_has_the_contract_keys():
    d = _run("--n", "16")
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["config"]["workload"] == "hex16_288dirs_8rhs"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_multigroup_reference_line():
    d = _run("--workload", "mg")
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["unit"] == "cell-angle-group updates/s"
    assert d["config"]["workload"] == "tet48x6_128dirs_4groups_fp32_si_tol1e-6"
    assert d["cpu_baseline"]["kind"] == "oracle" and "4-group iteration" in d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_recorded_sweep_traffic_belongs_to_the_committed_kernel():
    """The DRAM traffic the benchmark line reports was captured on the slot
    kernel's current sources (their hash is the key), and lies between the
    model's algorithmic bytes and a few times them."""
    sys.path.insert(0, ROOT)
    import bench

    t = bench.SWEEP_TRAFFIC
    assert t["sources_sha16"] == bench.sources_sha16(), "kernel sources changed: recapture the traffic"
    model = 2 * 8 * 4 + 5 + (128 + 2 * 8 * 4) / 288  # 128^3 hex, 288 directions, 8 rhs, FP32
    assert model < t["bytes_per_cell_dir"] < 10 * model
