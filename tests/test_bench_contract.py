"""Host logic of bench.py on CPU: the algorithmic byte count the roofline divides by, and
the JSON line of the reference arm (the FP64 oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_count_each_node_kind():
    flags = np.zeros((2, 3, 4), np.uint8)          # 24 nodes
    flags[0, 0, :2] = 1                              # 2 obstacle voxels
    flags[1, 2, 1:4] = 2                             # 3 inflow nodes
    flags[1, 0, 0] = 3                               # obstacle and inflow: counted as obstacle
    fluid, solid, inflow = 24 - 3 - 3, 3, 3
    total, per_fluid = bench._algorithmic_bytes(flags, "fp32")
    assert per_fluid == 27 * 4 * 2 + 12 * 2 + 4 * 2 + 1 == 249
    assert total == fluid * 249 + solid * (27 * 4 + 12 + 4 + 1) + inflow * (27 * 4 + 24 + 8 + 1)
    total16, per16 = bench._algorithmic_bytes(flags, "fp16")
    assert per16 == 141
    assert total16 == fluid * 141 + solid * (27 * 2 + 17) + inflow * (27 * 2 + 33)
    assert bench._algorithmic_bytes(flags, "fp32", local=True)[1] == 237


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "dtype", "data", "config"):
        assert k in line, k
    assert line["metric"] == "MLUPS" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["steps"] == 1 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "plume32_oracle"
    assert line["config"]["nodes"] == 32 ** 3


def test_repeat_record_reports_the_median_call():
    times = [0.30, 0.10, 0.20, 0.50]          # seconds per K-step call
    rec = bench.repeat_record(times, 10, 1000)
    assert rec["count"] == 4 and rec["steps_per_call"] == 10
    assert rec["ms_per_step_median"] == np.median(times) / 10 * 1e3
    assert rec["ms_per_step_best"] == 0.10 / 10 * 1e3 and rec["ms_per_step_worst"] == 50.0
    assert rec["value_best"] == 1000 * 10 / 0.10 / 1e6
    assert abs(rec["device_seconds"] - 1.1) < 1e-12


def test_coupling_bytes_of_a_worked_two_block_case():
    """s0 8^3 with a block at h = 1/2, origin (2, 2, 2), 7^3 nodes (reference span [2, 5]):
    every scale-boundary position has a coordinate on the cube's surface, so its corners of
    non-zero weight are the 4^3 - 2^3 = 56 surface nodes of s0 in [2, 5]^3; post-mapping
    targets the 8 s0 nodes with coordinates 3, 4, which sit exactly on fine nodes (one corner
    each).  Two sub-steps land on t_n + dt_0: no alignment."""
    import synth
    s0 = synth._empty_block((8, 8, 8))
    s1 = synth._empty_block((7, 7, 7), origin=(2.0, 2.0, 2.0), h=0.5)
    sc = synth.Scene(blocks=[s0, s1], periodic=(False,) * 3, nu=0.01)
    got = bench._coupling_bytes(sc, [1, 2])
    ghost_nodes = 7 ** 3 - 5 ** 3
    assert got["ghost"] == 3 * ghost_nodes * 124 + 4 * 56 * 113
    assert got["post"] == 8 * 124 + 8 * 113
    assert got["align"] == 0
    s1b = synth._empty_block((7, 7, 7), origin=(2.0, 2.0, 2.0), h=1 / 1.5)
    sc2 = synth.Scene(blocks=[synth._empty_block((8, 8, 8)), s1b], periodic=(False,) * 3, nu=0.01)
    assert bench._coupling_bytes(sc2, [1, 2])["align"] == 5 ** 3 * 112
