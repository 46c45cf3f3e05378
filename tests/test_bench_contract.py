"""bench.py without a GPU: the reference arm's JSON line, the algorithmic byte and flop counts the
roofline divides by, and the batch workload's shape."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1711_10855_gb300 import synth  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "small",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["config"]["workload"] == synth.small().name
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_algorithmic_counts_of_the_survey_plane():
    """4 B per cell of plane, the segments with their overlap, the template bank and twiddles; flops
    5 L log2 L + 6 L + 3 V per (segment, template) plus one forward transform per segment."""
    w = synth.survey()
    V = w.seg_len - w.tmpl_len
    nseg = -(-w.n_bins // V)
    assert nseg == 2731
    a = bench.algorithmic(w, nseg)
    assert a["bytes_plane"] == 4 * 201 * (1 << 22)
    assert a["bytes"] == 4 * 201 * (1 << 22) + 8 * 2731 * 2048 + 8 * 201 * 2048 + 8 * 2048
    assert abs(a["bytes"] / 1e9 - 3.420) < 1e-3
    assert a["flops"] == 2731 * 201 * (5 * 2048 * 11 + 6 * 2048 + 3 * 1536) + 2731 * 5 * 2048 * 11
    assert abs(a["flops"] / 1e9 - 71.41) < 0.01
    # co-limits: 3 x 16 KB of shared traffic per inverse transform, 2 x 16 KB per forward one;
    # the 3.3 MB bank streamed once per group of 8 segments (342 groups)
    assert a["smem_bytes"] == 2731 * 201 * 3 * 16384 + 2731 * 2 * 16384
    assert a["l2_template_bytes"] == 342 * 201 * 16384
    assert abs(a["l2_template_bytes"] / 1e9 - 1.126) < 1e-3


def test_batch_workload_shape():
    n, zmax = synth.batch_workload(256)
    assert n.size == zmax.size == 256
    assert np.all(n % 4 == 0) and n.min() >= (1 << 18) - 4 and n.max() <= 1 << 22
    assert set(np.unique(zmax)) <= {100, 200}
    n2, z2 = synth.batch_workload(256)
    np.testing.assert_array_equal(n, n2)
    np.testing.assert_array_equal(zmax, z2)


def test_replica_throughput_counts_every_rank_over_the_slowest():
    assert bench.replica_throughput(1000, 5, 4, 2.0) == 1000 * 5 * 4 / 2.0
    assert bench.max_over_ranks(3.5) == 3.5


def test_tensor_core_flop_count():
    """Per (segment, template): 3 x (2*32*128*128 + 2*64*64*64) = 4,718,592 tensor flops."""
    assert bench.tc_flops(1, 1) == 4_718_592
    assert abs(bench.tc_flops(2731, 201) / 1e12 - 2.590) < 1e-3


def test_operating_point_rule():
    """Fewest pairs among the points reaching the target; the best recall when none does."""
    pts = [{"z_halo": 0, "threshold": 0.1, "recall": 0.95, "pair_fraction": 0.05},
           {"z_halo": 8, "threshold": 0.1, "recall": 0.978, "pair_fraction": 0.18},
           {"z_halo": 12, "threshold": 0.1, "recall": 0.98, "pair_fraction": 0.22},
           {"z_halo": 8, "threshold": 0.05, "recall": 0.99, "pair_fraction": 0.35}]
    assert bench.choose_operating_point(pts, 0.97)["z_halo"] == 8
    assert bench.choose_operating_point(pts, 0.97)["threshold"] == 0.1
    assert bench.choose_operating_point(pts, 0.985)["threshold"] == 0.05
    best = bench.choose_operating_point(pts, 0.999)       # none reaches: the highest recall
    assert best["recall"] == 0.99
    tie = pts + [{"z_halo": 4, "threshold": 0.2, "recall": 0.99, "pair_fraction": 0.30}]
    assert bench.choose_operating_point(tie, 0.999)["pair_fraction"] == 0.30
