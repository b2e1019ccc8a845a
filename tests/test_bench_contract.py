"""bench.py's JSON contract, checked on the CPU: the reference arm (the oracle on the host cores)
prints one line with the required keys, and the helpers that fill the GPU line's roofline and
replica fields compute what they state."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "small_2d", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["value"] > 0 and d["config"]["workload"] == "small_2d"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_assembly_roofline_is_the_largest_leg():
    n, nnz, d, L = 1_000_000, 100_000_000, 3, 8
    r = bench.assembly_roofline(n, d, L, nnz, 10.0, 6789.6)["roofline"]
    pairs = 0.5 * (nnz + n)
    legs = {"hbm": (16.0 * nnz + 4.0 * (n + 1)) / 6789.6e9,
            "alu_fp32": pairs * 2 * d / bench.FP32_INSTR_PEAK,
            "alu_fp64": pairs * (2 * d + 1 + 7 + L + 3) / bench.FP64_INSTR_PEAK}
    assert r["bound"] == max(legs, key=legs.get)
    assert r["roof_ms"] == pytest.approx(1000.0 * max(legs.values()))
    assert r["frac"] == pytest.approx(r["roof_ms"] / 10.0)
    for k, v in legs.items():
        assert r["legs_ms"][k] == pytest.approx(1000.0 * v)
    # FP64 precision stores no FP32 copy
    r64 = bench.assembly_roofline(n, d, L, nnz, 10.0, 6789.6, mixed=False)["roofline"]
    assert r64["bytes"] == 12.0 * nnz + 4.0 * (n + 1)


def test_profile_traffic_reads_the_committed_summaries():
    t, src = bench.profile_traffic("clusters_3d", 1_000_000)
    assert src == os.path.join("profiles", "k_spmm_rb_clusters_3d_n1m.md") and 1e9 < t < 3e9
    assert bench.profile_traffic("clusters_3d", 2_000_000) == (None, None)
