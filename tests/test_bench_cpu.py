"""The benchmark's host-side contract, without a GPU: the reference arm's
JSON line and the byte model it and the GPU arm share."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_byte_model_counts_the_format_independent_bytes():
    import bench
    # nnz (value + index) + row pointers + x + y, fp64: 12 B per entry
    assert bench.byte_model(4, 5, 10, 8, 8) == 10 * 12 + 4 * 5 + 8 * 5 + 8 * 4
    # bf16 values with fp32 vectors; beta != 0 reads y as well
    assert bench.byte_model(4, 5, 10, 2, 4, beta_nonzero=True) == 10 * 6 + 4 * 5 + 4 * 5 + 4 * 4 * 2


def test_format_names():
    import bench
    assert bench.fmt_name({"format": 0, "threads_per_row": -1}) == "csr_split"
    assert bench.fmt_name({"format": 0, "threads_per_row": -1, "hyb_ell_width": 4096}) == "csr_tiles"
    assert bench.fmt_name({"format": 0, "threads_per_row": 4}) == "csr"
    assert [bench.fmt_name({"format": f}) for f in range(1, 6)] == ["ell", "coo", "hyb", "bsr", "sell"]


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--scale", "small",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
