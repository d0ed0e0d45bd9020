"""bench.py's JSON contract, checked on the CPU.

The reference arm (the oracle timed on the host cores) needs no GPU, so it
runs here end to end; the GPU arm's arithmetic (work counts, roofline
denominators) is checked from its module-level definitions.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_work_counts():
    n, perms, _ = bench.workload(22, 8)
    assert n == 1 << 22 and perms == (1 << 22) + (1 << 22) - 1
    assert bench.workload(10, 64)[1] == 8 * 1024 + 1023
    # per permutation: 118 S-boxes of 2 squares (3 partial products) and 2 products (4), full
    # rounds 8 x 144 products, partial rounds 22 x 23 products; 2 results per partial product
    assert bench.MUL_RESULTS_PER_PERM == 2 * (118 * (2 * 3 + 2 * 4) + 8 * 144 * 4 + 22 * 23 * 4) == 16568
    # pg12_small: seven full rounds with 8-bit entries use 2 partial products per term
    assert bench.MUL_RESULTS_PER_PERM_SMALL == 2 * (118 * 14 + 7 * 144 * 2 + 144 * 4 + 22 * 23 * 4) == 12536


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "perms/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]
