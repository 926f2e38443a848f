"""CPU checks of bench.py: the reference arm's JSON line (the oracle timed on the host)
and the default channel combinations it uses for several channels."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
         "ar1q-2^20-T256-m10", "--steps", "1", "--warmup", "0", "--ref-groups", "2"],
        cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "samples/s"
    assert rec["higher_is_better"] is True and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"] == {"value": rec["value"], "unit": "samples/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert rec["config"]["T"] == 256 and rec["config"]["m"] == 10


@pytest.mark.parametrize("C", [1, 2, 3, 4])
def test_default_combinations(C):
    sys.path.insert(0, ROOT)
    import bench

    sel = bench.default_combos(C)
    npair = C * (C + 1) // 2
    assert len(sel[2]) == npair
    assert len(sel[3]) == math.comb(C + 2, 3)
    assert len(sel[4]) == npair * (npair + 1) // 2
    # multisets in non-decreasing order, no repeats
    for order in (2, 3):
        assert all(list(c) == sorted(c) for c in sel[order])
        assert len(set(sel[order])) == len(sel[order])
    # S4: (a, b) <= (c, d) as pairs, each pair sorted
    for a, b, c, d in sel[4]:
        assert a <= b and c <= d and (a, b) <= (c, d)


def test_refused_workloads_exit_without_running():
    sys.path.insert(0, ROOT)
    import bench

    for name in bench.REFUSED:
        out = subprocess.run(
            [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", name, "--steps", "1"],
            cwd=ROOT, capture_output=True, text=True, timeout=300)
        assert out.returncode == 2
        assert "refused" in out.stderr
        assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
