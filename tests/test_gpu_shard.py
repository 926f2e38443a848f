"""Merging plan states through the C ABI (the per-rank step of the sharded path),
on one GPU: plans that each saw a whole-group shard of a record, merged by
ss_merge_state, must give the oracle's estimate on the whole record."""
import numpy as np
import pytest

import oracle
import synth
from paper_2505_01231_gb300 import shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def P():
    import paper_2505_01231_gb300 as mod
    return mod


def check(out, ref):
    for key in ("S2", "S3", "S4"):
        a, b = out[key][0].reshape(ref[key].shape), ref[key]
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err <= TOL, f"{key}: {err:.2e}"
        ea, eb = out[key + "_err"][0].reshape(ref[key + "_err"].shape), ref[key + "_err"]
        assert np.max(np.abs(ea - eb)) / np.max(np.abs(eb)) <= 1e-4, key + "_err"


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("world", [2, 3])
def test_merged_shards_match_the_whole_record(precision, world):
    mod = P()
    T, m = 128, 8
    n = 23 * m * T + 77
    z = synth.ar1_quadratic(n, seed=11)
    ref = oracle.polyspectra(z, T, 0.25, m, group_chunk=8)
    plans = []
    for a, b in shard.group_ranges(n, T, m, world):
        p = mod.Plan(T=T, dt=0.25, m=m, precision=precision)
        p.accumulate(torch.from_numpy(np.ascontiguousarray(z[a:b])).cuda(), b - a)
        plans.append(p)
    states = [p.export_state() for p in plans]  # before any merge
    # rank 0 merges the others: one from host memory, the rest from device memory
    for i, p in enumerate(plans[1:]):
        if i == 0:
            plans[0].merge_state(p.export_state())
        else:
            d = torch.empty(mod.ss_state_size(p.handle), dtype=torch.float64, device="cuda")
            p.export_state(d)
            plans[0].merge_state(d)
    out = plans[0].finalize()
    assert out["G"] == 23
    check(out, ref)
    # the all-reduce form (as shard.reduce_state does it): configuration words kept,
    # counts and sums added element-wise, merged into a reset plan
    total = states[0].copy()
    total[shard.CFG_WORDS:] = sum(st[shard.CFG_WORDS:] for st in states)
    plans[1].reset()
    plans[1].merge_state(total)
    out2 = plans[1].finalize()
    for key in ("S2", "S3", "S4"):
        assert np.allclose(out2[key], out[key], rtol=0, atol=1e-12 * np.max(np.abs(out[key])))
    for p in plans:
        p.close()


def test_state_of_another_configuration_is_refused():
    mod = P()
    a = mod.Plan(T=64, m=6)
    b = mod.Plan(T=64, m=7)
    c = mod.Plan(T=64, m=6, precision="tf32x3")
    z = torch.from_numpy(synth.ar1_quadratic(4 * 6 * 64, seed=2)).cuda()
    a.accumulate(z)
    before = a.export_state()
    for other in (b, c):
        with pytest.raises(mod.SSError) as ei:
            a.merge_state(other.export_state())
        assert ei.value.status == mod.SS_EINVAL
    assert np.array_equal(a.export_state(), before)  # nothing changed
    for p in (a, b, c):
        p.close()
