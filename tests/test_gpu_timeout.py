"""The timeout path of the bounded device waits, exercised without any fault.

Every kernel wait for staged data is bounded; a wait that runs out records
SS_ETIMEOUT in the plan's status word and its CTA stops cleanly (its issued
copies drain, its tensor memory is freed).  ss_inject_timeout makes the
bispectrum kernel run one such wait out on a barrier that nothing completes.
The checks: finalize reports SS_ETIMEOUT, the plan is unusable afterwards, and
the device is intact (a fresh plan on the same record matches the oracle).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def P():
    import paper_2505_01231_gb300 as mod
    return mod


def test_injected_wait_runs_out_and_the_device_stays_usable():
    mod = P()
    T, m = 256, 10
    z = synth.ar1_quadratic(T * m * 300 + 11, seed=21)
    dz = torch.from_numpy(z).cuda()
    plan = mod.Plan(T=T, m=m, orders=(2, 3))
    mod.ss_inject_timeout(plan.handle, 1)
    plan.accumulate(dz)
    with pytest.raises(mod.SSError) as ei:
        plan.finalize()
    assert ei.value.status == mod.SS_ETIMEOUT
    with pytest.raises(mod.SSError) as ei:  # the plan is unusable from then on
        plan.accumulate(dz)
    assert ei.value.status == mod.SS_ESTATE
    plan.close()
    torch.cuda.synchronize()

    # the same record through a fresh plan: the device and the library are intact
    ref = oracle.polyspectra(z, T, 1.0, m, orders=(2, 3), group_chunk=64)
    plan = mod.Plan(T=T, m=m, orders=(2, 3))
    plan.accumulate(dz)
    out = plan.finalize()
    plan.close()
    for key in ("S2", "S3"):
        a, b = out[key][0].reshape(ref[key].shape), ref[key]
        assert np.max(np.abs(a - b)) <= TOL * np.max(np.abs(b)), key


def test_injection_off_again_gives_the_normal_result():
    mod = P()
    T, m = 128, 6
    z = synth.ar1_quadratic(T * m * 40, seed=22)
    ref = oracle.polyspectra(z, T, 1.0, m, orders=(3,), group_chunk=64)
    plan = mod.Plan(T=T, m=m, orders=(3,))
    mod.ss_inject_timeout(plan.handle, 1)
    mod.ss_inject_timeout(plan.handle, 0)
    plan.accumulate(torch.from_numpy(z).cuda())
    out = plan.finalize()
    plan.close()
    a, b = out["S3"][0].reshape(ref["S3"].shape), ref["S3"]
    assert np.max(np.abs(a - b)) <= TOL * np.max(np.abs(b))
