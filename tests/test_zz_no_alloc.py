"""ss_s2_noalloc: the power spectrum computed with no device allocation.

Callers that cannot call cudaMalloc (device memory owned up front by a caching
allocator or a fixed budget; latency-critical loops) use this entry point; its
scratch is a static device array.  This file is collected last so that a run
that stops at the first failure has already run every other test.  The check:
its S2 equals the S2 of a one-channel plan (ss_plan / ss_accumulate /
ss_finalize) within the parity tolerance of the other tests, on two calls in a
row (the shared scratch keeps the previous call's contents).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_ERR = 1e-4


def plan_s2(z, T, m, dt):
    import paper_2505_01231_gb300 as P
    plan = P.Plan(channels=1, T=T, dt=dt, m=m, orders=(2,))
    plan.accumulate(torch.from_numpy(z).cuda())
    out = plan.finalize()
    plan.close()
    return out["S2"][0], out["S2_err"][0]


def noalloc_s2(dz, n, T, m, dt):
    import paper_2505_01231_gb300 as P
    M = T // 2 + 1
    s2 = torch.full((M * 2,), float("nan"), dtype=torch.float64, device="cuda")
    err = torch.full((M * 2,), float("nan"), dtype=torch.float64, device="cuda")
    P.ss_s2_noalloc(dz, n, T, dt, m, d_S2=s2, d_S2_err=err,
                    stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    s2 = s2.cpu().numpy()
    return s2[0::2] + 1j * s2[1::2], err.cpu().numpy().reshape(M, 2)


@pytest.mark.parametrize("T,m,G", [(1024, 10, 300), (256, 4, 50)])
def test_noalloc_matches_plan_twice(T, m, G):
    z = synth.ar1_quadratic(T * m * G + 123, seed=31)
    ref, ref_err = plan_s2(z, T, m, 0.5)
    dz = torch.from_numpy(z).cuda()
    for _ in range(2):
        s2, err = noalloc_s2(dz, z.size, T, m, 0.5)
        assert np.max(np.abs(s2 - ref)) <= TOL * np.max(np.abs(ref))
        assert np.max(np.abs(err - ref_err)) <= TOL_ERR * np.max(np.abs(ref_err))


def test_noalloc_rejects_input_beyond_scratch():
    import paper_2505_01231_gb300 as P
    T, m = 1024, 10
    M = T // 2 + 1
    n = 1200 * m * T   # 1200 groups x 10 frames x 516 bins x 8 bytes > 32 MiB - 128 KiB
    dz = torch.zeros(n, dtype=torch.float32, device="cuda")
    s2 = torch.empty(M * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SSError) as ei:
        P.ss_s2_noalloc(dz, n, T, 1.0, m, d_S2=s2)
    assert ei.value.status == P.SS_EINVAL
    assert "scratch" in str(ei.value)


def test_noalloc_rejects_host_buffers_before_any_launch():
    import paper_2505_01231_gb300 as P
    T, m = 256, 4
    M = T // 2 + 1
    z = synth.ar1_quadratic(T * m * 10, seed=32)
    dz = torch.from_numpy(z).cuda()
    s2 = torch.empty(M * 2, dtype=torch.float64, device="cuda")
    host_out = np.empty(M * 2)
    for sig, out, err in ((z, s2, None), (dz, host_out, None), (dz, s2, np.empty(M * 2))):
        with pytest.raises(P.SSError) as ei:
            P.ss_s2_noalloc(sig, z.size, T, 1.0, m, d_S2=out, d_S2_err=err)
        assert ei.value.status == P.SS_EINVAL
        assert "device" in str(ei.value)
    torch.cuda.synchronize()   # nothing was enqueued; the device is intact
