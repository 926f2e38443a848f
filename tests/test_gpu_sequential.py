"""Sequential spectra and the m sweep of Sec. 8 on the GPU against the oracle.

Each block of B consecutive groups gives the block's mean and standard error of
the per-group estimates, in the finalize layout; blocks run across ss_accumulate
calls and device batches; blocks past the buffer are counted, not written; a
reset restarts the count.  Tolerance: 1e-5 of each spectrum's peak (within the
block), 1e-4 for the standard errors.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, TOL_ERR = 1e-5, 1e-4


def P():
    import paper_2505_01231_gb300 as mod
    return mod


def check_blocks(got, ref, orders):
    for b, blk in enumerate(got):
        for n in orders:
            key = f"S{n}"
            a, e = blk[key][0], blk[key + "_err"][0]
            r, re = ref[key][b], ref[key + "_err"][b]
            assert np.max(np.abs(a.reshape(r.shape) - r)) <= TOL * np.max(np.abs(r)), (b, key)
            assert np.max(np.abs(e.reshape(re.shape) - re)) <= TOL_ERR * np.max(re), (b, key)


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_blocks_across_calls_and_batches_match_the_oracle(precision):
    mod = P()
    T, m, B = 64, 6, 5
    G = 23                      # 4 whole blocks and 3 groups that form none
    z = synth.ar1_quadratic(T * m * G + 41, seed=12)
    ref = oracle.sequential_spectra(z, T, 0.5, m, B)
    full = oracle.polyspectra(z, T, 0.5, m)
    assert ref["blocks"] == 4
    plan = mod.Plan(T=T, dt=0.5, m=m, precision=precision)
    mod.ss_set_batch(plan.handle, 3)          # device batches of 3 groups: blocks span them
    plan.sequential(B, 3)                     # room for 3 of the 4 blocks
    for a, b in ((0, 1000), (1000, 4000), (4000, 6001), (6001, z.size)):
        plan.accumulate(torch.from_numpy(z[a:b].copy()).cuda(), b - a)
    out = plan.finalize()
    n, done = mod.ss_sequential_info(plan.handle)
    assert done == 4
    got = plan.blocks()
    assert len(got) == 3
    check_blocks(got, ref, (2, 3, 4))
    for key in ("S2", "S3", "S4"):          # the whole-record estimate is unchanged
        r = full[key]
        assert np.max(np.abs(out[key][0].reshape(r.shape) - r)) <= TOL * np.max(np.abs(r))
    plan.reset()                              # the count restarts
    assert mod.ss_sequential_info(plan.handle)[1] == 0
    plan.accumulate(torch.from_numpy(z).cuda())
    assert mod.ss_sequential_info(plan.handle)[1] == 4
    check_blocks(plan.blocks(), ref, (2, 3, 4))
    plan.close()


def test_sequential_rules():
    mod = P()
    plan = mod.Plan(T=32, m=4)
    with pytest.raises(mod.SSError) as ei:
        mod.ss_set_sequential(plan.handle, 1, None, 0)
    assert ei.value.status == mod.SS_EINVAL
    with pytest.raises(mod.SSError) as ei:       # host memory
        mod.ss_set_sequential(plan.handle, 4, np.zeros(1 << 16), 2)
    assert ei.value.status == mod.SS_EINVAL
    mod.ss_set_sequential(plan.handle, 4, None, 0)   # count only
    with pytest.raises(mod.SSError) as ei:
        mod.ss_set_interlace(plan.handle, 1)
    assert ei.value.status == mod.SS_EUNSUPPORTED
    plan.accumulate(torch.from_numpy(synth.ar1_quadratic(32 * 4 * 9, seed=2)).cuda())
    assert mod.ss_sequential_info(plan.handle)[1] == 2
    with pytest.raises(mod.SSError) as ei:       # only before data
        mod.ss_set_sequential(plan.handle, 0, None, 0)
    assert ei.value.status == mod.SS_ESTATE
    plan.close()


def test_am_noise_blocks_and_m_sweep():
    # amplitude-modulated white noise: the block power follows a(t)^2, and the
    # quasi-trispectrum grows with m (a group spanning the modulation period)
    mod = P()
    T, P_, depth, n = 64, 1 << 14, 0.9, 1 << 20
    t = np.arange(n)
    a = 1.0 + depth * np.sin(2 * np.pi * t / P_)
    z = (a * synth.normal(n, seed=3)).astype(np.float32)
    dz = torch.from_numpy(z).cuda()
    for m in (4, 256):
        ref = oracle.sequential_spectra(z, T, 1.0, m, 8, orders=(2, 4))
        # the tensor-core S4 takes m <= 32; m = 256 runs on CUDA cores
        plan = mod.Plan(T=T, m=m, orders=(2, 4), precision="tf32x3" if m <= 32 else "fp32")
        plan.sequential(8, ref["blocks"])
        plan.accumulate(dz)
        check_blocks(plan.blocks(), ref, (2, 4))
        plan.close()
    sweep = mod.sweep_m(dz, T, (4, 256), orders=(2, 4), precision="fp32")
    d = np.arange(2, T // 2 - 1)
    for m, expect_large in ((4, False), (256, True)):
        ref = oracle.polyspectra(z, T, 1.0, m, orders=(2, 4), group_chunk=64)
        got = sweep[m]
        for key in ("S2", "S4"):
            r = ref[key]
            assert np.max(np.abs(got[key][0].reshape(r.shape) - r)) <= TOL * np.max(np.abs(r))
        s4 = got["S4"][0][d, d].real
        zscore = np.mean(s4) / np.sqrt(np.mean(got["S4_err"][0][d, d, 0] ** 2) / d.size)
        assert (zscore > 20) == expect_large, (m, zscore)
