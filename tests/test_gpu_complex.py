"""Spectra of complex-valued signals (App. D) and shifted S4 planes (App. E) on the
GPU against the oracle, which takes the complex signals themselves (the GPU
takes their real and imaginary parts as real channels).  Tolerance: 1e-5 of each
spectrum's peak, 1e-4 for the standard errors.
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


def signals(T, m, G, seed):
    n = T * m * G + 13
    x1 = synth.ar1_quadratic(n, seed=seed, phi=0.8)
    y1 = synth.ar1_quadratic(n, seed=seed + 1, phi=0.3)
    x2 = synth.ar1_quadratic(n, seed=seed + 2, phi=0.6)
    y2 = synth.ar1_quadratic(n, seed=seed + 3, phi=-0.5)
    real = np.stack([x1, y1, x2, y2]).astype(np.float32)
    z = np.stack([real[0] + 1j * real[1], real[2] + 1j * real[3]])
    return real, z


# complex channel c -> (real channel, imaginary channel)
PARTS = {0: (0, 1), 1: (2, 3)}


def gpu_records(recs):
    return [(len(r),) + tuple((PARTS[c][0], PARTS[c][1], int(cj)) for c, cj in r) for r in recs]


def check(got, ref, key):
    (S, E), (Sr, Er) = got, ref
    scale = np.max(np.abs(Sr))
    err = np.max(np.abs(S - Sr)) / scale
    assert err <= TOL, f"{key}: {err:.3e}"
    eerr = np.max(np.abs(E - Er)) / np.max(Er)
    assert eerr <= TOL_ERR, f"{key} err: {eerr:.3e}"


@pytest.mark.parametrize("T,m,G,shift", [(32, 6, 40, 0), (64, 5, 30, 3), (16, 8, 60, -5),
                                         (256, 4, 12, 7)])
def test_complex_records_match_the_oracle(T, m, G, shift):
    real, z = signals(T, m, G, seed=T + m)
    s2 = [((0, False), (1, True)), ((0, False), (0, True))]          # z1 z2*, power of z1
    s3 = [((0, False), (1, False), (0, True))]
    s4 = [((0, False), (1, True), (1, False), (0, True)), ((1, False), (1, False), (0, True),
                                                           (0, True))]
    ref = oracle.complex_polyspectra(z, T, 0.5, m, s2_combos=s2, s3_combos=s3, s4_combos=s4,
                                     s4_shift=shift)
    mod = P()
    plan = mod.Plan(channels=4, T=T, dt=0.5, m=m, orders=(2,), combos=[(2, 0, 0, -1, -1)])
    recs = gpu_records(s4[:1] + s2 + s3 + s4[1:])       # records in any order of orders
    mod.ss_set_complex(plan.handle, recs, shift)
    plan.accumulate(torch.from_numpy(real).cuda())
    got = plan.complex_spectra(recs)
    plan.close()
    refs = [ref[("S4", s4[0])]] + [ref[("S2", c)] for c in s2] + [ref[("S3", s3[0])]] + \
        [ref[("S4", s4[1])]]
    for i, (g, r) in enumerate(zip(got, refs)):
        check(g, r, f"record {i}")


def test_complex_records_rules():
    mod = P()
    plan = mod.Plan(channels=2, T=32, m=4, orders=(2,))
    with pytest.raises(mod.SSError) as ei:
        mod.ss_set_complex(plan.handle, [(2, (0, 5, 0), (1, -1, 0))])
    assert ei.value.status == mod.SS_EINVAL
    with pytest.raises(mod.SSError) as ei:
        mod.ss_finalize_complex(plan.handle)
    assert ei.value.status == mod.SS_ESTATE
    mod.ss_set_complex(plan.handle, [(2, (0, 1, 0), (0, 1, 1))])
    with pytest.raises(mod.SSError) as ei:
        mod.ss_set_interlace(plan.handle, 1)
    assert ei.value.status == mod.SS_EUNSUPPORTED
    plan.close()
