"""The autotuner and every kernel form it chooses between.

Each K1 form (resident groups in 74 KB or 96 KB, a warp per frame, frame at a time) and each K2
tiling (4 x 4 micro-tiles, 8 x 4 micro-tiles with two or three stages or in independent warps)
must give
the oracle's spectra; ss_autotune must leave a plan that does; the tuning text
round-trips and refuses a plan of another configuration.
Tolerance as in the parity tests: 1e-5 of each spectrum's peak, 1e-4 for the
standard errors.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, TOL_ERR = 1e-5, 1e-4
K1_FORMS = ["auto", "r96", "frames", "warp"]
K2_FORMS = ["44", "44s3", "84s2", "84s3", "84w"]


def P():
    import paper_2505_01231_gb300 as mod
    return mod


def close(a, b, tol):
    return np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))


def run(z, T, m, tuning, channels=1, orders=(2, 3), combos=None, precision="fp32"):
    mod = P()
    plan = mod.Plan(channels=channels, T=T, m=m, orders=orders, combos=combos,
                    precision=precision)
    mod.ss_set_tuning(plan.handle, tuning)
    plan.accumulate(torch.from_numpy(np.ascontiguousarray(z)).cuda())
    out = plan.finalize()
    plan.close()
    return out


@pytest.mark.parametrize("k2", K2_FORMS)
@pytest.mark.parametrize("T,m,G", [(8, 4, 50), (64, 17, 12), (256, 10, 50), (512, 7, 9),
                                   (4096, 4, 3), (32, 40, 8)])
def test_k2_forms_match_the_oracle(T, m, G, k2):
    # ragged tails; m = 17 and 40 take two or three staged chunks per group
    z = synth.ar1_quadratic(T * m * G + 2 * T + 1, seed=T + m)
    ref = oracle.polyspectra(z, T, 1.0, m, orders=(3,), group_chunk=8)
    out = run(z, T, m, f"k2={k2}", orders=(3,))
    a = out["S3"][0].reshape(ref["S3"].shape)
    assert close(a, ref["S3"], TOL)
    assert close(out["S3_err"][0].reshape(ref["S3_err"].shape), ref["S3_err"], TOL_ERR)


# the independent-warp form streams an item's frames four at a time across group
# boundaries: m = 10 (the bench's shape), 13 and 6 (groups ending inside a stage),
# 16 at T = 2048; ragged tails
@pytest.mark.parametrize("T,m,G", [(1024, 10, 20), (1024, 13, 7), (2048, 16, 4), (512, 6, 33)])
def test_k2_independent_warps_match_the_oracle(T, m, G):
    z = synth.ar1_quadratic(T * m * G + 3 * T + 7, seed=T + m)
    ref = oracle.polyspectra(z, T, 1.0, m, orders=(3,), group_chunk=8)
    out = run(z, T, m, "k2=84w", orders=(3,))
    assert close(out["S3"][0].reshape(ref["S3"].shape), ref["S3"], TOL)
    assert close(out["S3_err"][0].reshape(ref["S3_err"].shape), ref["S3_err"], TOL_ERR)


@pytest.mark.parametrize("k2", K2_FORMS)
def test_k2_forms_several_channels(k2):
    # cross domains with negative k: the tiles staged by the threads, not by TMA
    T, m, G, C = 64, 5, 30, 3
    zs = synth.multichannel_shared(C, T * m * G + 9, seed=41)
    c3 = [(0, 1, 2), (2, 2, 0), (1, 1, 1)]
    ref = oracle.cross_polyspectra(zs, T, 1.0, m, s3_combos=c3, group_chunk=8)
    out = run(zs, T, m, f"k2={k2}", channels=C, orders=(3,),
              combos=[(3,) + c + (-1,) for c in c3])
    for i, c in enumerate(c3):
        b = ref[("S3", c)][0]
        assert close(out["S3"][i].reshape(b.shape), b, TOL), c


@pytest.mark.parametrize("k1", K1_FORMS)
@pytest.mark.parametrize("T,m,G", [(256, 10, 40), (1024, 10, 6), (4096, 4, 3), (16, 300, 4),
                                   (8, 4, 50), (512, 20, 5)])
def test_k1_forms_match_the_oracle(T, m, G, k1):
    z = synth.ar1_quadratic(T * m * G + 5, seed=3 * T + m)
    ref = oracle.polyspectra(z, T, 1.0, m, orders=(2, 4), group_chunk=8)
    # the operand image of the tensor-core S4 is part of K1: written in TF32x3 at the
    # larger T (at T = 8 the split modes stay above 1e-5 of the S4 peak, see the
    # tensor-core size tests), FP32 otherwise
    out = run(z, T, m, f"k1={k1}", orders=(2, 4), precision="tf32x3" if T >= 256 else "fp32")
    for key in ("S2", "S4"):
        a = out[key][0].reshape(ref[key].shape)
        assert close(a, ref[key], TOL), key
        assert close(out[key + "_err"][0].reshape(ref[key + "_err"].shape),
                     ref[key + "_err"], TOL_ERR), key


def test_autotune_then_results_and_the_tuning_text():
    mod = P()
    T, m = 512, 10
    z = synth.ar1_quadratic(T * m * 60 + 77, seed=5)
    ref = oracle.polyspectra(z, T, 1.0, m, group_chunk=16)
    plan = mod.Plan(T=T, m=m, precision="tf32x3")
    best = mod.ss_autotune(plan.handle)
    assert best > 0
    text = mod.ss_get_tuning(plan.handle)
    assert text.startswith("polyspec-tuning 1 T=512 m=10 C=1 dtype=f32 prec=tf32x3")
    assert " k1=" in text and " k2=" in text and "k2:84s2=" in text
    plan.accumulate(torch.from_numpy(z).cuda())
    out = plan.finalize()
    for key in ("S2", "S3", "S4"):
        assert close(out[key][0].reshape(ref[key].shape), ref[key], TOL), key
    with pytest.raises(mod.SSError) as ei:   # only before data (or after a reset)
        mod.ss_autotune(plan.handle)
    assert ei.value.status == mod.SS_ESTATE
    plan.close()
    # the text applies to a plan of the same configuration, not to another one
    same = mod.Plan(T=T, m=m, precision="tf32x3")
    mod.ss_set_tuning(same.handle, text)
    assert mod.ss_get_tuning(same.handle).split(" | ")[1] == text.split(" | ")[1]
    same.close()
    other = mod.Plan(T=256, m=m, precision="tf32x3")
    with pytest.raises(mod.SSError) as ei:
        mod.ss_set_tuning(other.handle, text)
    assert ei.value.status == mod.SS_EINVAL
    with pytest.raises(mod.SSError):
        mod.ss_set_tuning(other.handle, "k2=99")
    other.close()
