"""Many independent recordings in one CUDA graph (ss_plan_many / ss_run_many):
every recording's spectra match the oracle on that recording; a replay of the
captured graph reproduces them; new inputs are captured anew."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
M_FR = 6


def P():
    import paper_2505_01231_gb300 as mod
    return mod


def recordings(seed):
    # frame lengths of their own, lengths from 3 to 40 groups with ragged tails
    Ts = [32, 64, 128, 256, 64, 32]
    groups = [40, 9, 17, 3, 25, 4]
    zs = [synth.ar1_quadratic(g * M_FR * T + 7 * i + 3, seed=seed + i, phi=0.5 + 0.08 * i)
          for i, (T, g) in enumerate(zip(Ts, groups))]
    return Ts, zs


def check(out, ref, tol4):
    assert out["G"] == ref["G"]
    for key in ("S2", "S3", "S4"):
        a, b = out[key][0].reshape(ref[key].shape), ref[key]
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err <= (tol4 if key == "S4" else TOL), f"{key}: {err:.2e}"
        ea, eb = out[key + "_err"][0].reshape(ref[key + "_err"].shape), ref[key + "_err"]
        assert np.max(np.abs(ea - eb)) / np.max(np.abs(eb)) <= 1e-4, key + "_err"


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_many_recordings_match_the_oracle_and_replay(precision):
    mod = P()
    Ts, zs = recordings(30)
    many = mod.ManyPlan(Ts, [len(z) + 1000 for z in zs], dt=0.5, m=M_FR, precision=precision)
    dz = [torch.from_numpy(z).cuda() for z in zs]
    many.run(dz)
    first = [many.results(i) for i in range(len(zs))]
    for i, (T, z) in enumerate(zip(Ts, zs)):
        check(first[i], oracle.polyspectra(z, T, 0.5, M_FR, group_chunk=8), TOL)
    many.run(dz)  # replay of the captured graph
    for i in range(len(zs)):
        again = many.results(i)
        for key in ("S2", "S3", "S4"):
            scale = np.max(np.abs(first[i][key]))
            assert np.max(np.abs(again[key] - first[i][key])) <= 1e-12 * scale
    # other inputs (new buffers, other lengths): captured anew
    Ts2, zs2 = recordings(50)
    zs2 = [z[: len(z) - (i % 3) * T] for i, (T, z) in enumerate(zip(Ts2, zs2))]
    dz2 = [torch.from_numpy(np.ascontiguousarray(z)).cuda() for z in zs2]
    many.run(dz2)
    for i, (T, z) in enumerate(zip(Ts2, zs2)):
        check(many.results(i), oracle.polyspectra(z, T, 0.5, M_FR, group_chunk=8), TOL)
    many.close()


def test_many_recordings_reject_bad_inputs():
    mod = P()
    Ts, zs = recordings(70)
    many = mod.ManyPlan(Ts, [len(z) for z in zs], m=M_FR)
    dz = [torch.from_numpy(z).cuda() for z in zs]
    with pytest.raises(mod.SSError) as ei:  # host memory input
        many.run([torch.from_numpy(zs[0])] + dz[1:])
    assert ei.value.status == mod.SS_EINVAL
    with pytest.raises(mod.SSError) as ei:  # more samples than planned
        many.run(dz, [len(z) + 1 for z in zs])
    assert ei.value.status == mod.SS_EINVAL
    many.run(dz)  # still usable
    assert many.results(0)["G"] == len(zs[0]) // (M_FR * Ts[0])
    many.close()
