"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/polyspec.h, and rejects invalid arguments before any CUDA call."""
import os
import re

import pytest

import paper_2505_01231_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ss_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert "ss_plan" in names and "ss_accumulate" in names and "ss_finalize" in names
    for n in names:
        assert hasattr(P.lib, n), n


def test_version():
    assert "sm_103a" in P.ss_version()


@pytest.mark.parametrize("kw,msg", [
    (dict(channels=0), "channels"),
    (dict(channels=5), "channels"),
    (dict(T=100), "power of two"),
    (dict(T=4), "power of two"),
    (dict(T=8192), "power of two"),
    (dict(dt=0.0), "dt"),
    (dict(dt=float("nan")), "dt"),
    (dict(m=3), "m >= 4"),
    (dict(m=2, orders=P.SS_ORDER3), "m >= 3"),
    (dict(m=1, orders=P.SS_ORDER2), "m >= 2"),
    (dict(orders=0), "orders"),
    (dict(orders=1), "orders"),
    (dict(orders=1 << 5), "orders"),
    (dict(window=7), "window"),
    (dict(window=P.SS_WIN_ACG, win_param=-1.0), "sigma_t"),
    (dict(dtype=9), "dtype"),
    (dict(precision=9), "precision"),
    (dict(combos=[(3, 0, 0, 0, -1)], orders=P.SS_ORDER2), "order"),
    (dict(combos=[(2, 0, 3, -1, -1)], channels=2, orders=P.SS_ORDER2), "channel"),
])
def test_plan_rejects_invalid_arguments(kw, msg):
    args = dict(channels=1, T=256, dt=1.0, m=10, window=P.SS_WIN_HANN, win_param=0.14,
                orders=P.SS_ORDER2 | P.SS_ORDER3 | P.SS_ORDER4, dtype=P.SS_F32,
                precision=P.SS_PREC_FP32, combos=None)
    args.update(kw)
    with pytest.raises(P.SSError) as ei:
        P.ss_plan(**args)
    assert ei.value.status == P.SS_EINVAL
    assert msg in str(ei.value)


def test_null_plan_calls_fail_cleanly():
    assert P.lib.ss_accumulate(None, None, 0) == P.SS_EINVAL
    assert P.lib.ss_finalize(None, None, None, None, None, None, None) == P.SS_EINVAL
    assert P.lib.ss_reset(None) == P.SS_EINVAL
    assert P.lib.ss_state_size(None, None) == P.SS_EINVAL
    assert P.lib.ss_export_state(None, None) == P.SS_EINVAL
    assert P.lib.ss_merge_state(None, None) == P.SS_EINVAL
    assert P.lib.ss_run_many(None, None, None, None, None, None, None, None, None) == P.SS_EINVAL
    assert P.lib.ss_many_plan(None, 0, None) == P.SS_EINVAL
    assert P.lib.ss_destroy_many(None) == P.SS_OK
    assert P.lib.ss_set_estimator(None, 0) == P.SS_EINVAL
    assert P.lib.ss_finalize_s1(None, None, None) == P.SS_EINVAL
    assert P.lib.ss_set_interlace(None, 1) == P.SS_EINVAL
    assert P.lib.ss_destroy(None) == P.SS_OK


@pytest.mark.parametrize("precision", ["SS_PREC_TF32X3", "SS_PREC_BF16X3", "SS_PREC_BF16"])
def test_tensor_core_s4_rejects_more_than_32_frames(precision):
    # the Gram contraction holds m(m+1)/2 products per bin: m <= 32 on the tensor cores
    args = dict(channels=1, T=256, dt=1.0, m=33, window=P.SS_WIN_HANN, win_param=0.14,
                orders=P.SS_ORDER2 | P.SS_ORDER4, dtype=P.SS_F32,
                precision=getattr(P, precision), combos=None)
    with pytest.raises(P.SSError) as ei:
        P.ss_plan(**args)
    assert ei.value.status == P.SS_EUNSUPPORTED
    assert "m <= 32" in str(ei.value)


@pytest.mark.parametrize("Ts,lens,msg", [([100, 64], [10000, 10000], "power of two"),
                                         ([64, 64], [10000, 700], "fewer than two groups"),
                                         ([], [], "n_rec")])
def test_plan_many_rejects_invalid_arguments(Ts, lens, msg):
    with pytest.raises(P.SSError) as ei:
        P.ss_plan_many(Ts, lens, 1.0, 6)
    assert ei.value.status == P.SS_EINVAL
    assert msg in str(ei.value)
