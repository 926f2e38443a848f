"""Spectrum-level pins for the oracle (Sec. 3-4, 7, 9; App. C).

* exact expectations for i.i.d. white noise (multilinearity of cumulants + Eq. 23,
  28, 31): E[S2] = dt k2, E[S3] = dt^2 k3, E[S4] = dt^3 k4 at every bin;
* closed-form finite-window S2 of an AR(1) Gaussian with independent frames;
* Gaussian null for S3 and S4 (Sec. 4.3) and the incomplete cumulant of Eq. 39 as a
  negative control;
* estimator-level symmetries (Sec. 9) and invariances (App. C) that hold to rounding.
"""
import numpy as np
import pytest

import oracle
import synth


def zscores(mean, err, expect):
    return (mean.real - expect) / err[..., 0]


def test_iid_exponential_noise_exact_expectations():
    # centred unit exponential: k2 = 1, k3 = 2, k4 = 6
    T, m, G, dt = 16, 5, 6000, 0.5
    z = synth.exponential_centred(T * m * G, seed=21)
    r = oracle.polyspectra(z, T, dt, m, group_chunk=500)
    M = T // 2 + 1
    z2 = zscores(r["S2"], r["S2_err"], dt * 1.0)
    kk, ll = oracle.s3_domain(M)
    z3 = zscores(r["S3"][kk, ll], r["S3_err"][kk, ll], dt * dt * 2.0)
    z4 = zscores(r["S4"], r["S4_err"], dt ** 3 * 6.0)
    for zz in (z2, z3, z4):
        assert np.max(np.abs(zz)) < 5.0
    # pooled over bins the ratio to the closed form is pinned to a few percent, far
    # tighter than any wrong prefactor or window sum would allow (m/(m-1) = 1.25,
    # sum g^3 / sum g^4 = 8/7 for the Hann window)
    assert abs(np.mean(r["S2"].real) / (dt * 1.0) - 1.0) < 0.02
    assert abs(np.mean(r["S3"][kk, ll].real) / (dt * dt * 2.0) - 1.0) < 0.03
    assert abs(np.mean(r["S4"].real) / (dt ** 3 * 6.0) - 1.0) < 0.05


def test_ar1_gaussian_s2_closed_form():
    # independent stationary AR(1) frames: E[S2(k)] = dt/sum g^2 v^T R v*, with
    # v_i = g_i e^{2 pi j ik/T} and R the AR(1) autocovariance phi^|i-i'|/(1-phi^2)
    T, m, G, dt, phi = 32, 10, 1500, 2.0, 0.8
    z = synth.iid_frames_ar1(m * G, T, phi, seed=4)
    r = oracle.polyspectra(z, T, dt, m, orders=(2,), group_chunk=500)
    g = oracle.window(T, "hann")
    i = np.arange(T)
    R = phi ** np.abs(i[:, None] - i[None, :]) / (1 - phi * phi)
    M = T // 2 + 1
    expect = np.empty(M)
    for k in range(M):
        v = g * np.exp(2j * np.pi * i * k / T)
        expect[k] = (dt / np.sum(g * g) * (v @ R @ np.conj(v))).real
    zz = zscores(r["S2"], r["S2_err"], expect)
    assert np.max(np.abs(zz)) < 5.0
    assert np.max(np.abs(r["S2"].imag)) < 1e-9 * np.max(expect)


def incomplete_c4(x, y, z, w):
    # Eq. 39: mean of the centred product with neither pair terms nor prefactors
    d = [v - v.mean(axis=-1, keepdims=True) for v in (x, y, z, w)]
    return (d[0] * d[1] * d[2] * d[3]).mean(axis=-1)


def test_gaussian_null_and_incomplete_cumulant_control():
    T, m, G, dt = 16, 10, 3000, 1.0
    z = synth.normal(T * m * G, seed=8)
    r = oracle.polyspectra(z, T, dt, m, orders=(3, 4), group_chunk=500)
    M = T // 2 + 1
    kk, ll = oracle.s3_domain(M)
    z3 = zscores(r["S3"][kk, ll], r["S3_err"][kk, ll], 0.0)
    z4 = zscores(r["S4"], r["S4_err"], 0.0)
    assert np.max(np.abs(z3)) < 5.0 and np.max(np.abs(z4)) < 5.0
    assert 0.5 < np.mean(z4 ** 2) < 2.0
    # the incomplete cumulant shows a spurious offset on Gaussian noise (Sec. 4.3)
    X = oracle.fourier_coefficients(z, T, m, oracle.window(T))
    k4, l4 = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    k4, l4 = k4.ravel(), l4.ravel()
    x = np.swapaxes(oracle.coef(X, k4), -1, -2)
    y = np.swapaxes(np.conj(oracle.coef(X, k4)), -1, -2)
    zc = np.swapaxes(oracle.coef(X, l4), -1, -2)
    w = np.swapaxes(np.conj(oracle.coef(X, l4)), -1, -2)
    bad = incomplete_c4(x, y, zc, w).real
    mean, er, _ = oracle.mean_and_stderr(bad)
    assert np.median(np.abs(mean / er)) > 20.0


@pytest.fixture(scope="module")
def two_channels():
    zs = synth.multichannel_shared(2, 32 * 6 * 40, seed=2)
    return zs


def test_single_channel_symmetries():
    z = synth.ar1_quadratic(64 * 6 * 30, seed=3)
    r = oracle.polyspectra(z, 64, 1.0, 6)
    S3, S4 = r["S3"], r["S4"]
    assert np.allclose(S3, S3.T, rtol=0, atol=1e-10 * np.abs(S3).max())
    assert np.allclose(S4, S4.T, rtol=0, atol=1e-10 * np.abs(S4).max())
    assert np.max(np.abs(S4.imag)) < 1e-10 * np.abs(S4).max()
    assert np.max(np.abs(r["S2"].imag)) < 1e-12 * np.abs(r["S2"]).max()


def test_cross_spectra_symmetries_and_isomorphisms(two_channels):
    zs = two_channels
    T, m = 32, 6
    M = T // 2 + 1
    r = oracle.cross_polyspectra(zs, T, 1.0, m, s2_combos=[(0, 1), (1, 0), (0, 0)],
                                 s3_combos=[(0, 1, 1), (1, 1, 0), (0, 0, 0)],
                                 s4_combos=[(0, 0, 0, 0), (0, 1, 0, 1), (0, 1, 1, 0)])
    # Eq. 56: S_xy = S_yx*
    assert np.allclose(r[("S2", (0, 1))][0], np.conj(r[("S2", (1, 0))][0]), atol=1e-10)
    # identical channels give the single-channel spectrum (Sec. 7)
    single = oracle.polyspectra(zs[0], T, 1.0, m)
    assert np.allclose(r[("S2", (0, 0))][0], single["S2"], atol=1e-10)
    S3c = r[("S3", (0, 0, 0))][0]
    assert np.allclose(S3c[M - 1:, :], single["S3"], atol=1e-8 * np.abs(single["S3"]).max())
    S4c = r[("S4", (0, 0, 0, 0))][0]
    assert np.allclose(S4c[M - 1:, :], single["S4"], atol=1e-8 * np.abs(single["S4"]).max())
    # Eq. 61: S_yyx(k, l) = S_xyy(-k-l, k) with x = channel 0, y = channel 1
    Sxyy, Syyx = r[("S3", (0, 1, 1))][0], r[("S3", (1, 1, 0))][0]
    kk, ll = oracle.cross_domain_s3(M)
    k2, l2 = -kk - ll, kk
    ok = (l2 >= 0)
    lhs = Syyx[kk[ok] + M - 1, ll[ok]]
    rhs = Sxyy[k2[ok] + M - 1, l2[ok]]
    assert np.allclose(lhs, rhs, atol=1e-10 * np.abs(Sxyy).max())
    # Sec. 9: S4_xyxy and S4_xyyx carry the same information.  Swapping the last two
    # cumulant arguments and using a_{-k} = a_k* gives S4_xyxy(k, l) = S4_xyyx(k, -l)
    # = conj S4_xyyx(-k, l)
    S_xyxy, S_xyyx = r[("S4", (0, 1, 0, 1))][0], r[("S4", (0, 1, 1, 0))][0]
    assert np.allclose(S_xyxy, np.conj(S_xyyx[::-1, :]), atol=1e-10 * np.abs(S_xyxy).max())
    # single channel: the cut is real and even in k (T13 of Sec. 9)
    assert np.allclose(S4c, S4c[::-1, :], atol=1e-10 * np.abs(S4c).max())


def test_invariances():
    T, m = 32, 6
    z = synth.ar1_quadratic(T * m * 25, seed=9).astype(np.float64)
    base = oracle.polyspectra(z, T, 0.7, m, window_kind="acg")
    # additive constant: k-statistics of order >= 2 are translation invariant
    shifted = oracle.polyspectra(z + 3.25, T, 0.7, m, window_kind="acg")
    for key in ("S2", "S3", "S4"):
        assert np.allclose(shifted[key], base[key], atol=1e-9 * np.abs(base[key]).max())
    # scaling z by s scales S_n by s^n
    scaled = oracle.polyspectra(2.0 * z, T, 0.7, m, window_kind="acg")
    for key, n in (("S2", 2), ("S3", 3), ("S4", 4)):
        assert np.allclose(scaled[key], 2.0 ** n * base[key], atol=1e-9 * 2 ** n * np.abs(base[key]).max())
    # App. C: time reversal conjugates every spectrum (window symmetric about (T-1)/2)
    rev = oracle.polyspectra(z[::-1].copy(), T, 0.7, m, window_kind="acg")
    for key in ("S2", "S3", "S4"):
        assert np.allclose(rev[key], np.conj(base[key]), atol=1e-9 * np.abs(base[key]).max())


def test_window_scale_invariance():
    T, m = 16, 5
    z = synth.ar1_quadratic(T * m * 20, seed=1)
    a = oracle.polyspectra(z, T, 1.0, m)
    # replacing g by c g leaves every spectrum unchanged (window defined up to a factor)
    import importlib
    op = importlib.import_module("oracle.polyspectra")
    orig = op.window
    try:
        op.window = lambda T_, kind="hann", s=0.14: 3.0 * orig(T_, kind, s)
        b = op.polyspectra(z, T, 1.0, m)
    finally:
        op.window = orig
    for key in ("S2", "S3", "S4"):
        assert np.allclose(a[key], b[key], atol=1e-9 * np.abs(a[key]).max())


def test_standard_error_matches_scipy_sem():
    # Eq. 35-36: Var with the N_p/(N_p-1) correction, sigma = sqrt(Var/N_p), i.e.
    # the standard error of the mean with ddof=1
    from scipy import stats
    rng = np.random.default_rng(0)
    Sg = rng.normal(size=(5, 7)) + 1j * rng.normal(size=(5, 7)) * 3
    mean, er, ei = oracle.mean_and_stderr(Sg)
    assert np.allclose(er, stats.sem(Sg.real, axis=0, ddof=1), rtol=1e-12)
    assert np.allclose(ei, stats.sem(Sg.imag, axis=0, ddof=1), rtol=1e-12)
    assert np.allclose(mean, Sg.mean(axis=0))


def test_running_sums_equal_per_group_statistics():
    # polyspectra() accumulates sums of S, Re^2, Im^2 over group chunks; its result
    # must equal the per-group values fed to scipy's standard error
    from scipy import stats
    T, m, dt = 16, 4, 1.5
    z = synth.ar1_quadratic(T * m * 6, seed=11)
    r = oracle.polyspectra(z, T, dt, m, group_chunk=4)
    g = oracle.window(T)
    X = oracle.fourier_coefficients(z, T, m, g)
    s2 = oracle.s2_groups(X, X, dt, g)
    kk, ll = oracle.s3_domain(T // 2 + 1)
    s3 = oracle.s3_groups(X, X, X, dt, g, kk, ll)
    assert r["G"] == 6
    assert np.allclose(r["S2_err"][:, 0], stats.sem(s2.real, axis=0, ddof=1), rtol=1e-9)
    assert np.allclose(r["S3_err"][kk, ll, 0], stats.sem(s3.real, axis=0, ddof=1), rtol=1e-8, atol=1e-12)
    assert np.allclose(r["S3_err"][kk, ll, 1], stats.sem(s3.imag, axis=0, ddof=1), rtol=1e-8, atol=1e-12)
    assert np.allclose(r["S3"][kk, ll], s3.mean(axis=0))


def test_interlaced_estimate_pools_the_two_window_sets():
    # with as many shifted groups as unshifted ones, the pooled estimate is the
    # average of the two spectra; the shifted set is the record without its first
    # T/2 samples
    T, m, G = 32, 5, 12
    z = synth.ar1_quadratic(T * m * G + T // 2, seed=8)
    both = oracle.polyspectra(z, T, 0.5, m, orders=(1, 2, 3, 4), interlaced=True)
    a = oracle.polyspectra(z, T, 0.5, m, orders=(1, 2, 3, 4))
    b = oracle.polyspectra(z[T // 2:], T, 0.5, m, orders=(1, 2, 3, 4))
    assert both["G"] == a["G"] + b["G"] == 2 * G
    for key in ("S1", "S2", "S3", "S4"):
        assert np.allclose(both[key], 0.5 * (a[key] + b[key]), rtol=1e-12, atol=1e-14)
