"""Pins for the oracle's windows (Sec. 3, Eq. 17; App. B, Eq. 71) and its DFT (Eq. 18)."""
import numpy as np
import pytest
from scipy import optimize, signal

import oracle


@pytest.mark.parametrize("T", [8, 16, 256, 1024])
def test_dft_plus_equals_direct_sum(T):
    rng = np.random.default_rng(T)
    x = rng.normal(size=(3, T))
    assert np.allclose(oracle.dft_plus(x), oracle.dft_plus_direct(x), atol=1e-9 * T)


def test_dft_sign_positive_exponent():
    # x_i = sin(2 pi k0 i / T): sum_i sin(t) e^{+jt} = j T/2 at k0 (it would be -j T/2
    # with the negative exponent of numpy's forward transform)
    T, k0 = 64, 5
    i = np.arange(T)
    X = oracle.dft_plus(np.sin(2 * np.pi * k0 * i / T))
    assert np.isclose(X[k0], 1j * T / 2, atol=1e-10)
    X[k0] = 0
    assert np.max(np.abs(X)) < 1e-10


def test_parseval():
    T = 128
    x = np.random.default_rng(1).normal(size=T)
    X = oracle.dft_plus(x)
    energy = (abs(X[0]) ** 2 + 2 * np.sum(abs(X[1:-1]) ** 2) + abs(X[-1]) ** 2) / T
    assert np.isclose(energy, np.sum(x * x), rtol=1e-12)


@pytest.mark.parametrize("T", [8, 100, 1024])
def test_hann_is_periodic_hann(T):
    assert np.allclose(oracle.window(T, "hann"), signal.windows.hann(T, sym=False), atol=1e-15)


@pytest.mark.parametrize("T", [64, 1023, 4096])
def test_acg_small_sigma_is_gaussian(T):
    # for narrow windows the confinement correction is negligible: a Gaussian of
    # standard deviation sqrt(2) N sigma_t centred at (N-1)/2
    s = 0.05
    g = oracle.window(T, "acg", s)
    ref = signal.windows.gaussian(T, np.sqrt(2.0) * T * s, sym=True)
    assert np.allclose(g / g.max(), ref / ref.max(), atol=1e-9)


@pytest.mark.parametrize("T,s", [(64, 0.14), (1024, 0.14), (256, 0.3)])
def test_acg_confinement_condition(T, s):
    # App. B defines the correction so that the window's continuation vanishes half a
    # sample beyond both ends.  Solve that condition numerically for the weight of the
    # two shifted Gaussians and compare (up to scale) with the oracle's window.
    c = (T - 1) / 2.0

    def Gs(x):
        return np.exp(-((x - c) ** 2) / (2.0 * (np.sqrt(2.0) * T * s) ** 2))

    def cont(x, alpha):
        return Gs(x) - alpha * (Gs(x + T) + Gs(x - T))

    alpha = optimize.brentq(lambda a: cont(-0.5, a), 0.0, 1e6, xtol=1e-300, rtol=1e-15)
    assert abs(cont(T - 0.5, alpha)) < 1e-14
    ref = cont(np.arange(T, dtype=float), alpha)
    g = oracle.window(T, "acg", s)
    assert np.allclose(g / g.max(), ref / ref.max(), atol=1e-12)
    assert np.allclose(g, g[::-1], atol=1e-15)


def test_frame_groups_layout_and_drop():
    z = np.arange(2 * 3 * 4 + 5)
    f = oracle.frame_groups(z, 4, 3)
    assert f.shape == (2, 3, 4)
    assert f[1, 2, 3] == (1 * 3 + 2) * 4 + 3

