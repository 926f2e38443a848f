"""Pins for the oracle's k-statistics (Sec. 4.1, Eq. 32-34; App. H, Eq. 85).

Each check ties the oracle to something other than its own formulas:
* exact expectations by brute-force enumeration equal population joint cumulants
  computed by the general set-partition (Moebius) formula -- unbiasedness, Sec. 4.1;
* the univariate case equals Fisher's k-statistics as implemented in scipy;
* the bivariate case equals the sample covariance (numpy, ddof=1).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def set_partitions(items):
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for p in set_partitions(rest):
        for i in range(len(p)):
            yield p[:i] + [[first] + p[i]] + p[i + 1:]
        yield [[first]] + p


def joint_cumulant(cols, support, probs):
    """kappa(V_cols[0], ..., V_cols[n-1]) of a discrete random vector V.

    kappa = sum over set partitions pi of (|pi|-1)! (-1)^(|pi|-1) prod_B E[prod_{i in B} V_i].
    """
    n = len(cols)
    total = 0.0 + 0.0j
    for part in set_partitions(list(range(n))):
        b = len(part)
        term = (-1) ** (b - 1) * math.factorial(b - 1)
        for block in part:
            v = np.ones(len(probs), dtype=np.complex128)
            for i in block:
                v = v * support[:, cols[i]]
            term = term * np.sum(probs * v)
        total += term
    return total


def brute_expectation(fn, cols, support, probs, m):
    """Exact E[fn(sample_1..m)] for m i.i.d. draws of the discrete vector."""
    S = len(probs)
    tuples = np.array(list(itertools.product(range(S), repeat=m)))  # [S^m, m]
    w = np.prod(probs[tuples], axis=1)
    args = [support[tuples, c] for c in cols]  # each [S^m, m]
    return np.sum(w * fn(*args))


@pytest.fixture(scope="module")
def distribution():
    rng = np.random.default_rng(12345)
    support = rng.normal(size=(3, 4)) + 1j * rng.normal(size=(3, 4)) + 0.7
    probs = np.array([0.2, 0.5, 0.3])
    return support, probs


@pytest.mark.parametrize("m", [4, 5, 6])
def test_c2_c3_c4_unbiased_by_enumeration(distribution, m):
    support, probs = distribution
    for cols in [(0, 1), (2, 2), (1, 3)]:
        e = brute_expectation(oracle.c2, cols, support, probs, m)
        assert abs(e - joint_cumulant(cols, support, probs)) < 1e-11
    for cols in [(0, 1, 2), (3, 3, 1), (2, 2, 2)]:
        e = brute_expectation(oracle.c3, cols, support, probs, m)
        assert abs(e - joint_cumulant(cols, support, probs)) < 1e-11
    for cols in [(0, 1, 2, 3), (0, 0, 1, 1), (3, 3, 3, 3), (2, 1, 2, 0)]:
        kappa = joint_cumulant(cols, support, probs)
        e_raw = brute_expectation(oracle.c4, cols, support, probs, m)
        e_fac = brute_expectation(oracle.c4_factorised, cols, support, probs, m)
        assert abs(e_raw - kappa) < 1e-10 * max(1.0, abs(kappa))
        assert abs(e_fac - kappa) < 1e-10 * max(1.0, abs(kappa))


def test_natural_estimator_is_biased(distribution):
    # negative control: dropping the k-statistic prefactors must fail the same check
    support, probs = distribution
    m = 5
    cols = (0, 1, 2, 3)

    def natural_c4(x, y, z, w):
        mm = x.shape[-1]
        return oracle.c4_factorised(x, y, z, w) * ((mm - 1) * (mm - 2) * (mm - 3)) / (mm * mm * (mm + 1))

    kappa = joint_cumulant(cols, support, probs)
    e = brute_expectation(natural_c4, cols, support, probs, m)
    assert abs(e - kappa) > 1e-3 * abs(kappa)


@pytest.mark.parametrize("m", [4, 7, 25])
def test_univariate_equals_fisher_kstat(m):
    rng = np.random.default_rng(m)
    x = rng.gamma(2.0, size=m) - 1.3
    assert np.isclose(oracle.c2(x, x), stats.kstat(x, 2), rtol=1e-12, atol=1e-14)
    assert np.isclose(oracle.c3(x, x, x), stats.kstat(x, 3), rtol=1e-11, atol=1e-13)
    assert np.isclose(oracle.c4(x, x, x, x), stats.kstat(x, 4), rtol=1e-10, atol=1e-12)
    assert np.isclose(oracle.c4_factorised(x, x, x, x), stats.kstat(x, 4), rtol=1e-10, atol=1e-12)


def test_c2_equals_sample_covariance():
    rng = np.random.default_rng(3)
    x, y = rng.normal(size=(2, 11))
    assert np.isclose(oracle.c2(x, y), np.cov(x, y, ddof=1)[0, 1], rtol=1e-13)


def test_c4_raw_equals_factorised_on_complex_data():
    rng = np.random.default_rng(7)
    v = rng.normal(size=(4, 50, 10)) + 1j * rng.normal(size=(4, 50, 10)) + 3.0
    a = oracle.c4(*v)
    b = oracle.c4_factorised(*v)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(a))


def test_translation_invariance_and_multilinearity():
    rng = np.random.default_rng(5)
    v = rng.normal(size=(4, 9)) + 1j * rng.normal(size=(4, 9))
    shift = np.array([1.5, -2.0 + 1j, 0.3j, 4.0])[:, None]
    w = v + shift
    assert np.allclose(oracle.c3(*w[:3]), oracle.c3(*v[:3]), atol=1e-11)
    assert np.allclose(oracle.c4(*w), oracle.c4(*v), atol=1e-10)
    u = rng.normal(size=9)
    lhs = oracle.c3(v[0] + 2.0 * u, v[1], v[2])
    rhs = oracle.c3(v[0], v[1], v[2]) + 2.0 * oracle.c3(u, v[1], v[2])
    assert np.allclose(lhs, rhs, atol=1e-11)


# ---------------------------------------------------------------- natural estimators
def _complex_samples(rng, m, n=4):
    return [rng.normal(size=m) + 1j * rng.normal(size=m) + 0.3 * i for i in range(n)]


@pytest.mark.parametrize("m", [3, 5, 11])
def test_natural_c2_c3_are_the_k_statistics_rescaled(m):
    # the empirical cumulants of orders 2 and 3 are the central moments, which differ
    # from the k-statistics by (m-1)/m and (m-1)(m-2)/m^2
    x, y, z, _ = _complex_samples(np.random.default_rng(m), m)
    assert np.isclose(oracle.c2_natural(x, y), (m - 1) / m * oracle.c2(x, y), rtol=1e-13)
    assert np.isclose(oracle.c3_natural(x, y, z), (m - 1) * (m - 2) / m ** 2 * oracle.c3(x, y, z),
                      rtol=1e-12)


@pytest.mark.parametrize("m", [4, 9, 30])
def test_natural_univariate_c4_equals_scipy_central_moments(m):
    x = np.random.default_rng(10 + m).gamma(2.0, size=m) - 1.1
    want = stats.moment(x, 4) - 3.0 * stats.moment(x, 2) ** 2
    assert np.isclose(oracle.c4_natural(x, x, x, x), want, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("m", [4, 6, 13])
def test_natural_estimators_are_the_cumulants_of_the_empirical_distribution(m):
    # the set-partition formula with raw empirical moments (each sample weight 1/m)
    # is an independent route to the same numbers, for complex multivariate data
    cols = _complex_samples(np.random.default_rng(20 + m), m)
    support = np.stack(cols, axis=1)
    probs = np.full(m, 1.0 / m)
    for fn, c in ((oracle.c2_natural, (0, 1)), (oracle.c3_natural, (0, 1, 2)),
                  (oracle.c4_natural, (0, 1, 2, 3)), (oracle.c4_natural, (2, 0, 3, 0))):
        got = fn(*[cols[i] for i in c])
        assert np.isclose(got, joint_cumulant(c, support, probs), rtol=1e-10, atol=1e-12)


def test_natural_estimator_bias_by_enumeration(distribution):
    # with m draws, the expected empirical c2 is (m-1)/m kappa2: the bias the
    # paper's comparison shows (the k-statistic removes it)
    support, probs = distribution
    m = 4
    kappa = joint_cumulant((0, 1), support, probs)
    e = brute_expectation(oracle.c2_natural, (0, 1), support, probs, m)
    assert np.isclose(e, (m - 1) / m * kappa, rtol=1e-12, atol=1e-14)


def test_first_order_spectrum_of_a_constant_and_of_a_shift():
    # S1 is the window-weighted mean of the signal: c for a constant record, and a
    # constant added to any record adds itself
    T, m = 32, 4
    z = np.full(T * m * 5, 2.5)
    r = oracle.polyspectra(z, T, 0.1, m, orders=(1,))
    assert np.isclose(r["S1"], 2.5) and np.allclose(r["S1_err"], 0.0)
    y = np.random.default_rng(3).normal(size=T * m * 7)
    a = oracle.polyspectra(y, T, 0.1, m, orders=(1,), window_kind="acg")
    b = oracle.polyspectra(y + 0.75, T, 0.1, m, orders=(1,), window_kind="acg")
    assert np.isclose(b["S1"], a["S1"] + 0.75, rtol=0, atol=1e-12)
    # and the groups' plain weighted means give it directly
    g = oracle.window(T, "acg")
    fr = y[: (len(y) // (T * m)) * T * m].reshape(-1, m, T)
    want = np.mean(np.sum(fr * g, axis=-1) / np.sum(g))
    assert np.isclose(a["S1"].real, want, rtol=1e-12)
