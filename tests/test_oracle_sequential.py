"""Pins of the oracle's sequential (short-time) spectra and of the quasi-polyspectra
of Sec. 8 against facts that do not come from the oracle itself:

* block structure: one block of all groups is the whole-record estimate; equal
  blocks average to it;
* a linear chirp: the power-weighted centre bin of each block's S2 follows the instantaneous
  frequency at the block's centre (f(t) = f0 + (f1 - f0) t / n);
* amplitude-modulated white noise x_t = a(t) e_t: each block's S2 is the
  block's mean of a^2 (times sigma^2 dt); and the quasi-trispectrum depends on m
  as Sec. 8 describes: near zero when a group spans a small part of the
  modulation period, and, when a group spans whole periods, the diagonal
  S4(k, k) / S2(k)^2 tends to 2 Var(a^2) / E[a^2]^2 x (sum g^2)^2 / sum g^4 (the
  fourth cumulant of a scale mixture of circular Gaussians, 2 Var(V), with
  E|X_k|^2 = sigma^2 sum g^2), while a stationary Gaussian record gives zero at
  every m.
"""
import numpy as np
import pytest

import oracle
import synth


def test_one_block_is_the_whole_record_and_blocks_average_to_it():
    T, m, B = 32, 6, 5
    z = synth.ar1_quadratic(T * m * B * 4 + 17, seed=8)
    full = oracle.polyspectra(z, T, 0.5, m)
    seq = oracle.sequential_spectra(z, T, 0.5, m, B)
    assert seq["blocks"] == 4
    for key in ("S2", "S3", "S4"):
        assert np.allclose(seq[key].mean(axis=0), full[key], rtol=1e-12, atol=1e-14)
    one = oracle.sequential_spectra(z, T, 0.5, m, full["G"])
    assert one["blocks"] == 1
    for key in ("S2", "S3", "S4"):
        assert np.allclose(one[key][0], full[key], rtol=1e-12, atol=1e-14)
        assert np.allclose(one[key + "_err"][0], full[key + "_err"], rtol=1e-10, atol=1e-14)


def test_chirp_centroid_follows_the_instantaneous_frequency():
    # each block sweeps a few bins; its power-weighted mean bin is the sweep's centre
    T, m, B = 256, 4, 4
    n = T * m * B * 24
    t = np.arange(n, dtype=np.float64)
    f0, f1 = 0.05, 0.40                        # cycles per sample
    phase = 2 * np.pi * (f0 * t + 0.5 * (f1 - f0) * t * t / n)
    z = np.cos(phase) + 0.05 * synth.normal(n, seed=4)
    seq = oracle.sequential_spectra(z, T, 1.0, m, B, orders=(2,))
    span = B * m * T
    k = np.arange(T // 2 + 1)
    for b in range(seq["blocks"]):
        fc = f0 + (f1 - f0) * (b + 0.5) * span / n
        p = seq["S2"][b].real
        centroid = np.sum(k * p) / np.sum(p)
        assert abs(centroid - fc * T) <= 0.5, (b, centroid, fc * T)


def am_noise(n, period, depth, seed):
    t = np.arange(n, dtype=np.float64)
    a = 1.0 + depth * np.sin(2 * np.pi * t / period)
    return a, a * synth.normal(n, seed=seed)


def test_am_noise_block_power_follows_the_modulation():
    T, m, B, P = 64, 4, 8, 1 << 15
    n = P * 4
    a, z = am_noise(n, P, 0.8, seed=5)
    seq = oracle.sequential_spectra(z, T, 1.0, m, B, orders=(2,))
    span = B * m * T
    for b in range(seq["blocks"]):
        expect = np.mean(a[b * span:(b + 1) * span] ** 2)     # sigma = 1, dt = 1
        s2 = seq["S2"][b].real[1:-1]
        err = seq["S2_err"][b, 1:-1, 0]
        # the white spectrum is flat: its bin average against the block's mean of a^2
        assert abs(s2.mean() - expect) <= 5 * np.sqrt(np.sum(err ** 2)) / s2.size + 0.02 * expect


def _diag_ratio(z, T, m):
    r = oracle.polyspectra(z, T, 1.0, m, orders=(2, 4), group_chunk=64)
    M = T // 2 + 1
    d = np.arange(2, M - 2)
    s4, e4, s2 = r["S4"][d, d].real, r["S4_err"][d, d, 0], r["S2"][d].real
    zscore = np.mean(s4) / np.sqrt(np.mean(e4 ** 2) / d.size)
    return float(np.mean(s4 / s2 ** 2)), float(zscore)


def test_quasi_trispectrum_depends_on_m_for_am_noise_only():
    T, P, depth = 64, 1 << 14, 0.9
    n = 1 << 21
    _, z = am_noise(n, P, depth, seed=3)
    g = oracle.window(T)
    s = 0.5 * depth * depth
    ea2 = 1 + s                                            # E[a^2]
    ea4 = 1 + 6 * depth ** 2 * 0.5 + depth ** 4 * 0.375     # E[a^4]
    limit = 2 * (ea4 - ea2 ** 2) / ea2 ** 2 * np.sum(g ** 2) ** 2 / np.sum(g ** 4)
    small, zs = _diag_ratio(z, T, 4)          # a group spans 1/64 of a period
    whole, zw = _diag_ratio(z, T, 256)        # a group spans one period
    assert abs(zs) < 4
    assert zw > 50
    assert abs(whole - limit) <= 0.03 * limit
    # a stationary Gaussian record: zero at both m
    w = synth.normal(n, seed=9)
    for m in (4, 256):
        _, zz = _diag_ratio(w, T, m)
        assert abs(zz) < 4
