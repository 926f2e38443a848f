"""Pins of the oracle's spectra of complex-valued signals (App. D) and of the
shifted S4 planes (App. E), against facts that do not come from that function:

* real channels (zero imaginary part) give the real cross-spectra of Eq. 47, 48,
  50 (the oracle's separate real path) on their half-plane domains, and the
  conjugate symmetry on the other half;
* the paper's multilinear decomposition (App. D): the spectra of z = x + j y are
  the sums of 4, 8 and 16 real cross-spectra with factors j^(number of
  imaginary parts), the real cross-spectra again from the real path;
* the sign convention for complex signals: a complex AR(1) process whose phase
  turns by +theta per sample has its power (the combination of z with its
  conjugate) at k = -theta T / (2 pi) under the positive exponent of Eq. 18 and
  App. A, and almost none at the mirrored bin;
* App. E: the plane with shift s equals the cut of the signals multiplied by
  e^{+-j dw t} in the time domain (dw = 2 pi s / T per sample), and s = 0 is the
  cut.
"""
import numpy as np
import pytest

import oracle
import synth

T, M_FR, DT = 16, 5, 0.5
M = T // 2 + 1


def complex_pair(n, seed):
    x = synth.ar1_quadratic(n, seed=seed, phi=0.7).astype(np.float64)
    y = synth.ar1_quadratic(n, seed=seed + 100, phi=0.4).astype(np.float64)
    return x, y


@pytest.fixture(scope="module")
def four_real():
    n = T * M_FR * 60 + 3
    x1, y1 = complex_pair(n, 1)
    x2, y2 = complex_pair(n, 2)
    return np.stack([x1, y1, x2, y2])


def test_real_channels_give_the_real_cross_spectra(four_real):
    zs = four_real[:2]
    c2, c3, c4 = [(0, 1)], [(0, 1, 1)], [(1, 0, 0, 1)]
    real = oracle.cross_polyspectra(zs, T, DT, M_FR, s2_combos=c2, s3_combos=c3, s4_combos=c4)
    ops = lambda cmb: tuple((c, False) for c in cmb)          # noqa: E731
    cplx = oracle.complex_polyspectra(zs.astype(np.complex128), T, DT, M_FR,
                                      s2_combos=[ops(c) for c in c2],
                                      s3_combos=[ops(c) for c in c3],
                                      s4_combos=[ops(c) for c in c4])
    S2r, E2r = real[("S2", c2[0])]
    S2c, E2c = cplx[("S2", ops(c2[0]))]
    assert np.allclose(S2c[M - 1:], S2r, rtol=1e-10, atol=1e-14)
    assert np.allclose(S2c[:M - 1], np.conj(S2r[1:][::-1]), rtol=1e-10, atol=1e-14)
    assert np.allclose(E2c[M - 1:], E2r, rtol=1e-9, atol=1e-14)
    S3r, _ = real[("S3", c3[0])]
    S3c, _ = cplx[("S3", ops(c3[0]))]
    assert np.allclose(S3c[:, M - 1:], S3r, rtol=1e-10, atol=1e-14)        # l >= 0
    # S3(-k, -l) = S3(k, l)* for real channels
    assert np.allclose(S3c[::-1, ::-1], np.conj(S3c), rtol=1e-10, atol=1e-14)
    S4r, _ = real[("S4", c4[0])]
    S4c, _ = cplx[("S4", ops(c4[0]))]
    assert np.allclose(S4c[:, M - 1:], S4r, rtol=1e-10, atol=1e-14)
    assert np.allclose(S4c[::-1, ::-1], np.conj(S4c), rtol=1e-10, atol=1e-14)


def test_multilinear_decomposition_of_app_d(four_real):
    # z1 = x1 + j y1 (channels 0, 1), z2 = x2 + j y2 (channels 2, 3)
    x1, y1, x2, y2 = four_real
    z = np.stack([x1 + 1j * y1, x2 + 1j * y2])
    parts = {0: (0, 1), 1: (2, 3)}   # complex channel -> (real, imaginary) channel

    def expand(cmb):
        """[(real combination, coefficient)] of a combination of complex channels."""
        terms = [((), 1.0 + 0j)]
        for c in cmb:
            re, im = parts[c]
            terms = [(t + (re,), f) for t, f in terms] + [(t + (im,), f * 1j) for t, f in terms]
        return terms

    c2, c3, c4 = (0, 1), (0, 1, 1), (1, 0, 1, 0)
    terms = {2: expand(c2), 3: expand(c3), 4: expand(c4)}
    assert [len(terms[n]) for n in (2, 3, 4)] == [4, 8, 16]
    real = oracle.cross_polyspectra(four_real, T, DT, M_FR,
                                    s2_combos=[t for t, _ in terms[2]],
                                    s3_combos=[t for t, _ in terms[3]],
                                    s4_combos=[t for t, _ in terms[4]])
    ops = lambda cmb: tuple((c, False) for c in cmb)          # noqa: E731
    cplx = oracle.complex_polyspectra(z, T, DT, M_FR, s2_combos=[ops(c2)], s3_combos=[ops(c3)],
                                      s4_combos=[ops(c4)])
    for n, cmb, cols in ((2, c2, None), (3, c3, slice(M - 1, None)), (4, c4, slice(M - 1, None))):
        key = f"S{n}"
        total = sum(f * real[(key, t)][0] for t, f in terms[n])
        got = cplx[(key, ops(cmb))][0]
        got = got[M - 1:] if n == 2 else got[:, cols]
        assert np.allclose(got, total, rtol=1e-10, atol=1e-12), key


def test_complex_ar1_power_sits_at_minus_theta():
    T2, m, n = 64, 6, 64 * 6 * 80
    theta = 2 * np.pi * 10 / T2                       # +10 bins of phase per frame length
    phi = 0.95 * np.exp(1j * theta)
    e = synth.normal(n, seed=5) + 1j * synth.normal(n, seed=6)
    z = np.empty(n, np.complex128)
    z[0] = e[0]
    for t in range(1, n):
        z[t] = phi * z[t - 1] + e[t]
    out = oracle.complex_polyspectra(z[None, :], T2, 1.0, m,
                                     s2_combos=[((0, False), (0, True))])
    S = out[("S2", ((0, False), (0, True)))][0].real   # power: z with its conjugate
    M2 = T2 // 2 + 1
    peak = int(np.argmax(S)) - (M2 - 1)
    assert peak == -10
    assert S[M2 - 1 + 10] < 0.01 * S.max()             # the mirrored bin


@pytest.mark.parametrize("s", [1, 3, -2])
def test_shifted_plane_equals_modulated_signals(four_real, s):
    x1, y1, x2, y2 = four_real
    z = np.stack([x1 + 1j * y1, x2 + 1j * y2, x2 - 0.5j * x1, y2 + 1j * x1])
    t = np.arange(z.shape[1])
    rot = np.exp(2j * np.pi * s * t / T)
    shifted = np.stack([z[0] * rot, z[1] / rot, z[2] / rot, z[3] * rot])
    ops = ((0, False), (1, False), (2, False), (3, False))
    cut = oracle.complex_polyspectra(shifted, T, DT, M_FR, s4_combos=[ops])
    plane = oracle.complex_polyspectra(z, T, DT, M_FR, s4_combos=[ops], s4_shift=s)
    assert np.allclose(plane[("S4", ops)][0], cut[("S4", ops)][0], rtol=1e-9, atol=1e-13)
    assert np.allclose(plane[("S4", ops)][1], cut[("S4", ops)][1], rtol=1e-7, atol=1e-13)
    zero = oracle.complex_polyspectra(z, T, DT, M_FR, s4_combos=[ops], s4_shift=0)
    assert not np.allclose(zero[("S4", ops)][0], plane[("S4", ops)][0])
