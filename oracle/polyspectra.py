"""FP64 CPU oracle of the unbiased polyspectrum estimator (arXiv 2505.01231).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA path never
calls it, and it shares no code with the CUDA path (only the seeded signal
generators in ``synth`` feed both).

Every step follows the paper literally, in float64, with no blocking, fusion or
reordering beyond what the cited formula states:

* frames and window ........ Sec. 3, Eq. 16-17 (z_i, g_i); App. B, Eq. 71 (confined Gaussian)
* Fourier coefficients ..... Sec. 3, Eq. 18 (a_k with the POSITIVE exponent e^{+2 pi j ik/N},
                              t0 = 0); App. A, Eq. 63 (sign convention)
* cumulant estimators ...... Sec. 4.1, Eq. 32 (c2), Eq. 33 (c3), Eq. 34 (c4, raw-moment form);
                              App. H, Eq. 85 (factorised c4)
* spectra + normalisation .. Sec. 3, Eq. 23 (S2); Sec. 4, Eq. 28 (S3), Eq. 31 (S4 cut);
                              Sec. 7, Eq. 47, 48, 50 (multi-channel S2, S3, S4 cut)
* error bars ............... Sec. 4.2, Eq. 35-36 (variance over N_p parts, standard error)
* first-order spectrum ..... Sec. 4, S1 = N C1(a_0) / (T sum g); App. G
* interlaced spectra ....... Sec. 3: the same estimate from windows shifted by T/2, pooled with
                              the unshifted one (the groups of both window sets are the parts)
* complex-valued signals ... App. D: the spectra of complex channels from the cumulants of
                              their own Fourier coefficients at +k and -k (the multilinear
                              extension of Eq. 47, 48, 50); App. E: planes of the 3-D
                              trispectrum parallel to the cut, by a shift of s bins
* sequential spectra ....... Sec. 8 (quasi-polyspectra): the short-time estimates, each from m
                              windows, averaged over blocks of consecutive groups
* natural (biased) estimators, for the paper's unbiased-vs-biased comparison
                              (Sec. 4.1, Fig. 6): the cumulants of the m samples'
                              own empirical distribution, from their central moments

Notation: ``T`` is the number of samples per frame (the paper's N), ``dt`` the
sample interval (the paper's T/N), ``M = T/2 + 1`` the number of real-FFT bins,
``m`` the number of frames per k-statistic sample set ("group") and ``G`` the
number of groups; the paper's parts N_p are the groups.

With a_k = dt * X_k (X the plain windowed DFT sum), the paper's prefactor N/T
equals 1/dt, so Eq. 23, 28 and 31 become
    S2 = dt   c2(X_k, X_k*)                 / sum g^2
    S3 = dt^2 c3(X_k, X_l, X_{k+l}*)        / sum g^3
    S4 = dt^3 c4(X_k, X_k*, X_l, X_l*)      / sum g^4.
For real channels X_{-k} = X_k* (the DFT of a real frame).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "window",
    "dft_plus",
    "dft_plus_direct",
    "frame_groups",
    "fourier_coefficients",
    "c2",
    "c3",
    "c4",
    "c4_factorised",
    "c2_natural",
    "c3_natural",
    "c4_natural",
    "coef",
    "s2_groups",
    "s3_groups",
    "s4_groups",
    "s1_groups",
    "mean_and_stderr",
    "s3_domain",
    "polyspectra",
    "cross_domain_s3",
    "cross_polyspectra",
    "sequential_spectra",
    "dft_plus_complex",
    "complex_polyspectra",
]


# --------------------------------------------------------------------------- window
def window(T: int, kind: str = "hann", sigma_t: float = 0.14) -> np.ndarray:
    """Window coefficients g_i, i = 0..T-1 (float64).

    ``hann``: periodic Hann, g_i = 0.5 - 0.5 cos(2 pi i / T).
    ``acg``: approximate confined Gaussian of App. B, Eq. 71,
        g_k ~ G(k) - G(-1/2) [G(k+N) + G(k-N)] / [G(-1/2+N) + G(-1/2-N)],
        G(x) = exp(-(x - (N-1)/2)^2 / (4 N^2 sigma_t^2)), N = T.
    The estimator is invariant under g -> c g, so no normalisation is applied.
    """
    i = np.arange(T, dtype=np.float64)
    if kind == "hann":
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * i / T)
    if kind == "acg":
        N = float(T)

        def G(x):
            return np.exp(-((x - (N - 1.0) / 2.0) ** 2) / (4.0 * N * N * sigma_t * sigma_t))

        return G(i) - G(-0.5) * (G(i + N) + G(i - N)) / (G(-0.5 + N) + G(-0.5 - N))
    raise ValueError(f"unknown window {kind!r}")


# --------------------------------------------------------------------------- DFT
def dft_plus(x: np.ndarray) -> np.ndarray:
    """X_k = sum_i x_i exp(+2 pi j i k / T), k = 0..T/2, over the last axis.

    Eq. 18 with t0 = 0 and without the dt prefactor.  For real x this is the
    complex conjugate of numpy's forward real FFT (which uses exp(-2 pi j ik/T)),
    so the library FFT serves as the summation step.
    """
    return np.conj(np.fft.rfft(np.asarray(x, dtype=np.float64), axis=-1))


def dft_plus_direct(x: np.ndarray) -> np.ndarray:
    """The same sum as ``dft_plus`` evaluated term by term, O(T^2) (pinning only)."""
    x = np.asarray(x, dtype=np.float64)
    T = x.shape[-1]
    k = np.arange(T // 2 + 1)
    i = np.arange(T)
    w = np.exp(2j * np.pi * np.outer(i, k) / T)
    return x @ w


# --------------------------------------------------------------------------- framing
def frame_groups(z: np.ndarray, T: int, m: int) -> np.ndarray:
    """Cut a channel into consecutive frames z_i = z[jT + i] (Eq. 16) and group m frames.

    Returns float64 [G, m, T]; trailing samples that do not fill a whole group
    are dropped.
    """
    z = np.asarray(z)
    G = z.shape[-1] // (m * T)
    return z[..., : G * m * T].astype(np.float64).reshape(z.shape[:-1] + (G, m, T))


def fourier_coefficients(z: np.ndarray, T: int, m: int, g: np.ndarray) -> np.ndarray:
    """X[g, j, k] = sum_i g_i z_{(g m + j) T + i} e^{+2 pi j ik/T}: complex128 [G, m, M]."""
    return dft_plus(frame_groups(z, T, m) * g)


# --------------------------------------------------------------------------- k-statistics
def _mean(v):
    return v.mean(axis=-1)


def c2(x, y):
    """Eq. 32: m/(m-1) (mean(xy) - mean(x) mean(y)); samples on the last axis."""
    m = x.shape[-1]
    return m / (m - 1) * (_mean(x * y) - _mean(x) * _mean(y))


def c3(x, y, z):
    """Eq. 33: m^2/((m-1)(m-2)) (xyz - xy z - xz y - yz x + 2 x y z), bars = sample means."""
    m = x.shape[-1]
    mx, my, mz = _mean(x), _mean(y), _mean(z)
    return m * m / ((m - 1) * (m - 2)) * (
        _mean(x * y * z)
        - _mean(x * y) * mz
        - _mean(x * z) * my
        - _mean(y * z) * mx
        + 2.0 * mx * my * mz
    )


def c4(x, y, z, w):
    """Eq. 34, the raw-moment form of the fourth k-statistic."""
    m = x.shape[-1]
    mx, my, mz, mw = _mean(x), _mean(y), _mean(z), _mean(w)
    xy, xz, xw = _mean(x * y), _mean(x * z), _mean(x * w)
    yz, yw, zw = _mean(y * z), _mean(y * w), _mean(z * w)
    xyz, xyw = _mean(x * y * z), _mean(x * y * w)
    xzw, yzw = _mean(x * z * w), _mean(y * z * w)
    xyzw = _mean(x * y * z * w)
    bracket = (
        (m + 1) * xyzw
        - (m + 1) * (xyz * mw + xyw * mz + xzw * my + yzw * mx)
        - (m - 1) * (xy * zw + xz * yw + xw * yz)
        + 2 * m * (xy * mz * mw + xz * my * mw + xw * my * mz
                   + yz * mx * mw + yw * mx * mz + zw * mx * my)
        - 6 * m * mx * my * mz * mw
    )
    return m * m / ((m - 1) * (m - 2) * (m - 3)) * bracket


def c4_factorised(x, y, z, w):
    """App. H, Eq. 85: the same statistic written with centred samples."""
    m = x.shape[-1]
    dx = x - _mean(x)[..., None]
    dy = y - _mean(y)[..., None]
    dz = z - _mean(z)[..., None]
    dw = w - _mean(w)[..., None]
    bracket = (m + 1) * _mean(dx * dy * dz * dw) - (m - 1) * (
        _mean(dx * dy) * _mean(dz * dw)
        + _mean(dx * dz) * _mean(dy * dw)
        + _mean(dx * dw) * _mean(dy * dz)
    )
    return m * m / ((m - 1) * (m - 2) * (m - 3)) * bracket


# --------------------------------------------------------------------------- spectra
def _central(v):
    return v - _mean(v)[..., None]


def c2_natural(x, y):
    """Second cumulant of the samples' empirical distribution: the mean product of
    the centred samples (no m/(m-1) correction; biased)."""
    return _mean(_central(x) * _central(y))


def c3_natural(x, y, z):
    """Third cumulant of the empirical distribution: the mean triple product of the
    centred samples (biased)."""
    return _mean(_central(x) * _central(y) * _central(z))


def c4_natural(x, y, z, w):
    """Fourth cumulant of the empirical distribution: the fourth central moment
    minus the three pairings of second central moments (biased)."""
    dx, dy, dz, dw = _central(x), _central(y), _central(z), _central(w)
    return _mean(dx * dy * dz * dw) - (
        _mean(dx * dy) * _mean(dz * dw)
        + _mean(dx * dz) * _mean(dy * dw)
        + _mean(dx * dw) * _mean(dy * dz)
    )


_ESTIMATORS = {
    "unbiased": (None, None, None),
    "natural": (c2_natural, c3_natural, c4_natural),
}


def coef(X: np.ndarray, k) -> np.ndarray:
    """Coefficients at (possibly negative) bins k: X_{-k} = X_k* for a real channel.

    X: [..., m, M]; returns [..., m, len(k)].
    """
    k = np.asarray(k)
    v = X[..., np.abs(k)]
    return np.where(k < 0, np.conj(v), v)


def _samples_last(v):
    # [..., m, P] -> [..., P, m] so the k-statistics reduce over the last axis
    return np.swapaxes(v, -1, -2)


def s2_groups(Xa, Xb, dt, g, k=None, estimator="unbiased"):
    """Per-group S2 (Eq. 23 / Eq. 47): dt c2(a_k, b_k*) / sum g^2.  Returns [G, P]."""
    M = Xa.shape[-1]
    k = np.arange(M) if k is None else np.asarray(k)
    x = _samples_last(coef(Xa, k))
    y = _samples_last(np.conj(coef(Xb, k)))
    f = _ESTIMATORS[estimator][0] or c2
    return dt * f(x, y) / np.sum(g ** 2)


def s3_groups(Xa, Xb, Xc, dt, g, k, l, estimator="unbiased"):
    """Per-group S3 (Eq. 28 / Eq. 48): dt^2 c3(a_k, b_l, c_{k+l}*) / sum g^3."""
    k, l = np.asarray(k), np.asarray(l)
    x = _samples_last(coef(Xa, k))
    y = _samples_last(coef(Xb, l))
    z = _samples_last(np.conj(coef(Xc, k + l)))
    f = _ESTIMATORS[estimator][1] or c3
    return dt * dt * f(x, y, z) / np.sum(g ** 3)


def s4_groups(Xa, Xb, Xc, Xd, dt, g, k, l, factorised=False, estimator="unbiased"):
    """Per-group S4 cut (Eq. 31 / Eq. 50): dt^3 c4(a_k, b_k*, c_l, d_l*) / sum g^4."""
    k, l = np.asarray(k), np.asarray(l)
    x = _samples_last(coef(Xa, k))
    y = _samples_last(np.conj(coef(Xb, k)))
    z = _samples_last(coef(Xc, l))
    w = _samples_last(np.conj(coef(Xd, l)))
    f = _ESTIMATORS[estimator][2] or (c4_factorised if factorised else c4)
    return dt ** 3 * f(x, y, z, w) / np.sum(g ** 4)


def s1_groups(X, g):
    """Per-group first-order spectrum S1 = N C1(a_0) / (T sum g) = mean_j X_j0 / sum g
    (a_0 = dt X_0 and N/T = 1/dt); C1 is the plain mean, the same for both
    estimators.  Returns [G]."""
    return _mean(_samples_last(X[..., 0:1]))[..., 0] / np.sum(g)


def mean_and_stderr(Sg: np.ndarray):
    """Average over the N_p = G parts and standard error of Re and Im (Eq. 35-36).

    Var(x) = N_p/(N_p - 1) (mean(x^2) - mean(x)^2), sigma = sqrt(Var / N_p).
    Returns (mean complex, err_re, err_im), each with the part axis (0) removed.
    """
    Np = Sg.shape[0]

    def err(x):
        var = Np / (Np - 1) * (np.mean(x * x, axis=0) - np.mean(x, axis=0) ** 2)
        return np.sqrt(np.maximum(var, 0.0) / Np)

    return Sg.mean(axis=0), err(Sg.real), err(Sg.imag)


class _Acc:
    """Running sums over groups of S, Re(S)^2 and Im(S)^2 (float64)."""

    def __init__(self, shape):
        self.s = np.zeros(shape, np.complex128)
        self.qr = np.zeros(shape, np.float64)
        self.qi = np.zeros(shape, np.float64)
        self.n = 0

    def add(self, Sg):
        self.s += Sg.sum(axis=0)
        self.qr += (Sg.real ** 2).sum(axis=0)
        self.qi += (Sg.imag ** 2).sum(axis=0)
        self.n += Sg.shape[0]

    def result(self):
        Np = self.n
        mean = self.s / Np
        var_r = Np / (Np - 1) * (self.qr / Np - mean.real ** 2)
        var_i = Np / (Np - 1) * (self.qi / Np - mean.imag ** 2)
        return mean, np.sqrt(np.maximum(var_r, 0) / Np), np.sqrt(np.maximum(var_i, 0) / Np)


def s3_domain(M: int):
    """Single-channel bispectrum grid points: 0 <= k, l and k + l <= M - 1 (row-major)."""
    kk, ll = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    sel = (kk + ll) <= M - 1
    return kk[sel], ll[sel]


def polyspectra(z, T, dt, m, window_kind="hann", sigma_t=0.14, orders=(2, 3, 4),
                group_chunk=16, max_groups=None, factorised_c4=False, estimator="unbiased",
                interlaced=False):
    """Single-channel S1 (a number), S2 [M], S3 [M, M], S4 [M, M] with standard errors.

    Returns a dict with keys 'S2', 'S2_err', 'S3', 'S3_err', 'S4', 'S4_err', 'G'
    (and 'S1', 'S1_err' with order 1; '*_err' arrays carry a trailing axis
    (err_re, err_im)).  S3 is zero outside k + l <= M - 1.  ``max_groups`` limits
    the record to its first groups.  ``estimator``: "unbiased" (k-statistics,
    Eq. 32-34) or "natural" (cumulants of each group's empirical distribution).
    ``interlaced``: add the groups of the frames that start T/2 samples later.
    """
    g = window(T, window_kind, sigma_t)
    frames = frame_groups(z, T, m)
    if max_groups is not None:
        frames = frames[:max_groups]
    if interlaced:
        shifted = frame_groups(np.asarray(z)[T // 2:], T, m)
        if max_groups is not None:
            shifted = shifted[:max_groups]
        frames = np.concatenate([frames, shifted], axis=0)
    G = frames.shape[0]
    if G < 2:
        raise ValueError("need at least two groups for an error estimate")
    M = T // 2 + 1
    out = {"G": G}
    kk3, ll3 = s3_domain(M)
    kk4, ll4 = [a.ravel() for a in np.meshgrid(np.arange(M), np.arange(M), indexing="ij")]
    acc = {}
    if 1 in orders:
        acc[1] = _Acc(())
    if 2 in orders:
        acc[2] = _Acc((M,))
    if 3 in orders:
        acc[3] = _Acc((kk3.size,))
    if 4 in orders:
        acc[4] = _Acc((kk4.size,))
    for g0 in range(0, G, group_chunk):
        X = dft_plus(frames[g0:g0 + group_chunk] * g)
        if 1 in orders:
            acc[1].add(s1_groups(X, g))
        if 2 in orders:
            acc[2].add(s2_groups(X, X, dt, g, estimator=estimator))
        if 3 in orders:
            acc[3].add(s3_groups(X, X, X, dt, g, kk3, ll3, estimator=estimator))
        if 4 in orders:
            acc[4].add(s4_groups(X, X, X, X, dt, g, kk4, ll4, factorised=factorised_c4,
                                 estimator=estimator))
    if 1 in orders:
        mean, er, ei = acc[1].result()
        out["S1"], out["S1_err"] = mean, np.stack([er, ei], -1)
    if 2 in orders:
        mean, er, ei = acc[2].result()
        out["S2"], out["S2_err"] = mean, np.stack([er, ei], -1)
    if 3 in orders:
        mean, er, ei = acc[3].result()
        S3 = np.zeros((M, M), np.complex128)
        E3 = np.zeros((M, M, 2))
        S3[kk3, ll3] = mean
        E3[kk3, ll3, 0], E3[kk3, ll3, 1] = er, ei
        out["S3"], out["S3_err"] = S3, E3
    if 4 in orders:
        mean, er, ei = acc[4].result()
        out["S4"] = mean.reshape(M, M)
        out["S4_err"] = np.stack([er, ei], -1).reshape(M, M, 2)
    return out


# --------------------------------------------------------------------------- multi-channel
def cross_domain_s3(M: int):
    """Cross bispectrum grid: k in [-(M-1), M-1], l in [0, M-1], |k + l| <= M - 1.

    Returned as index arrays (k, l) in row-major order of the [2M-1, M] output,
    whose row r holds k = r - (M - 1).
    """
    kk, ll = np.meshgrid(np.arange(-(M - 1), M), np.arange(M), indexing="ij")
    sel = np.abs(kk + ll) <= M - 1
    return kk[sel], ll[sel]


def cross_polyspectra(zs, T, dt, m, s2_combos=(), s3_combos=(), s4_combos=(),
                      window_kind="hann", sigma_t=0.14, group_chunk=8, max_groups=None,
                      estimator="unbiased"):
    """Multi-channel spectra (Sec. 7, Eq. 47, 48, 50) for the listed channel combinations.

    zs: [C, n] real channels.  s2_combos: (a, b) pairs -> S2_ab [M] = C2(a_k, b_k*).
    s3_combos: (a, b, c) -> S3_abc [2M-1, M] = C3(a_k, b_l, c_{k+l}*) on the cross
    domain of ``cross_domain_s3`` (zero elsewhere).  s4_combos: (a, b, c, d) ->
    S4_abcd [2M-1, M] = C4(a_k, b_k*, c_l, d_l*), k in [-(M-1), M-1], l in [0, M-1].
    Returns a dict keyed by ('S2', combo) etc. holding (mean, err[..., 2]), plus 'G'.
    """
    g = window(T, window_kind, sigma_t)
    frames = frame_groups(np.asarray(zs), T, m)  # [C, G, m, T]
    if max_groups is not None:
        frames = frames[:, :max_groups]
    C, G = frames.shape[0], frames.shape[1]
    M = T // 2 + 1
    kk3, ll3 = cross_domain_s3(M)
    kk4, ll4 = [a.ravel() for a in
                np.meshgrid(np.arange(-(M - 1), M), np.arange(M), indexing="ij")]
    accs = {}
    for cmb in s2_combos:
        accs[("S2", tuple(cmb))] = _Acc((M,))
    for cmb in s3_combos:
        accs[("S3", tuple(cmb))] = _Acc((kk3.size,))
    for cmb in s4_combos:
        accs[("S4", tuple(cmb))] = _Acc((kk4.size,))
    for g0 in range(0, G, group_chunk):
        X = [dft_plus(frames[c, g0:g0 + group_chunk] * g) for c in range(C)]
        for cmb in s2_combos:
            a, b = cmb
            accs[("S2", tuple(cmb))].add(s2_groups(X[a], X[b], dt, g, estimator=estimator))
        for cmb in s3_combos:
            a, b, c = cmb
            accs[("S3", tuple(cmb))].add(s3_groups(X[a], X[b], X[c], dt, g, kk3, ll3,
                                                   estimator=estimator))
        for cmb in s4_combos:
            a, b, c, d = cmb
            accs[("S4", tuple(cmb))].add(s4_groups(X[a], X[b], X[c], X[d], dt, g, kk4, ll4,
                                                   estimator=estimator))
    out = {"G": G}
    for key, acc in accs.items():
        mean, er, ei = acc.result()
        if key[0] == "S2":
            out[key] = (mean, np.stack([er, ei], -1))
        elif key[0] == "S3":
            S = np.zeros((2 * M - 1, M), np.complex128)
            E = np.zeros((2 * M - 1, M, 2))
            S[kk3 + M - 1, ll3] = mean
            E[kk3 + M - 1, ll3, 0], E[kk3 + M - 1, ll3, 1] = er, ei
            out[key] = (S, E)
        else:
            out[key] = (mean.reshape(2 * M - 1, M),
                        np.stack([er, ei], -1).reshape(2 * M - 1, M, 2))
    return out


# --------------------------------------------------------------------------- sequential spectra
def sequential_spectra(z, T, dt, m, block_groups, window_kind="hann", sigma_t=0.14,
                       orders=(2, 3, 4), estimator="unbiased"):
    """Sequential (short-time) spectra of a single channel (Sec. 8).

    Each group of m consecutive frames gives one short-time estimate S_g (the
    estimate whose average over all groups is the spectrum, and which for a
    non-stationary signal is a quasi-polyspectrum of that stretch).  The groups
    are taken ``block_groups`` at a time, consecutively from the first one; block
    b is the average of the S_g of groups b*B .. (b+1)*B - 1 with the standard
    error over those groups (Eq. 35-36 with the block's groups as the parts),
    i.e. exactly the estimate of that stretch of the record.  Groups after the
    last whole block form no block.  Returns a dict with 'blocks' and, per
    order, 'S2' [blocks, M], 'S3'/'S4' [blocks, M, M] and the '*_err' arrays
    with a trailing (err_re, err_im) axis.
    """
    if block_groups < 2:
        raise ValueError("a block needs at least two groups for its error estimate")
    z = np.asarray(z)
    span = block_groups * m * T
    nb = (z.shape[-1] // (m * T)) // block_groups
    out = {"blocks": nb}
    parts = [polyspectra(z[b * span:(b + 1) * span], T, dt, m, window_kind, sigma_t, orders,
                         group_chunk=max(1, block_groups), estimator=estimator)
             for b in range(nb)]
    for n in orders:
        if n < 2:
            continue
        key = f"S{n}"
        out[key] = np.stack([q[key] for q in parts]) if nb else None
        out[key + "_err"] = np.stack([q[key + "_err"] for q in parts]) if nb else None
    return out


# --------------------------------------------------------------------------- complex signals
def dft_plus_complex(x: np.ndarray) -> np.ndarray:
    """X_k = sum_i x_i exp(+2 pi j i k / T) of complex frames, all T bins k = 0..T-1
    over the last axis (bin T - k is the negative frequency -k).  numpy's inverse
    FFT uses the same exponent and a factor 1/T, so it serves as the summation
    step."""
    x = np.asarray(x, dtype=np.complex128)
    return np.fft.ifft(x, axis=-1) * x.shape[-1]


def _coef_full(X, k, conj):
    """Coefficient at (signed) bin k of a channel, or of its complex conjugate
    (the transform of z* at k is the conjugate of z's at -k); bins wrap mod T."""
    T = X.shape[-1]
    if conj:
        return np.conj(X[..., (-np.asarray(k)) % T])
    return X[..., np.asarray(k) % T]


def complex_polyspectra(zs, T, dt, m, s2_combos=(), s3_combos=(), s4_combos=(), s4_shift=0,
                        window_kind="hann", sigma_t=0.14, group_chunk=8):
    """Spectra of complex-valued channels (App. D) and shifted S4 planes (App. E).

    zs: [C, n] complex channels.  A combination lists its operands as (channel,
    conjugate) pairs; operand (c, True) is the conjugate signal z_c*.  With A, B,
    C, D the Fourier coefficients of the operands (all T bins, Eq. 18 with the
    positive exponent) and the window sums of Eq. 23, 28, 31:
      S2(k)    = dt   c2(A(k), B(-k))                       / sum g^2
      S3(k, l) = dt^2 c3(A(k), B(l), C(-k-l))                / sum g^3
      S4(k, l) = dt^3 c4(A(k+s), B(-k-s), C(l-s), D(-l+s))   / sum g^4
    for k, l in [-(M-1), M-1] (M = T/2 + 1; S3 where also |k + l| <= M-1, zero
    elsewhere), bins taken mod T.  For real channels A(-k) = A(k)*, so these are
    the spectra of Eq. 47, 48, 50 on the whole plane.  s = s4_shift: the plane
    of the 3-D trispectrum through (k + s, -k - s, l - s, -l + s), the S4 of the
    shifted signals z1 e^{+j dw t}, z2 e^{-j dw t}, z3 e^{-j dw t}, z4 e^{+j dw t}
    with dw = 2 pi s / (T dt) (frames start at multiples of T samples, where
    e^{j dw t} = 1).  Returns {(order key, combo): (mean, err[..., 2])} and 'G';
    the arrays are [2M-1] (S2) or [2M-1, 2M-1] (S3, S4), row r holding k = r-(M-1)
    and column c holding l = c-(M-1).
    """
    g = window(T, window_kind, sigma_t)
    zs = np.asarray(zs)
    G = zs.shape[-1] // (m * T)
    frames = zs[:, : G * m * T].astype(np.complex128).reshape(zs.shape[0], G, m, T)
    M = T // 2 + 1
    ks = np.arange(-(M - 1), M)
    kk, ll = [a.ravel() for a in np.meshgrid(ks, ks, indexing="ij")]
    in3 = np.abs(kk + ll) <= M - 1
    s = int(s4_shift)
    accs = {}
    for cmb in s2_combos:
        accs[("S2", tuple(cmb))] = _Acc((ks.size,))
    for cmb in s3_combos:
        accs[("S3", tuple(cmb))] = _Acc((int(in3.sum()),))
    for cmb in s4_combos:
        accs[("S4", tuple(cmb))] = _Acc((kk.size,))
    k3, l3 = kk[in3], ll[in3]
    for g0 in range(0, G, group_chunk):
        X = [dft_plus_complex(frames[c, g0:g0 + group_chunk] * g) for c in range(zs.shape[0])]

        def op(o, k):
            c, cj = o
            return _samples_last(_coef_full(X[c], k, cj))

        for cmb in s2_combos:
            a, b = cmb
            v = c2(op(a, ks), op(b, -ks))
            accs[("S2", tuple(cmb))].add(dt * v / np.sum(g ** 2))
        for cmb in s3_combos:
            a, b, c = cmb
            v = c3(op(a, k3), op(b, l3), op(c, -k3 - l3))
            accs[("S3", tuple(cmb))].add(dt * dt * v / np.sum(g ** 3))
        for cmb in s4_combos:
            a, b, c, d = cmb
            v = c4(op(a, kk + s), op(b, -kk - s), op(c, ll - s), op(d, -ll + s))
            accs[("S4", tuple(cmb))].add(dt ** 3 * v / np.sum(g ** 4))
    out = {"G": G}
    n = 2 * M - 1
    for key, acc in accs.items():
        mean, er, ei = acc.result()
        if key[0] == "S2":
            out[key] = (mean, np.stack([er, ei], -1))
        elif key[0] == "S3":
            S = np.zeros((n, n), np.complex128)
            E = np.zeros((n, n, 2))
            S[k3 + M - 1, l3 + M - 1] = mean
            E[k3 + M - 1, l3 + M - 1, 0], E[k3 + M - 1, l3 + M - 1, 1] = er, ei
            out[key] = (S, E)
        else:
            out[key] = (mean.reshape(n, n), np.stack([er, ei], -1).reshape(n, n, 2))
    return out
