"""Seeded synthetic signal generators shared by the tests, the bench and the oracle.

This module only produces input samples.  It contains none of the estimator's
arithmetic (no windowing, no Fourier transform, no cumulant estimators), so
both the CUDA path and the FP64 oracle can read identical bytes from it.

Random numbers come from a counter-based generator written from its published
definition: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; finaliser constants as published there),
turned into uniforms on (0, 1) with 53 random bits and into Gaussians with the
Box-Muller transform (Box & Muller, Ann. Math. Stat. 1958).  Being counter
based, sample ``i`` of stream ``seed`` is the same on every machine and does
not depend on how the stream is cut into pieces.

Workload shapes follow the synthetic signals the paper analyses (stochastic
oscillators, telegraph noise, filtered Gaussian noise; Sec. 4, Sec. 6.1) in the
concrete forms below:

* ``ar1_quadratic``: x_t = y_t + c (y_t^2 - 1), y an AR(1) process with
  unit-variance Gaussian innovations started from its stationary law.
* ``multichannel_shared``: c_k = g + n_k + 0.2 g^2 + s_k with a shared AR(1)
  Gaussian g, independent white Gaussian n_k and random telegraph s_k.
* ``adc_telegraph_int16``: int16 samples of a low-passed telegraph signal plus
  Gaussian noise (an ADC record).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64",
    "uniform",
    "normal",
    "exponential_centred",
    "ar1",
    "ar1_quadratic",
    "telegraph",
    "multichannel_shared",
    "adc_telegraph_int16",
    "adc_telegraph_int16_parallel",
    "iid_frames_ar1",
    "uneven_recordings",
]

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _stream_key(seed: int, stream: int) -> np.uint64:
    # distinct streams for one seed: hash (seed, stream) through one SplitMix64 step
    x = np.array([(seed * 0x100000001B3 + stream * 0xC2B2AE3D27D4EB4F) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return splitmix64(x)[0]


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for the given 64-bit states (vectorised, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = (counter.astype(np.uint64) + _GOLDEN) & _MASK
        z = ((z ^ (z >> np.uint64(30))) * _M1) & _MASK
        z = ((z ^ (z >> np.uint64(27))) * _M2) & _MASK
        return z ^ (z >> np.uint64(31))


def _raw(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = (np.arange(start, start + n, dtype=np.uint64) * _GOLDEN + key) & _MASK
    return splitmix64(ctr)


def uniform(n: int, seed: int, stream: int = 0, start: int = 0) -> np.ndarray:
    """n uniforms on the open interval (0, 1), float64, 53 random bits each."""
    r = _raw(seed, stream, start, n)
    return ((r >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(n: int, seed: int, stream: int = 0, start: int = 0) -> np.ndarray:
    """n standard Gaussians (float64), elements [start, start+n) of the stream.

    Box-Muller: pair p uses uniforms 2p and 2p+1 and yields elements 2p (cos
    branch) and 2p+1 (sin branch).
    """
    p0, p1 = start // 2, (start + n - 1) // 2 + 1
    u = uniform(2 * (p1 - p0), seed, stream, 2 * p0)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    out = np.empty(2 * (p1 - p0), dtype=np.float64)
    out[0::2] = r * np.cos(2.0 * np.pi * u[1::2])
    out[1::2] = r * np.sin(2.0 * np.pi * u[1::2])
    off = start - 2 * p0
    return out[off:off + n]


def exponential_centred(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """Unit exponential minus its mean: cumulants k2=1, k3=2, k4=6."""
    return -np.log(uniform(n, seed, stream)) - 1.0


def ar1(n: int, phi: float, seed: int, stream: int = 0, sigma_e: float = 1.0) -> np.ndarray:
    """AR(1) y_t = phi y_{t-1} + e_t, e ~ N(0, sigma_e^2), stationary start (float64)."""
    from scipy.signal import lfilter

    e = sigma_e * normal(n, seed, stream)
    e[0] /= np.sqrt(1.0 - phi * phi)  # y_0 ~ N(0, sigma_e^2 / (1 - phi^2))
    return lfilter([1.0], [1.0, -phi], e)


def ar1_quadratic(n: int, seed: int, phi: float = 0.9, c: float = 0.3,
                  dtype=np.float32) -> np.ndarray:
    """x = y + c (y^2 - 1) with y an AR(1) process (unit innovations), cast to dtype."""
    y = ar1(n, phi, seed)
    return (y + c * (y * y - 1.0)).astype(dtype)


def telegraph(n: int, p: float, seed: int, stream: int = 0) -> np.ndarray:
    """Random telegraph signal with values +-1; each sample flips with probability p."""
    flips = uniform(n, seed, stream) < p
    s0 = 1.0 if uniform(1, seed, stream + 7919)[0] < 0.5 else -1.0
    parity = np.cumsum(flips, dtype=np.int64) & 1
    return s0 * (1.0 - 2.0 * parity.astype(np.float64))


def multichannel_shared(channels: int, n: int, seed: int, phi: float = 0.95,
                        sigma_n: float = 0.5, p_switch: float = 1e-3, quad: float = 0.2,
                        dtype=np.float32) -> np.ndarray:
    """[channels][n] array: c_k = g + n_k + quad g^2 + s_k, g shared AR(1)."""
    g = ar1(n, phi, seed, stream=0)
    out = np.empty((channels, n), dtype=dtype)
    for k in range(channels):
        nk = sigma_n * normal(n, seed, stream=1 + k)
        sk = telegraph(n, p_switch, seed, stream=101 + k)
        out[k] = (g + nk + quad * g * g + sk).astype(dtype)
    return out


def adc_telegraph_int16(n: int, seed: int, start: int = 0, state=None, p: float = 1e-4,
                        gain: float = 2000.0, sigma: float = 800.0, cutoff: float = 0.05):
    """int16 ADC record: rint(gain * LP4(telegraph) + N(0, sigma^2)), saturated to int16.

    LP4 is a 4th-order Butterworth low-pass at ``cutoff`` x sampling rate (bilinear
    design).  The record is produced piecewise: the first call passes ``start=0,
    state=None``; each later call passes the previous call's returned ``state`` and
    ``start`` advanced by the samples already produced.  Returns (samples, state).
    """
    from scipy.signal import butter, lfilter, lfilter_zi

    b, a = butter(4, 2.0 * cutoff)
    flips = uniform(n, seed, 11, start) < p
    sign0 = 1.0 if state is None else state[1]
    s = sign0 * (1.0 - 2.0 * (np.cumsum(flips, dtype=np.int64) & 1).astype(np.float64))
    zi = lfilter_zi(b, a) * s[0] if state is None else state[0]
    y, zf = lfilter(b, a, s, zi=zi)
    v = np.rint(gain * y + sigma * normal(n, seed, 12, start))
    return np.clip(v, -32768, 32767).astype(np.int16), (zf, float(s[-1]))


def _adc_flips(n, seed, start, p):
    return np.flatnonzero(uniform(n, seed, 11, start) < p)


def _adc_noise(y, seed, start, gain, sigma):
    v = np.rint(gain * y + sigma * normal(len(y), seed, 12, start))
    return np.clip(v, -32768, 32767).astype(np.int16)


def adc_telegraph_int16_parallel(n: int, seed: int, p: float = 1e-4, gain: float = 2000.0,
                                 sigma: float = 800.0, cutoff: float = 0.05,
                                 piece: int = 1 << 24, processes: int = 8) -> np.ndarray:
    """The record ``adc_telegraph_int16(n, seed)`` returns, produced with a process
    pool: the telegraph's flip positions and the noise are drawn in parallel
    pieces (the generator is counter based), the low-pass filter runs over the
    pieces in order with its state carried across.  The pool uses the ``spawn``
    start method, so it may be created after CUDA has been initialised."""
    import multiprocessing as mp

    from scipy.signal import butter, lfilter, lfilter_zi

    starts = list(range(0, n, piece))
    lens = [min(piece, n - a) for a in starts]
    with mp.get_context("spawn").Pool(processes) as pool:
        flips = pool.starmap(_adc_flips, [(ln, seed, a, p) for a, ln in zip(starts, lens)])
        b, a_coef = butter(4, 2.0 * cutoff)
        out = np.empty(n, np.int16)
        sign, zi, pending = 1.0, None, []
        for a, ln, fl in zip(starts, lens, flips):
            cnt = np.zeros(ln, np.int64)
            cnt[fl] = 1
            s = sign * (1.0 - 2.0 * (np.cumsum(cnt) & 1).astype(np.float64))
            if zi is None:
                zi = lfilter_zi(b, a_coef) * s[0]
            y, zi = lfilter(b, a_coef, s, zi=zi)
            sign = float(s[-1])
            pending.append((a, pool.apply_async(_adc_noise, (y, seed, a, gain, sigma))))
        for a, r in pending:
            v = r.get()
            out[a:a + len(v)] = v
    return out


def iid_frames_ar1(n_frames: int, T: int, phi: float, seed: int,
                   dtype=np.float64) -> np.ndarray:
    """n_frames independent stationary AR(1) segments of T samples, concatenated."""
    from scipy.signal import lfilter

    e = normal(n_frames * T, seed, stream=3).reshape(n_frames, T)
    e[:, 0] /= np.sqrt(1.0 - phi * phi)
    return lfilter([1.0], [1.0, -phi], e, axis=1).reshape(-1).astype(dtype)


def uneven_recordings(count: int, seed: int, log2_min: int = 20, log2_max: int = 26,
                      frame_lengths=(128, 256, 512, 1024)):
    """Recipe for a batch of independent recordings of uneven length.

    Returns a list of dicts (length n, frame length T, AR coefficient phi, seed);
    the samples themselves come from ``ar1_quadratic(n, seed, phi)``.
    """
    u = uniform(3 * count, seed, stream=501).reshape(count, 3)
    out = []
    for r in range(count):
        n = int(round(2.0 ** (log2_min + (log2_max - log2_min) * u[r, 0])))
        T = int(frame_lengths[min(int(u[r, 1] * len(frame_lengths)), len(frame_lengths) - 1)])
        phi = 0.5 + (0.98 - 0.5) * u[r, 2]
        out.append({"n": n, "T": T, "phi": float(phi), "seed": int(seed * 1000 + r)})
    return out
