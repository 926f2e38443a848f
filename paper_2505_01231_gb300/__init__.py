"""Python binding of the GB300 polyspectrum library (libpolyspec.so, C ABI).

Argument marshalling only: every step of the estimator runs in the library's
CUDA kernels.  The functions mirror include/polyspec.h one to one
(``ss_plan``, ``ss_accumulate``, ``ss_finalize``, ...); ``Plan`` is a small
convenience wrapper over them.  Buffers may be torch tensors (CPU or CUDA),
numpy arrays or raw integer addresses.

Importing this module loads the compiled library and raises ImportError if it
is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "SS_OK", "SS_EINVAL", "SS_ENOMEM", "SS_ECUDA", "SS_ESTATE", "SS_ETIMEOUT", "SS_EUNSUPPORTED",
    "SS_WIN_HANN", "SS_WIN_ACG", "SS_ORDER2", "SS_ORDER3", "SS_ORDER4", "SS_F32", "SS_I16",
    "SS_PREC_FP32", "SS_PREC_TF32X3", "SS_PREC_BF16X3", "SS_PREC_BF16", "SS_PREC_FP16X3",
    "SSError", "ss_info", "ss_stats_t", "lib", "LIB_PATH",
    "ss_plan", "ss_accumulate", "ss_finalize", "ss_reset", "ss_query", "ss_combos",
    "ss_set_timing", "ss_stats", "ss_set_batch", "ss_destroy", "ss_last_error", "ss_version",
    "ss_s2_noalloc", "ss_layout", "ss_layout_warps", "Plan",
]

SS_OK, SS_EINVAL, SS_ENOMEM, SS_ECUDA, SS_ESTATE, SS_ETIMEOUT, SS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
SS_WIN_HANN, SS_WIN_ACG = 0, 1
SS_ORDER1, SS_ORDER2, SS_ORDER3, SS_ORDER4 = 1 << 1, 1 << 2, 1 << 3, 1 << 4
SS_EST_UNBIASED, SS_EST_NATURAL = 0, 1
SS_F32, SS_I16 = 0, 1
SS_PREC_FP32, SS_PREC_TF32X3, SS_PREC_BF16X3, SS_PREC_BF16, SS_PREC_FP16X3 = 0, 1, 2, 3, 4
SS_STATE_HEADER = 16

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpolyspec.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it first (python paper_2505_01231_gb300/build.py); "
        "this package has no CPU fallback")
lib = ctypes.CDLL(LIB_PATH)


class ss_info(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_int), ("T", ctypes.c_int), ("M", ctypes.c_int),
                ("m", ctypes.c_int), ("n_s2", ctypes.c_int), ("n_s3", ctypes.c_int),
                ("n_s4", ctypes.c_int), ("rows3", ctypes.c_int), ("rows4", ctypes.c_int),
                ("groups", ctypes.c_longlong), ("samples", ctypes.c_longlong),
                ("carried", ctypes.c_longlong), ("groups_per_batch", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("kernels_per_batch", ctypes.c_int)]


class ss_stats_t(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 5), ("launches", ctypes.c_longlong * 5),
                ("pairs3", ctypes.c_longlong), ("pairs4", ctypes.c_longlong)]


_P = ctypes.c_void_p
_sig = {
    "ss_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint,
                               ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P]),
    "ss_accumulate": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "ss_finalize": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "ss_reset": (ctypes.c_int, [_P]),
    "ss_query": (ctypes.c_int, [_P, ctypes.POINTER(ss_info)]),
    "ss_combos": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "ss_layout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                 ctypes.c_int, _P, _P, ctypes.c_int, _P, _P]),
    "ss_layout_warps": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int, _P, _P, ctypes.c_int,
                                       _P]),
    "ss_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "ss_stats": (ctypes.c_int, [_P, ctypes.POINTER(ss_stats_t)]),
    "ss_set_batch": (ctypes.c_int, [_P, ctypes.c_int]),
    "ss_destroy": (ctypes.c_int, [_P]),
    "ss_last_error": (ctypes.c_char_p, [_P]),
    "ss_version": (ctypes.c_char_p, []),
    "ss_s2_noalloc": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P]),
    "ss_noalloc_last_error": (ctypes.c_char_p, []),
    "ss_state_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "ss_finalize_s1": (ctypes.c_int, [_P, _P, _P]),
    "ss_set_estimator": (ctypes.c_int, [_P, ctypes.c_int]),
    "ss_set_interlace": (ctypes.c_int, [_P, ctypes.c_int]),
    "ss_inject_timeout": (ctypes.c_int, [_P, ctypes.c_int]),
    "ss_set_complex": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int]),
    "ss_complex_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "ss_finalize_complex": (ctypes.c_int, [_P, _P, _P]),
    "ss_set_sequential": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_longlong]),
    "ss_sequential_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t),
                                          ctypes.POINTER(ctypes.c_longlong)]),
    "ss_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "ss_get_tuning": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "ss_set_tuning": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "ss_export_state": (ctypes.c_int, [_P, _P]),
    "ss_merge_state": (ctypes.c_int, [_P, _P]),
    "ss_plan_many": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, _P, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint,
                                    ctypes.c_int, _P]),
    "ss_run_many": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ss_many_plan": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "ss_destroy_many": (ctypes.c_int, [_P]),
    "ss_many_last_error": (ctypes.c_char_p, [_P]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class SSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _addr(buf):
    """Raw address of a torch tensor, numpy array, int or None."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        return buf.ctypes.data
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _check(status, handle):
    if status != SS_OK:
        raise SSError(status, lib.ss_last_error(handle).decode())


def ss_plan(channels, T, dt, m, window=SS_WIN_HANN, win_param=0.14,
            orders=SS_ORDER2 | SS_ORDER3 | SS_ORDER4, dtype=SS_F32, precision=SS_PREC_FP32,
            combos=None, stream=None):
    """Create a plan; returns its handle (int).  ``combos``: list of 5-int records."""
    h = _P()
    arr = None
    if combos is not None:
        arr = (ctypes.c_int * (5 * len(combos)))(*[int(v) for rec in combos for v in rec])
    st = lib.ss_plan(ctypes.byref(h), channels, T, float(dt), m, window, float(win_param),
                     orders, dtype, precision, arr, 0 if combos is None else len(combos),
                     _addr(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream)
    _check(st, None)
    return h.value


def ss_accumulate(plan, chunk, n_samples):
    _check(lib.ss_accumulate(plan, _addr(chunk), n_samples), plan)


def ss_finalize(plan, S2=None, S3=None, S4=None, S2_err=None, S3_err=None, S4_err=None):
    _check(lib.ss_finalize(plan, _addr(S2), _addr(S3), _addr(S4), _addr(S2_err), _addr(S3_err),
                           _addr(S4_err)), plan)


def ss_finalize_s1(plan, S1=None, S1_err=None):
    _check(lib.ss_finalize_s1(plan, _addr(S1), _addr(S1_err)), plan)


def ss_set_estimator(plan, estimator):
    _check(lib.ss_set_estimator(plan, estimator), plan)


def ss_set_interlace(plan, on):
    _check(lib.ss_set_interlace(plan, int(on)), plan)


def ss_inject_timeout(plan, on):
    _check(lib.ss_inject_timeout(plan, int(bool(on))), plan)


def ss_set_sequential(plan, block_groups, out=None, max_blocks=0):
    _check(lib.ss_set_sequential(plan, int(block_groups), _addr(out), int(max_blocks)), plan)


def ss_sequential_info(plan):
    """(doubles per block, blocks completed since the last reset)"""
    n, b = ctypes.c_size_t(), ctypes.c_longlong()
    _check(lib.ss_sequential_info(plan, ctypes.byref(n), ctypes.byref(b)), plan)
    return n.value, b.value


def ss_set_complex(plan, records, s4_shift=0):
    """records: [(order, (re, im, conj), ...)] operands of complex-signal spectra."""
    flat = []
    for rec in records:
        order, ops = rec[0], list(rec[1:])
        ops += [(-1, -1, 0)] * (4 - len(ops))
        flat += [int(order)] + [int(v) for op in ops for v in op]
    arr = (ctypes.c_int * max(1, len(flat)))(*flat)
    _check(lib.ss_set_complex(plan, arr, len(records), int(s4_shift)), plan)


def ss_complex_size(plan):
    n = ctypes.c_size_t()
    _check(lib.ss_complex_size(plan, ctypes.byref(n)), plan)
    return n.value


def ss_finalize_complex(plan, S=None, S_err=None):
    _check(lib.ss_finalize_complex(plan, _addr(S), _addr(S_err)), plan)


def ss_autotune(plan):
    """Time every kernel form on this plan's shapes and keep the fastest; returns
    the best pass time in ms."""
    ms = ctypes.c_double()
    _check(lib.ss_autotune(plan, ctypes.byref(ms)), plan)
    return ms.value


def ss_get_tuning(plan):
    buf = ctypes.create_string_buffer(512)
    _check(lib.ss_get_tuning(plan, buf, 512), plan)
    return buf.value.decode()


def ss_set_tuning(plan, text):
    _check(lib.ss_set_tuning(plan, text.encode()), plan)


def ss_reset(plan):
    _check(lib.ss_reset(plan), plan)


def ss_query(plan):
    info = ss_info()
    _check(lib.ss_query(plan, ctypes.byref(info)), plan)
    return info


def ss_combos(plan):
    info = ss_query(plan)
    n = info.n_s2 + info.n_s3 + info.n_s4
    buf = (ctypes.c_int * (5 * max(n, 1)))()
    _check(lib.ss_combos(plan, buf, n), plan)
    return [tuple(buf[5 * i:5 * i + 5]) for i in range(n)]


def ss_layout(channels, T):
    """The work decomposition of a plan of this shape (host only): S3 tiles
    [(k0, l0)], S3 points left to the point kernel [(k, l)], tensor-core S4
    tiles [(k0, l0, columns)] and whether the column l = M - 1 is left to the
    column kernel."""
    n3, np_, n4, col = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.ss_layout(channels, T, None, 0, ctypes.byref(n3), None, 0, ctypes.byref(np_),
                         None, 0, ctypes.byref(n4), ctypes.byref(col)), None)
    t3 = (ctypes.c_int * (2 * max(n3.value, 1)))()
    pts = (ctypes.c_int * (2 * max(np_.value, 1)))()
    t4 = (ctypes.c_int * (3 * max(n4.value, 1)))()
    _check(lib.ss_layout(channels, T, t3, n3.value, ctypes.byref(n3), pts, np_.value,
                         ctypes.byref(np_), t4, n4.value, ctypes.byref(n4), ctypes.byref(col)),
           None)
    return ([(t3[2 * i], t3[2 * i + 1]) for i in range(n3.value)],
            [(pts[2 * i], pts[2 * i + 1]) for i in range(np_.value)],
            [(t4[3 * i], t4[3 * i + 1], t4[3 * i + 2]) for i in range(n4.value)],
            bool(col.value))


def ss_layout_warps(T):
    """The S3 decomposition of the independent-warp K2 form (one channel, host
    only): 32 x 32 sub-tiles [(k0, l0)] and the points left to the point kernel
    [(k, l)]."""
    n, np_ = ctypes.c_int(), ctypes.c_int()
    _check(lib.ss_layout_warps(T, None, 0, ctypes.byref(n), None, 0, ctypes.byref(np_)), None)
    t = (ctypes.c_int * (2 * max(n.value, 1)))()
    pts = (ctypes.c_int * (2 * max(np_.value, 1)))()
    _check(lib.ss_layout_warps(T, t, n.value, ctypes.byref(n), pts, np_.value,
                               ctypes.byref(np_)), None)
    return ([(t[2 * i], t[2 * i + 1]) for i in range(n.value)],
            [(pts[2 * i], pts[2 * i + 1]) for i in range(np_.value)])


def ss_set_timing(plan, enable):
    _check(lib.ss_set_timing(plan, int(bool(enable))), plan)


def ss_stats(plan):
    s = ss_stats_t()
    _check(lib.ss_stats(plan, ctypes.byref(s)), plan)
    return s


def ss_set_batch(plan, groups_per_batch):
    _check(lib.ss_set_batch(plan, groups_per_batch), plan)


def ss_destroy(plan):
    _check(lib.ss_destroy(plan), None)


def ss_last_error(plan=None):
    return lib.ss_last_error(plan).decode()


def ss_version():
    return lib.ss_version().decode()


def ss_state_size(plan):
    n = ctypes.c_size_t()
    _check(lib.ss_state_size(plan, ctypes.byref(n)), plan)
    return n.value


def ss_export_state(plan, dst):
    _check(lib.ss_export_state(plan, _addr(dst)), plan)


def ss_merge_state(plan, src):
    _check(lib.ss_merge_state(plan, _addr(src)), plan)


def _check_many(status, handle):
    if status != SS_OK:
        raise SSError(status, lib.ss_many_last_error(handle).decode())


def ss_plan_many(T_list, max_samples, dt, m, window=SS_WIN_HANN, win_param=0.14,
                 orders=SS_ORDER2 | SS_ORDER3 | SS_ORDER4, precision=SS_PREC_FP32, stream=None):
    """One-channel plans for many recordings; returns the handle (int)."""
    n = len(T_list)
    t = (ctypes.c_int * n)(*[int(v) for v in T_list])
    ms = (ctypes.c_size_t * n)(*[int(v) for v in max_samples])
    h = _P()
    st = lib.ss_plan_many(ctypes.byref(h), n, t, ms, float(dt), m, window, float(win_param),
                          orders, precision,
                          _addr(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream)
    _check_many(st, None)
    return h.value


def _ptr_array(bufs):
    if bufs is None:
        return None
    return (_P * len(bufs))(*[_addr(b) for b in bufs])


def ss_run_many(handle, chunks, n_samples, S2=None, S3=None, S4=None, S2_err=None,
                S3_err=None, S4_err=None):
    n = len(chunks)
    ns = (ctypes.c_size_t * n)(*[int(v) for v in n_samples])
    _check_many(lib.ss_run_many(handle, _ptr_array(chunks), ns, _ptr_array(S2), _ptr_array(S3),
                                _ptr_array(S4), _ptr_array(S2_err), _ptr_array(S3_err),
                                _ptr_array(S4_err)), handle)


def ss_many_plan(handle, i):
    h = _P()
    _check_many(lib.ss_many_plan(handle, i, ctypes.byref(h)), handle)
    return h.value


def ss_destroy_many(handle):
    _check_many(lib.ss_destroy_many(handle), handle)


def ss_s2_noalloc(d_signal, n_samples, T, dt, m, window=SS_WIN_HANN, win_param=0.14,
                  d_S2=None, d_S2_err=None, stream=None):
    """Power spectrum of one device-resident float32 channel with no device allocation
    (see include/polyspec.h).  Outputs are device buffers; the call is stream-ordered."""
    st = lib.ss_s2_noalloc(_addr(d_signal), n_samples, T, float(dt), m, window,
                           float(win_param), _addr(d_S2), _addr(d_S2_err),
                           _addr(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream)
    if st != SS_OK:
        raise SSError(st, lib.ss_noalloc_last_error().decode())


class ManyPlan:
    """Many one-channel recordings in one CUDA graph (ss_plan_many / ss_run_many).
    Keeps device output buffers per recording, so repeated runs on the same input
    tensors replay the captured graph."""

    def __init__(self, T_list, max_samples, dt=1.0, m=10, window="hann", sigma_t=0.14,
                 orders=(2, 3, 4), precision="fp32", stream=None):
        import torch

        win = {"hann": SS_WIN_HANN, "acg": SS_WIN_ACG}[window]
        ords = 0
        for o in orders:
            ords |= 1 << o
        prec = {"fp32": SS_PREC_FP32, "tf32x3": SS_PREC_TF32X3, "bf16x3": SS_PREC_BF16X3,
                "bf16": SS_PREC_BF16, "fp16x3": SS_PREC_FP16X3}[precision]
        self.handle = ss_plan_many(T_list, max_samples, dt, m, win, sigma_t, ords, prec, stream)
        self.n = len(T_list)
        self.outs = {}
        for key in ("S2", "S3", "S4"):
            self.outs[key], self.outs[key + "_err"] = [], []
            for i in range(self.n):
                info = ss_query(ss_many_plan(self.handle, i))
                shape = {"S2": (info.n_s2, info.M), "S3": (info.n_s3, info.rows3, info.M),
                         "S4": (info.n_s4, info.rows4, info.M)}[key]
                cnt = int(np.prod(shape)) * 2
                for k2 in (key, key + "_err"):
                    self.outs[k2].append(torch.empty(max(cnt, 1), dtype=torch.float64,
                                                     device="cuda") if cnt else None)

    def plan(self, i):
        return ss_many_plan(self.handle, i)

    def run(self, chunks, n_samples=None):
        if n_samples is None:
            n_samples = [c.shape[-1] for c in chunks]
        o = self.outs
        ss_run_many(self.handle, chunks, n_samples, o["S2"], o["S3"], o["S4"], o["S2_err"],
                    o["S3_err"], o["S4_err"])

    def results(self, i):
        """Spectra of recording i as numpy arrays (as Plan.finalize returns them)."""
        info = ss_query(ss_many_plan(self.handle, i))
        shapes = {"S2": (info.n_s2, info.M), "S3": (info.n_s3, info.rows3, info.M),
                  "S4": (info.n_s4, info.rows4, info.M)}
        out = {"G": info.groups}
        for key, sh in shapes.items():
            if self.outs[key][i] is None:
                continue
            v = self.outs[key][i].cpu().numpy().reshape(sh + (2,))
            out[key] = v[..., 0] + 1j * v[..., 1]
            out[key + "_err"] = self.outs[key + "_err"][i].cpu().numpy().reshape(sh + (2,))
        return out

    def close(self):
        if self.handle:
            ss_destroy_many(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Convenience wrapper: owns a plan handle, returns spectra as numpy arrays."""

    def __init__(self, channels=1, T=256, dt=1.0, m=10, window="hann", sigma_t=0.14,
                 orders=(2, 3, 4), dtype="f32", precision="fp32", combos=None, stream=None,
                 estimator="unbiased", interlaced=False):
        win = {"hann": SS_WIN_HANN, "acg": SS_WIN_ACG}[window]
        ords = 0
        for o in orders:
            ords |= 1 << o
        dt_code = {"f32": SS_F32, "i16": SS_I16}[dtype]
        prec = {"fp32": SS_PREC_FP32, "tf32x3": SS_PREC_TF32X3, "bf16x3": SS_PREC_BF16X3,
                "bf16": SS_PREC_BF16, "fp16x3": SS_PREC_FP16X3}[precision]
        self.handle = ss_plan(channels, T, dt, m, win, sigma_t, ords, dt_code, prec, combos, stream)
        self.orders = tuple(orders)
        if estimator != "unbiased":
            ss_set_estimator(self.handle, {"unbiased": SS_EST_UNBIASED,
                                           "natural": SS_EST_NATURAL}[estimator])
        if interlaced:
            ss_set_interlace(self.handle, 1)
        self.info = ss_query(self.handle)

    def accumulate(self, chunk, n_samples=None):
        if n_samples is None:
            n_samples = chunk.shape[-1]
        ss_accumulate(self.handle, chunk, n_samples)

    def shapes(self):
        i = ss_query(self.handle)
        return {"S2": (i.n_s2, i.M), "S3": (i.n_s3, i.rows3, i.M), "S4": (i.n_s4, i.rows4, i.M)}

    def finalize(self):
        """Returns dict of complex128 arrays S2/S3/S4 and float64 errors [..., 2]."""
        sh = self.shapes()
        out = {}
        bufs = {}
        for key in ("S2", "S3", "S4"):
            n = int(np.prod(sh[key]))
            bufs[key] = np.zeros(sh[key] + (2,), np.float64) if n else None
            bufs[key + "_err"] = np.zeros(sh[key] + (2,), np.float64) if n else None
        ss_finalize(self.handle, bufs["S2"], bufs["S3"], bufs["S4"], bufs["S2_err"],
                    bufs["S3_err"], bufs["S4_err"])
        for key in ("S2", "S3", "S4"):
            if bufs[key] is not None:
                out[key] = bufs[key][..., 0] + 1j * bufs[key][..., 1]
                out[key + "_err"] = bufs[key + "_err"]
        if 1 in self.orders:
            C = ss_query(self.handle).channels
            s1 = np.zeros((C, 2), np.float64)
            e1 = np.zeros((C, 2), np.float64)
            ss_finalize_s1(self.handle, s1, e1)
            out["S1"] = s1[:, 0] + 1j * s1[:, 1]
            out["S1_err"] = e1
        out["G"] = ss_query(self.handle).groups
        return out

    def reset(self):
        ss_reset(self.handle)

    def complex_spectra(self, records):
        """Means and errors of the complex-signal records (ss_set_complex) as a list
        of (mean, err) numpy arrays in record order."""
        M = ss_query(self.handle).M
        nn = 2 * M - 1
        total = ss_complex_size(self.handle)
        mean = np.zeros(total)
        err = np.zeros(total)
        ss_finalize_complex(self.handle, mean, err)
        out, o = [], 0
        for rec in records:
            shape = (nn,) if rec[0] == 2 else (nn, nn)
            k = 2 * int(np.prod(shape))
            v = mean[o:o + k].reshape(shape + (2,))
            out.append((v[..., 0] + 1j * v[..., 1], err[o:o + k].reshape(shape + (2,))))
            o += k
        return out

    def sequential(self, block_groups, max_blocks):
        """Turn on sequential spectra (ss_set_sequential) into a device buffer this
        wrapper owns; ``blocks()`` reads them back."""
        import torch

        n, _ = ss_sequential_info(self.handle)
        self._seq = torch.zeros(max(1, n * max_blocks), dtype=torch.float64, device="cuda")
        self._seq_cap = max_blocks
        ss_set_sequential(self.handle, block_groups, self._seq, max_blocks)

    def blocks(self):
        """The written blocks as a list of dicts like ``finalize()`` returns."""
        import torch

        torch.cuda.synchronize()
        n, done = ss_sequential_info(self.handle)
        sh = self.shapes()
        host = self._seq.cpu().numpy()
        out = []
        for b in range(min(done, self._seq_cap)):
            v, d = host[b * n:(b + 1) * n], {}
            o = 0
            for key in ("S2", "S3", "S4"):
                k = int(np.prod(sh[key])) * 2
                if k:
                    mean = v[o:o + k].reshape(sh[key] + (2,))
                    d[key] = mean[..., 0] + 1j * mean[..., 1]
                    d[key + "_err"] = v[o + k:o + 2 * k].reshape(sh[key] + (2,))
                o += 2 * k
            out.append(d)
        return out

    def export_state(self, out=None):
        """The plan's group sums with their header (float64); a new host array unless
        ``out`` (host or device, ss_state_size doubles) is given."""
        if out is None:
            out = np.empty(ss_state_size(self.handle), np.float64)
        ss_export_state(self.handle, out)
        return out

    def merge_state(self, src):
        """Add a state exported by an identically configured plan."""
        ss_merge_state(self.handle, src)

    def combos(self):
        return ss_combos(self.handle)

    def stats(self):
        return ss_stats(self.handle)

    def close(self):
        if self.handle:
            ss_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_m(record, T, ms, **plan_kw):
    """Quasi-polyspectra of one record for several group sizes m (Sec. 8: spectra
    that change with m reveal non-stationarity): one plan per m over the same
    device record; returns {m: finalize() dict}."""
    out = {}
    for m in ms:
        plan = Plan(T=T, m=m, **plan_kw)
        plan.accumulate(record)
        out[m] = plan.finalize()
        plan.close()
    return out
