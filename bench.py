"""Throughput of the polyspectrum hot path (S2 + S3 + S4) on GB300.

One step = one pass of the whole path over one synthetic record: ss_reset,
ss_accumulate (frame/window/FFT/centre + S2, bispectrum, trispectrum cut) and
ss_finalize (means and standard errors), through the C ABI.

  value : input samples/s with the record already resident in HBM (device
          pointers in and out), CUDA events on the plan's stream.
  e2e   : the same metric through the same C-ABI calls with HOST buffers: the
          record is read from pinned host memory and all spectra and error
          bars are copied back to host memory inside the timed region.

Default workload: one channel, 2^28 float32 samples of x = y + 0.3 (y^2 - 1), y an
AR(1) process (coefficient 0.9, seed 1); frames T = 1024 (513 bins), Hann
window, groups of m = 10 frames; full S2, S3 and S4 grids.  The record (1 GiB)
is larger than L2, so no extra L2 flush is done between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun the ranks shard one record of N x 2^28 samples into contiguous
runs of whole groups (2^28 samples' worth per rank: weak scaling); each rank
runs its plan on its run, and one step ends with the product's merge: the
plans' exported states summed by one all-reduce, merged into rank 0's plan and
finalized there.  Rank 0 prints one JSON line.

Peaks: HBM from MEASURED_PEAKS.json; the FP32-FMA and the tcgen05 TF32 / BF16
peaks are measured at the start of the run by the microbenchmarks of
libsspeaks.so, with the SM clock sampled meanwhile.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input samples/s for S2+S3+S4 at stated T,m; % of HBM/FP32/tensor peak; err vs FP64"

WORKLOADS = {
    # name: (channels, n samples per channel, T, m, seed)
    "ar1q-2^28-T1024-m10": dict(channels=1, n=1 << 28, T=1024, m=10, seed=1, phi=0.9),
    "ar1q-2^20-T256-m10": dict(channels=1, n=1 << 20, T=256, m=10, seed=0, phi=0.9),
    # same shapes as the default at 1/8 of the length (profiling captures)
    "ar1q-2^25-T1024-m10": dict(channels=1, n=1 << 25, T=1024, m=10, seed=1, phi=0.9),
    # 64 independent recordings, lengths log-uniform in [2^20, 2^26], T from
    # {128, 256, 512, 1024}, AR coefficients uniform in [0.5, 0.98], one CUDA graph;
    # refused (REFUSED below)
    "many64-2^20..2^26-m10": dict(channels=1, many=64, m=10, seed=100),
    # int16 ADC record (low-passed telegraph plus noise) streamed from page-locked
    # host memory in 256 MiB chunks; 1/16 of the 2^34-sample streamed configuration
    "adc16-2^30-T4096-m10": dict(channels=1, n=1 << 30, T=4096, m=10, seed=5, dtype="i16",
                                 chunk=1 << 27, cpu_groups=3),
    # four channels sharing an AR(1) component (plus white noise, a quadratic term
    # and a telegraph signal each), every default cross combination of S2/S3/S4
    "mc4-2^26-T512-m20": dict(channels=4, n=1 << 26, T=512, m=20, seed=3, cpu_groups=2),
    # same shapes at 1/16 of the length (profiling captures)
    "mc4-2^22-T512-m20": dict(channels=4, n=1 << 22, T=512, m=20, seed=3, cpu_groups=2),
}
DEFAULT_WORKLOAD = "ar1q-2^28-T1024-m10"
# workloads this build does not run, with the reason
REFUSED = {
    "many64-2^20..2^26-m10": "its runs ended in a fault (first an 'unspecified launch failure' "
                             "at the first graph launch with four concurrent branches, then a "
                             "host segfault with GPU Xid 43 with one stream); the cause is not "
                             "found, so it stays off",
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_record(w, rank):
    import synth

    if w.get("dtype") == "i16":
        return synth.adc_telegraph_int16_parallel(w["n"], seed=w["seed"] + rank,
                                                  processes=min(16, os.cpu_count() or 1))
    if w["channels"] > 1:
        return synth.multichannel_shared(w["channels"], w["n"], seed=w["seed"] + rank)

    return synth.ar1_quadratic(w["n"], seed=w["seed"] + rank, phi=w["phi"])


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


def fp32_peak_tflops(nsm, pk):
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock, at the maximum
    # SM clock: the fallback when the FMA microbenchmark could not run
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    return nsm * 128 * 2 * mhz * 1e6 / 1e12


def measure_peaks(gpu_index):
    """FP32-FMA and tcgen05 TF32 / BF16 / FP16 dense peaks of this GPU, measured
    now by libsspeaks.so (CUDA events, about 0.1 s each), with the SM clock sampled
    during the runs.  Returns {} if the library is missing."""
    path = os.path.join(ROOT, "paper_2505_01231_gb300", "libsspeaks.so")
    if not os.path.exists(path):
        return {}
    lib = ctypes.CDLL(path)
    lib.ssp_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    lib.ssp_mma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    sec, rate = ctypes.c_double(), ctypes.c_double()
    out = {}
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.2)
    if lib.ssp_fma_peak(100000, ctypes.byref(sec), ctypes.byref(rate)) == 0:
        out["fp32_tflops"] = rate.value / 1e12
    for kind, key in ((0, "tf32_tflops"), (1, "bf16_tflops"), (2, "fp16_tflops")):
        if lib.ssp_mma_peak(kind, 300000, ctypes.byref(sec), ctypes.byref(rate)) == 0:
            out[key] = rate.value / 1e12
    out["clocks"] = clocks.stop()
    out["how"] = ("libsspeaks.so: FP32 FMA, 2048 threads per SM x 16 independent chains; "
                  "tcgen05.mma 128x256 (K 8 tf32 / 16 bf16, fp16) from shared memory into TMEM, one "
                  "CTA per SM, one issuing thread; CUDA events, the whole device")
    return out


def mma_shapes(gpu_index):
    """tcgen05 product rate against N (M = 128; K = 8 TF32 or 16 BF16 per product),
    the measurement behind the cross-channel S4 tile width: narrow products are
    paced by their operand reads from shared memory, not by the multipliers."""
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2505_01231_gb300", "libsspeaks.so"))
    lib.ssp_mma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    import torch
    nsm = torch.cuda.get_device_properties(gpu_index).multi_processor_count
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.2)
    iters, out = 100000, {}
    for kind, name in ((0, "tf32"), (1, "bf16")):
        for n in (32, 64, 96, 128, 256):
            sec, rate = ctypes.c_double(), ctypes.c_double()
            if lib.ssp_mma_rate(kind, n, iters, ctypes.byref(sec), ctypes.byref(rate)) != 0:
                continue
            per_product = sec.value / (iters * 4)              # one SM's products are serial
            kbytes = 128 * 32 / 1024 + n * 32 / 1024           # A and B read per product (KB)
            out[f"{name}_n{n}"] = {"tflops": rate.value / 1e12, "ns_per_product": per_product * 1e9,
                                   "operand_kb_per_product": kbytes,
                                   "operand_gb_s_per_sm": kbytes * 1024 / per_product / 1e9}
    info = clocks.stop()
    return {"mma_shapes": out, "sms": nsm, "clocks": info,
            "how": "libsspeaks.so ssp_mma_rate: one CTA per SM, one thread issuing 128 x N products "
                   "from shared memory (K-major, no swizzle) into two TMEM accumulators; CUDA events"}


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is
    unchanged since the capture (source hash recorded beside the figure)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2505_01231_gb300", "csrc", rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec["bytes_per_launch"] if h == rec["sha256_16"] else None


def default_combos(C):
    """The plan's default channel combinations (listed in the C header): every
    multiset for S2 and S3, every unordered pair of unordered channel pairs for the
    S4 cut C4(a_k, b_k*, c_l, d_l*).  {order: [tuple, ...]} in the plan's order."""
    pairs = [(a, b) for a in range(C) for b in range(a, C)]
    return {2: pairs,
            3: [(a, b, c) for a in range(C) for b in range(a, C) for c in range(b, C)],
            4: [pairs[i] + pairs[j] for i in range(len(pairs)) for j in range(i, len(pairs))]}


# ------------------------------------------------------------------ CPU oracle
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_job(z, T, m, combos):
    """One host core: the FP64 oracle on one slice of whole groups (single-threaded
    numpy), timed inside the worker."""
    import oracle

    t0 = time.perf_counter()
    if z.ndim == 1:
        ref = oracle.polyspectra(z, T, 1.0, m, group_chunk=64)
    else:
        ref = oracle.cross_polyspectra(z, T, 1.0, m, s2_combos=combos[2], s3_combos=combos[3],
                                       s4_combos=combos[4], group_chunk=64)
    return time.perf_counter() - t0, ref


def oracle_on_cores(z, T, m, groups, cores, combos=None, offset_groups=0):
    """The oracle as it stands on `cores` host cores at once: core i takes the i-th
    slice of `groups` whole groups (from `offset_groups` on).  Returns (samples/s
    over all cores, the slowest core's seconds, the first slice's estimate).  The
    pool is spawned (no fork after CUDA) and single-threaded per worker."""
    import multiprocessing as mp

    n = groups * m * T
    C = 1 if z.ndim == 1 else z.shape[0]
    avail = (z.shape[-1] // (m * T) - offset_groups) // groups
    cores = max(1, min(cores, avail))
    jobs = []
    for i in range(cores):
        a = (offset_groups + i * groups) * m * T
        jobs.append((np.ascontiguousarray(z[..., a:a + n]), T, m, combos))
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_job, jobs)
    slowest = max(r[0] for r in res)
    return cores * C * n / slowest, slowest, res[0][1], cores


# ------------------------------------------------------------------ reference arm
def run_reference(args, w, rank, world):
    if rank != 0:
        return
    if "many" in w:  # a bounded sample: the first recording's process, T = 512
        import synth

        z = synth.ar1_quadratic(1 << 22, seed=w["seed"] + 1, phi=0.74)
        w = dict(w, T=512)
    else:
        z = make_record(w, 0)
    T, m = w["T"], w["m"]
    C = 1 if z.ndim == 1 else z.shape[0]
    combos = default_combos(C) if C > 1 else None
    cores = host_cores()
    ts, vals, used = [], [], 1
    for i in range(args.warmup + args.steps):
        # each step a fresh stretch of the record (wrapping at its end)
        span = args.ref_groups * max(1, cores)
        total = z.shape[-1] // (m * T)
        off = (i * span) % max(1, total - span)
        value, sec, _, used = oracle_on_cores(z, T, m, args.ref_groups, cores, combos, off)
        if i >= args.warmup:
            ts.append(sec)
            vals.append(value)
    value = float(np.mean(vals))
    sec = float(np.mean(ts))
    n_step = args.ref_groups * m * T
    sample = (f"{args.ref_groups} groups ({n_step} samples per channel, {C} channels) per core "
              f"and step on {used} host cores at once, full S2/S3/S4 grids"
              + (", every default combination" if C > 1 else "") + ", numpy float64")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "T": T, "m": m,
                   "samples_per_step": n_step * used * C},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(w, z, groups, combos=None):
    """The FP64 oracle on all host cores, each on its own prefix slice of `groups`
    groups; returns the baseline line and the estimate of the first slice (the
    record's first `groups` groups, for the error check)."""
    T, m = w["T"], w["m"]
    sel = None
    if z.ndim > 1:
        sel = {o: [tuple(r[1:1 + o]) for r in combos if r[0] == o] for o in (2, 3, 4)}
    value, sec, ref, used = oracle_on_cores(z, T, m, groups, host_cores(), sel)
    what = ("full S2/S3/S4 grids" if z.ndim == 1 else
            f"{z.shape[0]} channels, full grids of every default combination")
    line = {"value": value, "unit": "samples/s", "cores": used, "kind": "oracle",
            "sample": f"{groups} groups ({groups * m * T} samples per channel) per core, the "
                      f"record's first {groups * used} groups, {what}, numpy float64, one "
                      f"process per host core ({used} of {os.cpu_count()}), slowest core "
                      f"{sec:.1f} s"}
    return line, ref


def error_vs_oracle(P, w, z, ref, groups, precision):
    """max |GPU - oracle| / max |oracle| per spectrum on the oracle's prefix, through the
    same C-ABI path and precision as the timed run."""
    import torch

    T, m = w["T"], w["m"]
    n = groups * m * T
    C = 1 if z.ndim == 1 else z.shape[0]
    plan = P.Plan(channels=C, T=T, dt=1.0, m=m, orders=(2, 3, 4), precision=precision,
                  dtype=w.get("dtype", "f32"))
    combos = plan.combos()
    plan.accumulate(torch.from_numpy(np.ascontiguousarray(z[..., :n])).cuda(), n)
    out = plan.finalize()
    plan.close()
    errs = {}
    for key in ("S2", "S3", "S4"):
        if C == 1:
            a, b = out[key][0].reshape(ref[key].shape), ref[key]
            errs[key] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
            continue
        o = int(key[1])
        worst = 0.0
        for i, c in enumerate([tuple(r[1:1 + o]) for r in combos if r[0] == o]):
            b = ref[(key, c)][0]
            a = out[key][i].reshape(b.shape)
            worst = max(worst, float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
        errs[key] = worst
    errs["groups"] = groups
    errs["precision"] = precision
    return errs


def make_many(w):
    """Lengths, frame lengths and AR coefficients of the batched workload, then the
    records (one seed per recording)."""
    import synth

    k = w["many"]
    u = synth.uniform(3 * k, seed=w["seed"])
    lens = [int(2.0 ** (20 + 6 * u[i])) for i in range(k)]
    Ts = [(128, 256, 512, 1024)[min(3, int(4 * u[k + i]))] for i in range(k)]
    phis = [0.5 + 0.48 * u[2 * k + i] for i in range(k)]
    jobs = [(n, w["seed"] + 1 + i, phi) for i, (n, phi) in enumerate(zip(lens, phis))]
    import multiprocessing as mp

    # records generated in parallel, in spawned processes, before any CUDA call
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        zs = pool.starmap(_ar1q_job, jobs)
    return Ts, zs


def _ar1q_job(n, seed, phi):
    import synth

    return synth.ar1_quadratic(n, seed=seed, phi=phi)


def run_many(args, w, rank, world):
    """The batched-recordings workload: every step is one replay of the graph that
    processes all recordings (reset, accumulate, finalize each)."""
    Ts, zs = make_many(w)
    import torch

    import paper_2505_01231_gb300 as P

    torch.cuda.set_device(0)
    total = sum(len(z) for z in zs)
    stream = torch.cuda.current_stream()
    many = P.ManyPlan(Ts, [len(z) for z in zs], m=w["m"], precision=args.precision,
                      stream=stream)
    dz = [torch.from_numpy(z).cuda() for z in zs]
    for _ in range(args.warmup):
        many.run(dz)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        many.run(dz)
    t1.record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    line = {
        "metric": METRIC, "value": total * args.steps / elapsed, "unit": "samples/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "recordings": len(zs), "samples": total,
                   "T_counts": {str(t): Ts.count(t) for t in (128, 256, 512, 1024)},
                   "m": w["m"], "s4_precision": args.precision,
                   "l2": f"records of {4 * total / 2**30:.1f} GiB per step are larger than L2"},
        "tuning": {str(t): P.ss_get_tuning(many.plan(Ts.index(t))).split(" | ")[1]
                   for t in sorted(set(Ts))},
        "e2e": None, "gpu_launches": None, "roofline": None, "cpu_baseline": None,
        "clocks": clock_info,
    }
    print(json.dumps(line), flush=True)
    many.close()


# ------------------------------------------------------------------ our arm
def timed_steps(P, plan, step, steps, stream):
    """Device time of `steps` calls of step() with CUDA events on the plan's stream,
    and the per-stage event sums of the plan (ss_stats, reset by each ss_reset)."""
    import torch

    stage_ms = np.zeros(5)
    stage_launches = np.zeros(5)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step()
        st = P.ss_stats(plan.handle)   # per-stage event times of this step (reset clears)
        stage_ms += np.array(st.ms[:])
        stage_launches += np.array(st.launches[:])
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / 1e3, stage_ms, stage_launches


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-groups", type=int, default=16,
                    help="groups per host core of the CPU oracle baseline")
    ap.add_argument("--ref-groups", type=int, default=4,
                    help="groups per host core and step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the peak microbenchmarks")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plan's default kernel forms")
    ap.add_argument("--tuning", default=None,
                    help="apply this tuning text (ss_set_tuning) instead of autotuning")
    ap.add_argument("--fp32-steps", type=int, default=3,
                    help="steps of the all-FP32 S4 arm (0 = skip)")
    ap.add_argument("--mma-shapes", action="store_true",
                    help="print the tcgen05 product rate against N and exit")
    ap.add_argument("--precision", default="fp16x3",
                    choices=["fp32", "tf32x3", "bf16x3", "bf16", "fp16x3"],
                    help="arithmetic of the S4 moment sums")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    rank, world, local = dist_env()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    if args.mma_shapes:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(mma_shapes(local)), flush=True)
        return
    if args.workload in REFUSED:
        if rank == 0:
            print(f"bench.py: workload {args.workload} is refused: {REFUSED[args.workload]}",
                  file=sys.stderr)
        sys.exit(2)
    if "many" in w:
        if rank == 0:
            run_many(args, w, rank, world)
        return

    import torch

    import paper_2505_01231_gb300 as P
    from paper_2505_01231_gb300 import shard

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    T, m, C = w["T"], w["m"], w["channels"]
    if world > 1:
        # one record of world x n samples, sharded into contiguous runs of whole
        # groups; each rank draws its own run (seed + rank) of the synthetic record
        ranges = shard.group_ranges(world * w["n"], T, m, world)
        a, b = ranges[rank]
        z = make_record(dict(w, n=b - a), rank)
    else:
        z = make_record(w, 0)
    n = z.shape[-1]
    pk = peaks()
    measured = {}
    if not args.no_peaks:
        measured = measure_peaks(local)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = measured.get("fp32_tflops") or fp32_peak_tflops(nsm, pk)
    fp32_src = ("measured now (FP32 FMA microbenchmark)" if measured.get("fp32_tflops") else
                "derived: SMs x 128 FP32 lanes x 2 flop x max SM clock")

    stream = torch.cuda.current_stream()
    plan = P.Plan(channels=C, T=T, dt=1.0, m=m, orders=(2, 3, 4), stream=stream,
                  dtype=w.get("dtype", "f32"), precision=args.precision)
    info = P.ss_query(plan.handle)
    if args.tuning:
        P.ss_set_tuning(plan.handle, args.tuning)
    elif not args.no_autotune:
        P.ss_autotune(plan.handle)   # the fastest kernel forms for these shapes on this GPU
    tuning = P.ss_get_tuning(plan.handle)
    dz = torch.from_numpy(z).cuda()
    sh = plan.shapes()
    outs = {k: torch.empty(int(np.prod(v)) * 2, dtype=torch.float64, device="cuda")
            for k, v in sh.items()}
    errs = {k: torch.empty_like(v) for k, v in outs.items()}
    state = None
    if world > 1:
        state = torch.empty(P.ss_state_size(plan.handle), dtype=torch.float64, device="cuda")

    def merge_and_finalize(S, E):
        # the product's sharded path: export, one sum all-reduce of the states,
        # merge into rank 0's (reset) plan, finalize there
        P.ss_export_state(plan.handle, state)
        shard.reduce_state(state)
        if rank == 0:
            P.ss_reset(plan.handle)
            P.ss_merge_state(plan.handle, state)
            P.ss_finalize(plan.handle, S["S2"], S["S3"], S["S4"], E["S2"], E["S3"], E["S4"])

    def step_device(merge=True):
        P.ss_reset(plan.handle)
        P.ss_accumulate(plan.handle, dz, n)
        if world == 1:
            P.ss_finalize(plan.handle, outs["S2"], outs["S3"], outs["S4"], errs["S2"],
                          errs["S3"], errs["S4"])
        elif merge:
            merge_and_finalize(outs, errs)
        else:
            torch.cuda.current_stream().synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(args.warmup):
        step_device()
    barrier()
    P.ss_reset(plan.handle)
    P.ss_set_timing(plan.handle, 1)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    elapsed, stage_ms, stage_launches = timed_steps(P, plan, step_device, args.steps, stream)
    barrier()
    clock_info = clocks.stop()
    P.ss_set_timing(plan.handle, 0)
    elapsed = max_over_ranks(elapsed)
    ms_per_step = elapsed / args.steps * 1e3
    groups = n // (m * T)
    value = world * C * n * args.steps / elapsed  # input samples of all channels, all ranks
    merge_info = None
    if world > 1:
        barrier()
        e2, _, _ = timed_steps(P, plan, lambda: step_device(merge=False), args.steps, stream)
        e2 = max_over_ranks(e2)
        merge_info = {"ms_per_step_with_merge": ms_per_step,
                      "ms_per_step_without_merge": e2 / args.steps * 1e3,
                      "value_without_merge": world * C * n * args.steps / e2,
                      "state_doubles": int(state.numel()),
                      "path": "ss_export_state -> shard.reduce_state (one SUM all-reduce) -> "
                              "ss_merge_state into rank 0's reset plan -> ss_finalize"}

    # ---- per-stage rooflines (live CUDA events on the plan's stream)
    st = P.ss_stats(plan.handle)
    frames = groups * m
    M = T // 2 + 1
    Mp = (M + 15) // 16 * 16
    s4_name = "k3_trispec" if C == 1 else "k3_trispec_cross"
    if args.precision != "fp32":
        s4_name = "k3_trispec_tc" if C == 1 else "k3_trispec_cross_tc"
    # several channels: the cross S4 runs FP16x3 with fp16x3, TF32x3 with the other
    # tensor-core precisions
    s4_prec = (args.precision if C == 1 or args.precision in ("fp32", "fp16x3") else "tf32x3")
    # the K2 form the autotuner (or --tuning) chose: its kernel's name; the
    # independent-warp form runs only with one channel (the plan takes the 8 x 4
    # tiling for several)
    k2_form = (tuning.split(" k2=")[1].split()[0] if " k2=" in tuning else "44")
    k2_name = {"84s2": "k2_bispec84", "84s3": "k2_bispec84",
               "84w": "k2_bispec84w" if C == 1 else "k2_bispec84"}.get(k2_form, "k2_bispec")
    names = ["k1_spectra", "k2_bispec", s4_name, "k4_finalize", "h2d"]
    n_batches = max(1, int(np.ceil(groups / info.groups_per_batch)))
    hbm = float(pk.get("hbm_gbs", 6800.0))

    # K1 against HBM on the algorithmic bytes of the step (section (d) of the
    # design): the samples read and the centred spectra written, M bins per frame;
    # what the kernel moves beyond that (bins padded to Mp, the tensor-core operand
    # image and its FP16 row scales in the split modes) is reported as overhead
    k1_ms = stage_ms[0] / args.steps
    k1_bytes = frames * C * (T * z.itemsize + M * 8)
    k1_over = frames * C * (Mp - M) * 8
    if args.precision != "fp32" and C == 1:
        # K chunks: the diagonal entries, then the pairs and ps; image rows for the
        # bins the tiles read (up to M - 2 when the last column has a kernel of its own)
        nkc = (m + 15) // 16 + (m * (m - 1) // 2 + 16) // 16
        img_bins = M - 1 if (M - 1) % 128 == 0 else Mp
        k1_over += groups * C * img_bins * (nkc * 16 * 2 * (4 if args.precision == "tf32x3" else 2) +
                                            (4 if args.precision == "fp16x3" else 0))
    k1_ach = k1_bytes / (k1_ms / 1e3) / 1e9 if k1_ms > 0 else None
    roofline_k1 = {"bound": "hbm", "kernel": "k1_spectra", "achieved": k1_ach, "peak": hbm,
                   "unit": "GB/s", "frac": (k1_ach / hbm) if k1_ach else None,
                   "traffic": (traffic_for("k1_spectra_" + args.precision) if C == 1 else None),
                   "traffic_note": f"DRAM bytes per launch (ncu); a step is {n_batches} launches",
                   "algorithmic_bytes_per_step": k1_bytes, "overhead_bytes_per_step": k1_over,
                   "frac_with_overhead": ((k1_bytes + k1_over) / (k1_ms / 1e3) / 1e9 / hbm)
                   if k1_ms > 0 else None,
                   "peak_source": "measured (MEASURED_PEAKS.json, copy)", "ms_per_step": k1_ms}

    # K2 against the FP32 pipe: 14 flop per (grid point, frame)
    k2_ms = stage_ms[1] / args.steps
    k2_flops = 14.0 * st.pairs3 * frames * info.n_s3
    k2_ach = k2_flops / (k2_ms / 1e3) / 1e12 if k2_ms > 0 else None
    roofline_k2 = {"bound": "alu", "kernel": k2_name, "achieved": k2_ach, "peak": fp32_peak,
                   "unit": "TFLOP/s", "frac": (k2_ach / fp32_peak) if k2_ach else None,
                   "traffic": traffic_for(k2_name), "peak_source": fp32_src,
                   "flop_per_step": k2_flops, "ms_per_step": k2_ms}

    # S4: the tensor pipe in the split modes.  One channel: the method's work is one
    # pass of the Gram contraction, m(m+1) flop per grid point (k <= l) and group.
    # Several channels: five complex products per point and frame, 40 flop (as the
    # real products of the tensor-core form: 10 columns x K = 2m x 2 flop).  The
    # split modes issue it three times (hi*hi, hi*lo, lo*hi), padded to whole tiles
    # and K chunks.  The CUDA-core forms: 10 (one channel) or 40 (several) flop per
    # point and frame against the FP32 pipe.
    s4_ms = stage_ms[2] / args.steps
    if args.precision == "fp32":
        s4_flops = (10.0 if C == 1 else 40.0) * st.pairs4 * frames * info.n_s4
        s4_peak, s4_bound, s4_src, passes = fp32_peak, "alu", fp32_src, 1
    else:
        passes = 1 if s4_prec == "bf16" else 3
        s4_flops = (float(st.pairs4) * groups * m * (m + 1) if C == 1
                    else 40.0 * st.pairs4 * frames * info.n_s4)
        key = {"tf32x3": "tf32_tflops", "fp16x3": "fp16_tflops"}.get(s4_prec, "bf16_tflops")
        if measured.get(key):
            s4_peak, s4_src = measured[key], f"measured now (tcgen05 {key[:4]} microbenchmark)"
        elif s4_prec == "tf32x3":
            s4_peak = float(pk.get("bf16_tflops", 1900.0)) * 1.1 / 2.25
            s4_src = "measured bf16 x nominal tf32/bf16 dense ratio (1.1/2.25 PFLOP/s)"
        else:
            s4_peak, s4_src = float(pk.get("bf16_tflops", 1900.0)), "MEASURED_PEAKS.json bf16"
        s4_bound = "tensor"
    s4_ach = s4_flops / (s4_ms / 1e3) / 1e12 if s4_ms > 0 else None
    roofline_s4 = {"bound": s4_bound, "kernel": s4_name, "achieved": s4_ach, "peak": s4_peak,
                   "unit": "TFLOP/s", "frac": (s4_ach / s4_peak) if s4_ach else None,
                   "traffic": traffic_for(s4_name), "peak_source": s4_src,
                   "flop_per_step": s4_flops, "ms_per_step": s4_ms}
    if s4_bound == "tensor" and s4_ach:
        roofline_s4["passes"] = passes
        roofline_s4["issued_frac"] = s4_ach * passes / s4_peak
        roofline_s4["note"] = ("frac: the method's one-pass products per second; issued_frac: "
                               "the split mode's passes, before tile and K-chunk padding")

    # the dominant kernel of the step carries the contract's roofline
    stage_rl = [roofline_k1, roofline_k2, roofline_s4]
    dom = int(np.argmax(stage_ms[:3]))
    roofline = dict(stage_rl[dom])
    roofline["stage_ms_per_step"] = {nm: float(stage_ms[i] / args.steps)
                                     for i, nm in enumerate(names[:4])}
    roofline["launch_ms"] = float(stage_ms[dom] / max(1, stage_launches[dom]))
    gpu_launches = int(args.steps * (n_batches * info.kernels_per_batch + 3))

    # ---- end to end through the same calls with host buffers
    e2e = None
    if not args.no_e2e:
        hz = torch.from_numpy(z).pin_memory()
        # the caller's result buffers in page-locked host memory, so that finalize's
        # device-to-host copies run as DMA
        def pinned(count):
            return torch.empty(count, dtype=torch.float64, pin_memory=True).numpy()

        host_out = {k: pinned(int(np.prod(v)) * 2) for k, v in sh.items()}
        host_err = {k: pinned(int(np.prod(v)) * 2) for k, v in sh.items()}

        chunk = w.get("chunk", n)  # samples per ss_accumulate call (a streaming caller)

        def step_host():
            P.ss_reset(plan.handle)
            for a in range(0, n, chunk):
                P.ss_accumulate(plan.handle, hz[..., a:a + chunk], min(chunk, n - a))
            if world == 1:
                P.ss_finalize(plan.handle, host_out["S2"], host_out["S3"], host_out["S4"],
                              host_err["S2"], host_err["S3"], host_err["S4"])
            else:
                merge_and_finalize(host_out, host_err)

        for _ in range(2):
            step_host()
        barrier()
        h0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        barrier()
        he = max_over_ranks(time.perf_counter() - h0)
        d2h = sum(v.nbytes for v in host_out.values()) + sum(v.nbytes for v in host_err.values())
        e2e = {"value": world * C * n * args.steps / he, "unit": "samples/s",
               "h2d_bytes_per_step": int(z.nbytes) * world,
               "d2h_bytes_per_step": int(d2h)}

    cpu, err_fp64, ref, cg = None, None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cg = w.get("cpu_groups", args.cpu_groups)
        cpu, ref = cpu_baseline(w, z, cg, plan.combos())
        err_fp64 = error_vs_oracle(P, w, z, ref, cg, args.precision)

    # ---- the all-FP32 CUDA-core form of the same step (S4 on CUDA cores), for the
    # mixed-precision speed-up at the accuracy each reaches
    fp32_arm = None
    if world == 1 and args.precision != "fp32" and args.fp32_steps > 0:
        plan.close()
        plan = P.Plan(channels=C, T=T, dt=1.0, m=m, orders=(2, 3, 4), stream=stream,
                      dtype=w.get("dtype", "f32"), precision="fp32")
        if not args.no_autotune:
            P.ss_autotune(plan.handle)
        step_device()
        torch.cuda.synchronize()
        P.ss_reset(plan.handle)
        P.ss_set_timing(plan.handle, 1)
        e32, ms32, _ = timed_steps(P, plan, step_device, args.fp32_steps, stream)
        fp32_arm = {"value": C * n * args.fp32_steps / e32, "unit": "samples/s",
                    "ms_per_step": e32 / args.fp32_steps * 1e3,
                    "s4_ms_per_step": float(ms32[2] / args.fp32_steps),
                    "steps": args.fp32_steps}
        fp32_arm["speedup_of_mixed"] = value / fp32_arm["value"]
        fp32_arm["s4_speedup_of_mixed"] = fp32_arm["s4_ms_per_step"] / s4_ms if s4_ms else None
        if ref is not None:
            fp32_arm["err_vs_fp64"] = error_vs_oracle(P, w, z, ref, cg, "fp32")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "channels": C, "samples_per_rank": n, "T": T,
                       "M": M, "m": m, "groups": groups, "window": "hann",
                       "orders": "S2+S3+S4 full grids",
                       "s4_precision": s4_prec if s4_prec == args.precision
                       else f"{s4_prec} (several channels; --precision {args.precision})",
                       "dtype_in": w.get("dtype", "f32"),
                       "parallelism": (f"dp{world}: one record sharded in whole groups, states "
                                       "merged by one all-reduce" if world > 1 else "1 GPU"),
                       "l2": f"record of {z.nbytes / 2**30:.0f} GiB per step is larger than L2; "
                             "no flush"},
            "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roofline,
            "roofline_k1": roofline_k1, "roofline_k2": roofline_k2, "roofline_s4": roofline_s4,
            "tuning": tuning,
            "peaks_measured": measured or None, "err_vs_fp64": err_fp64, "fp32_arm": fp32_arm,
            "merge": merge_info, "cpu_baseline": cpu, "clocks": clock_info,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
