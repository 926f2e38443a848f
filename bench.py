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
Under torchrun each rank processes its own record (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
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
    # {128, 256, 512, 1024}, AR coefficients uniform in [0.5, 0.98], one CUDA graph
    "many64-2^20..2^26-m10": dict(channels=1, many=64, m=10, seed=100),
    # int16 ADC record (low-passed telegraph plus noise) streamed from page-locked
    # host memory in 256 MiB chunks; 1/16 of the 2^34-sample streamed configuration
    "adc16-2^30-T4096-m10": dict(channels=1, n=1 << 30, T=4096, m=10, seed=5, dtype="i16",
                                 chunk=1 << 27, cpu_groups=3),
    # four channels sharing an AR(1) component (plus white noise, a quadratic term
    # and a telegraph signal each), every default cross combination of S2/S3/S4
    "mc4-2^26-T512-m20": dict(channels=4, n=1 << 26, T=512, m=20, seed=3, cpu_groups=2),
}
DEFAULT_WORKLOAD = "ar1q-2^28-T1024-m10"


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
    # SM clock; no FP32 FMA peak is measured, so this is derived from unit counts
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    return nsm * 128 * 2 * mhz * 1e6 / 1e12


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


# ------------------------------------------------------------------ reference arm
def run_reference(args, w, rank, world):
    if rank != 0:
        return
    import oracle

    if "many" in w:  # a bounded sample: the first recording's process, T = 512
        import synth

        z = synth.ar1_quadratic(1 << 20, seed=w["seed"] + 1, phi=0.74)
        w = dict(w, T=512)
    else:
        z = make_record(w, 0)
    T, m = w["T"], w["m"]
    groups_per_step = args.ref_groups
    n_step = groups_per_step * m * T
    C = 1 if z.ndim == 1 else z.shape[0]
    if C > 1:
        sel = default_combos(C)
    ts = []
    for i in range(args.warmup + args.steps):
        off = (i * n_step) % max(1, (z.shape[-1] - n_step))
        t0 = time.perf_counter()
        if C == 1:
            oracle.polyspectra(z[off:off + n_step], T, 1.0, m, group_chunk=groups_per_step)
        else:
            oracle.cross_polyspectra(z[:, off:off + n_step], T, 1.0, m, s2_combos=sel[2],
                                     s3_combos=sel[3], s4_combos=sel[4],
                                     group_chunk=groups_per_step)
        if i >= args.warmup:
            ts.append(time.perf_counter() - t0)
    sec = float(np.mean(ts))
    value = C * n_step / sec
    sample = (f"{groups_per_step} groups ({n_step} samples per channel, {C} channels) of the "
              f"same record per step, full S2/S3/S4 grids, numpy float64")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "T": T, "m": m, "samples_per_step": n_step},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(w, z, groups, combos=None):
    """Time the FP64 oracle on a prefix of the record; return the line and its spectra.
    Several channels: the oracle's cross-spectra of every combination in `combos`."""
    import oracle

    T, m = w["T"], w["m"]
    n = groups * m * T
    t0 = time.perf_counter()
    if z.ndim == 1:
        ref = oracle.polyspectra(z[:n], T, 1.0, m, group_chunk=groups)
    else:
        sel = {o: [tuple(r[1:1 + o]) for r in combos if r[0] == o] for o in (2, 3, 4)}
        ref = oracle.cross_polyspectra(z[:, :n], T, 1.0, m, s2_combos=sel[2],
                                       s3_combos=sel[3], s4_combos=sel[4], group_chunk=groups)
    sec = time.perf_counter() - t0
    what = ("full S2/S3/S4 grids" if z.ndim == 1 else
            f"{z.shape[0]} channels, full grids of every default combination")
    line = {"value": (1 if z.ndim == 1 else z.shape[0]) * n / sec, "unit": "samples/s",
            "cores": 1, "kind": "oracle",
            "sample": f"first {groups} groups ({n} samples per channel) of the record, {what}, "
                      f"numpy float64 on one host core, {sec:.1f} s"}
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
        "e2e": None, "gpu_launches": None, "roofline": None, "cpu_baseline": None,
        "clocks": clock_info,
    }
    print(json.dumps(line), flush=True)
    many.close()


# ------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-groups", type=int, default=24)
    ap.add_argument("--ref-groups", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32x3", "bf16x3", "bf16"],
                    help="arithmetic of the S4 moment sums")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    rank, world, local = dist_env()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    if "many" in w:
        if rank == 0:
            run_many(args, w, rank, world)
        return

    import torch

    import paper_2505_01231_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    z = make_record(w, rank)
    n = z.shape[-1]
    T, m, C = w["T"], w["m"], w["channels"]
    stream = torch.cuda.current_stream()
    plan = P.Plan(channels=C, T=T, dt=1.0, m=m, orders=(2, 3, 4), stream=stream,
                  dtype=w.get("dtype", "f32"),
                  precision=args.precision)
    info = P.ss_query(plan.handle)
    dz = torch.from_numpy(z).cuda()
    sh = plan.shapes()
    outs = {k: torch.empty(int(np.prod(v)) * 2, dtype=torch.float64, device="cuda")
            for k, v in sh.items()}
    errs = {k: torch.empty_like(v) for k, v in outs.items()}

    def step_device():
        P.ss_reset(plan.handle)
        P.ss_accumulate(plan.handle, dz, n)
        P.ss_finalize(plan.handle, outs["S2"], outs["S3"], outs["S4"], errs["S2"], errs["S3"],
                      errs["S4"])

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step_device()
    barrier()
    P.ss_reset(plan.handle)
    P.ss_set_timing(plan.handle, 1)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    stage_ms = np.zeros(5)
    stage_launches = np.zeros(5)
    for _ in range(args.steps):
        step_device()
        st = P.ss_stats(plan.handle)   # per-stage event times of this step (reset clears)
        stage_ms += np.array(st.ms[:])
        stage_launches += np.array(st.launches[:])
    t1.record(stream)
    barrier()
    clock_info = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    P.ss_set_timing(plan.handle, 0)
    if dist is not None:
        t = torch.tensor([elapsed], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    ms_per_step = elapsed / args.steps * 1e3
    G = info.groups if info.groups else (n // (m * T))
    groups = n // (m * T)
    value = world * C * n * args.steps / elapsed  # input samples of all channels

    # ---- roofline of the dominant kernel (live CUDA events on the plan's stream)
    pk = peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    st = P.ss_stats(plan.handle)
    frames = groups * m
    # several channels: S4 of every combination on CUDA cores in FP32 (k3_trispec_cross)
    s4_name = "k3_trispec" if C == 1 else "k3_trispec_cross"
    names = ["k1_spectra", "k2_bispec", s4_name, "k4_finalize", "h2d"]
    dom = int(np.argmax(stage_ms[:3]))
    n_batches = max(1, int(np.ceil(groups / info.groups_per_batch)))
    launches = stage_launches[dom]
    if dom == 0:
        bytes_per_step = frames * (4 * T * C + 8 * (T // 2 + 1) * C)
        achieved = bytes_per_step * args.steps / (stage_ms[0] / 1e3) / 1e9
        peak, unit, bound = float(pk.get("hbm_gbs", 6800.0)), "GB/s", "hbm"
    elif dom == 1:
        flops_per_step = 14.0 * st.pairs3 * frames * info.n_s3
        achieved = flops_per_step * args.steps / (stage_ms[1] / 1e3) / 1e12
        peak, unit, bound = fp32_peak_tflops(nsm, pk), "TFLOP/s", "alu"
    else:
        # several channels: 40 flop per point and frame (five complex multiply-adds)
        flops_per_step = (10.0 if C == 1 else 40.0) * st.pairs4 * frames * info.n_s4
        achieved = flops_per_step * args.steps / (stage_ms[2] / 1e3) / 1e12
        peak, unit, bound = fp32_peak_tflops(nsm, pk), "TFLOP/s", "alu"
    roofline = {"bound": bound, "kernel": names[dom], "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak, "traffic": traffic_for(names[dom]),
                "peak_source": ("measured (MEASURED_PEAKS.json)" if bound == "hbm" else
                                "derived: SMs x 128 FP32 lanes x 2 flop x max SM clock"),
                "stage_ms_per_step": {nm: float(stage_ms[i] / args.steps)
                                      for i, nm in enumerate(names[:4])},
                "launch_ms": float(stage_ms[dom] / max(1, launches))}
    gpu_launches = int(args.steps * (n_batches * info.kernels_per_batch + 3))

    # ---- the S4 stage against its own bound: the tensor pipe in the split modes
    # (useful products of the Gram contraction, K = m(m+1)/2 per grid point and
    # group, times the hi/lo passes), the FP32 pipe otherwise
    s4_ms = stage_ms[2] / args.steps
    if args.precision == "fp32" or C > 1:
        s4_flops = (10.0 if C == 1 else 40.0) * st.pairs4 * frames * info.n_s4
        s4_peak, s4_unit, s4_bound = fp32_peak_tflops(nsm, pk), "TFLOP/s", "alu"
        s4_src = "derived: SMs x 128 FP32 lanes x 2 flop x max SM clock"
    else:
        passes = 1 if args.precision == "bf16" else 3
        s4_flops = float(st.pairs4) * groups * m * (m + 1) * passes
        bf16_peak = float(pk.get("bf16_tflops", 1900.0))
        if args.precision == "tf32x3":
            s4_peak = bf16_peak * 1.1 / 2.25
            s4_src = "measured bf16 x nominal tf32/bf16 dense ratio (1.1/2.25 PFLOP/s)"
        else:
            s4_peak, s4_src = bf16_peak, "measured (MEASURED_PEAKS.json, bf16 burst)"
        s4_unit, s4_bound = "TFLOP/s", "tensor"
    # ---- K1 against HBM: algorithmic bytes = samples in (4 B), centred spectra out
    # (8 B per bin and frame, bins padded to a multiple of 16) and, in the split
    # modes, the operand image (hi and lo of ceil(m/16) + ceil(m(m-1)/2 / 16) chunks of
    # 16 products per bin, TF32 4 B, BF16 2 B each part) and the ps values (4 B per bin)
    Mp = ((T // 2 + 1) + 15) // 16 * 16
    k1_bytes = groups * (m * T * z.itemsize * C + m * Mp * 8 * C)
    if args.precision != "fp32" and C == 1:
        nkc = (m + 15) // 16 + (m * (m - 1) // 2 + 15) // 16
        k1_bytes += groups * C * Mp * (nkc * 16 * 2 * (4 if args.precision == "tf32x3" else 2) + 4)
    k1_ms = stage_ms[0] / args.steps
    k1_ach = k1_bytes / (k1_ms / 1e3) / 1e9 if k1_ms > 0 else None
    roofline_k1 = {"bound": "hbm", "kernel": "k1_spectra", "achieved": k1_ach,
                   "peak": float(pk.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                   "frac": (k1_ach / float(pk.get("hbm_gbs", 6800.0))) if k1_ach else None,
                   "traffic": (traffic_for("k1_spectra_" + args.precision) if C == 1
                               else None),
                   "traffic_note": "DRAM bytes per launch (ncu); a step is "
                                   f"{n_batches} launches",
                   "algorithmic_bytes_per_step": k1_bytes,
                   "peak_source": "measured (MEASURED_PEAKS.json)", "ms_per_step": k1_ms}
    s4_ach = s4_flops / (s4_ms / 1e3) / 1e12 if s4_ms > 0 else None
    roofline_s4 = {"bound": s4_bound, "kernel": s4_name, "achieved": s4_ach,
                   "peak": s4_peak, "unit": s4_unit,
                   "frac": (s4_ach / s4_peak) if s4_ach else None,
                   "traffic": traffic_for("k3_trispec_tc" if args.precision != "fp32" and C == 1
                                          else s4_name),
                   "peak_source": s4_src, "ms_per_step": s4_ms}

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
            P.ss_finalize(plan.handle, host_out["S2"], host_out["S3"], host_out["S4"],
                          host_err["S2"], host_err["S3"], host_err["S4"])

        for _ in range(2):
            step_host()
        barrier()
        h0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        barrier()
        he = time.perf_counter() - h0
        if dist is not None:
            t = torch.tensor([he], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            he = float(t.item())
        d2h = sum(v.nbytes for v in host_out.values()) + sum(v.nbytes for v in host_err.values())
        e2e = {"value": world * C * n * args.steps / he, "unit": "samples/s",
               "h2d_bytes_per_step": int(z.nbytes), "d2h_bytes_per_step": int(d2h)}

    cpu, err_fp64 = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cg = w.get("cpu_groups", args.cpu_groups)
        cpu, ref = cpu_baseline(w, z, cg, plan.combos())
        err_fp64 = error_vs_oracle(P, w, z, ref, cg, args.precision)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "channels": C, "samples_per_rank": n, "T": T,
                       "M": T // 2 + 1, "m": m, "groups": groups, "window": "hann",
                       "orders": "S2+S3+S4 full grids",
                       "s4_precision": args.precision if C == 1 else "fp32 (several channels)",
                       "dtype_in": w.get("dtype", "f32"),
                       "l2": f"record of {z.nbytes / 2**30:.0f} GiB per step is larger than L2; "
                             "no flush"},
            "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roofline,
            "roofline_s4": roofline_s4, "roofline_k1": roofline_k1, "err_vs_fp64": err_fp64,
            "cpu_baseline": cpu, "clocks": clock_info,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
