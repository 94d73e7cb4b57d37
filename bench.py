#!/usr/bin/env python3
"""FDAS f-z plane throughput on GB300.

One step = one pass of the whole hot path over one series: the long real FFT, the
overlap-save plane (segment FFTs, per-template multiply, inverse FFT, |.|^2, overlap
discard), harmonic sums (1..16 harmonics) and the peak list; the template bank is built once
at plan time.  Workload: N = 2^23 samples at 64 us of seeded Gaussian noise with 8 injected
accelerated pulse trains, 85 templates (zmax 84), 256 taps, 8192-bin segments.

  python bench.py [--gpus N] [--steps K] [--warmup W]
                  [--precision fp32|bf16|bf16_split|fp16_scaled|bf16_direct|fp8_direct]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Beside the plane metric, the line carries "refine": sub-bin refinement of 100k candidates seeded
within half a bin of the injected harmonics of a series like the one above (20 FP32 gradient
steps and a final FP64 step per candidate), in candidates/s, with the oracle's own ascent timed
on a sample of the same candidates; and "batch": 256 dispersion-trial series of uneven length
(2^21 .. 2^23) and zmax (20, 50, 84) searched with 16-harmonic sums as one graph-launched BF16
batch, in cells/s, beside the same series searched one by one on the FP32 path.

Prints one JSON line (rank 0).  Multi-GPU: one process per GPU (torchrun), each searching
its own series (dispersion trials are independent: weak scaling, no data-path collective);
the timed region is bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "f-z plane cells/s, BF16 vs FP32 path on 1 GB300 at <=3% peak-power error"
UNIT = "cells/s"
# noise false-alarm ~1 per level on this plane: chi^2 with 2H dof isf(1/cells_H)
THRESHOLDS = (40.0, 44.0, 51.0, 64.0, 88.0)
MAX_HARM = 16
MAX_PEAKS = 16384
SM_COUNT = 152
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:        # fallback figures for GB300 when the measured file is absent
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


MEASURED = _measured_peaks()


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("own", "reference"), default="own")
    ap.add_argument("--precision", choices=("auto", "fp32", "bf16", "bf16_split", "fp16_scaled", "bf16_direct",
                                           "fp8_direct"),
                    default="auto")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the other-precision comparison runs")
    ap.add_argument("--quick", action="store_true", help="no clocks, e2e or CPU baseline (profiling runs)")
    ap.add_argument("--no-refine", action="store_true", help="skip the candidate-refinement measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the many-series batch measurement")
    ap.add_argument("--no-sensitivity", action="store_true", help="skip the precision sensitivity sweep")
    ap.add_argument("--sensitivity-series", type=int, default=32,
                    help="series of the sensitivity sweep (the full sweep is 2000)")
    ap.add_argument("--n-log2", type=int, default=23,
                    help="series length 2^n (23 = the benchmark workload; smaller only for profiler captures)")
    return ap.parse_args()


def workload(series_index: int = 0, n_log2: int = 23):
    import fdas_synth as synth
    w = synth.pulse_train_workload(config_index=1, series_index=series_index, n=1 << n_log2)
    w.max_harm = MAX_HARM
    w.thr = THRESHOLDS
    return w


# The FP32 path's overlap-save segment length.  The plane does not depend on it (the
# linear-correlation identity), and 2048-bin segments run fastest on GB300 (correlation kernel at
# N = 2^23, 85 templates, 256 taps: 0.93 ms against 1.31 ms with the workload's 8192).
FP32_SEG_LEN = 2048


def seg_len_run(w, precision: str):
    """The overlap-save segment length a precision actually runs (the plane does not depend on
    it): the tensor-core DFT paths always use 4096-bin segments (64 x 64), the direct forms have
    no segments, the FP32 path runs FP32_SEG_LEN."""
    if precision in ("bf16", "bf16_split", "fp16_scaled"):
        return 4096
    if precision in ("bf16_direct", "fp8_direct", "fp64-oracle"):
        return None                        # direct correlation: no segments
    return FP32_SEG_LEN


def config_json(w, precision: str):
    return {
        "workload": w.name,
        "n_samples": w.n, "tsamp_s": w.tsamp, "zmax": w.zmax, "templates": w.K, "taps": w.taps,
        "seg_len": w.seg_len, "seg_len_run": seg_len_run(w, precision),
        "max_harm": MAX_HARM, "thresholds": list(THRESHOLDS),
        "precision": precision, "cells_per_step": w.K * w.nb, "series_per_gpu": 1,
        "l2": "a 256 MiB buffer is written before every timed step (L2 is 129 MB); the plane written "
              "each step (0.71 GB BF16, 1.43 GB FP32) is also larger than L2",
    }


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while it runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to $FDAS_CLOCKS_CSV when set (to keep them), else to a temporary file
        self.path = os.environ.get("FDAS_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                       f"fdas_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ rooflines
def _peaks_file():
    return os.path.join(ROOT, "profiles", "traffic.json")


def _traffic(kernel: str, precision: str, workload: str):
    """Per-launch DRAM bytes from a committed ncu capture, or None when there is none or the
    kernel's source has changed since it was taken."""
    import hashlib
    try:
        with open(_peaks_file()) as f:
            rec = json.load(f).get(f"{kernel}:{precision}:{workload}")
        if not rec:
            return None
        with open(os.path.join(ROOT, rec["src"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest()[:16] != rec["sha"]:
                return None
        return rec["bytes"]
    except Exception:
        return None


def roofline_correlate(w, precision: str, prof):
    """The plane kernel: FP32 CUDA-core FFT (ALU-bound) or the tensor-core DFT stages."""
    n = max(1, prof["n_timed"]["correlate"])
    ms = prof["ms"]["correlate"] / n
    if precision == "fp32":
        S = FP32_SEG_LEN
        L = (S - w.taps + 1) // 32 * 32
        n_seg = math.ceil(w.nb / L)
        flops = n_seg * w.K * (5.0 * S * math.log2(S) + 6.0 * S + 3.0 * L)
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.070 / 1e3
        ach = flops / (ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": _traffic("k3_plane_fp32", "fp32", w.name), "kernel": f"k3_plane_fp32<{S}>",
                "avg_launch_ms": ms, "flops_per_launch": flops,
                "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz (no measured FP32 figure)"}
    if precision == "bf16_direct":
        # the Hankel-matrix GEMM: 2 outputs x 2 m products x 2 flops per (bin, template)
        flops = 8.0 * w.taps * w.K * w.nb
        ach = flops / (ms / 1e3) / 1e12
        peak = MEASURED["bf16_tflops"]
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": _traffic("k3_plane_direct", precision, w.name), "kernel": "k3_plane_direct",
                "avg_launch_ms": ms, "flops_per_launch": flops,
                "peak_note": "of measured: MEASURED_PEAKS bf16_tflops (burst; the kernel runs under a millisecond)",
                "hbm_GBps_algorithmic": (w.K * w.nb * 2 + w.nb * 4) / (ms / 1e3) / 1e9}
    if precision == "fp8_direct":
        # the same GEMM with E4M3 operands: its peak is the measured BF16 one times the nominal
        # FP8 / BF16 ratio (4.5 / 2.25 PFLOP/s dense)
        flops = 8.0 * w.taps * w.K * w.nb
        ach = flops / (ms / 1e3) / 1e12
        peak = MEASURED["bf16_tflops"] * 2.0
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": _traffic("k3_plane_direct_f8", precision, w.name), "kernel": "k3_plane_direct_f8",
                "avg_launch_ms": ms, "flops_per_launch": flops,
                "peak_note": "of measured: MEASURED_PEAKS bf16_tflops x 2 (burst; nominal FP8/BF16 dense ratio)",
                "hbm_GBps_algorithmic": (w.K * w.nb * 4 + w.nb * 8) / (ms / 1e3) / 1e9}
    # tensor-core DFT paths: 4096-bin segments as a four-step 64 x 64 DFT, two real 128 x 128 x 128
    # GEMMs per (segment, template pair)
    S = 4096
    L = (S - w.taps + 1) // 64 * 64
    n_seg = math.ceil(w.nb / L)
    items = n_seg * math.ceil(w.K / 2)
    mult = 3 if precision == "bf16_split" else 1
    executed = items * 2 * (2 * 128 * 128 * 128) * mult
    cells = w.K * w.nb
    # algorithmic tensor work: the real-ified DFT-GEMM stages of the radix-32.16.16 plan of an
    # 8192-bin segment, 8 (32 + 16 + 16) S' / L' real flops per cell (S' = 8192, L' = S' - m + 1),
    # which is less than the radix-64.64 plan executes (8 (64 + 64) S / L)
    S8 = 8192
    L8 = S8 - w.taps + 1
    alg_cell = 8.0 * (32 + 16 + 16) * S8 / L8 * mult
    alg_flops = alg_cell * cells
    # algorithmic bytes: the plane stored once and the segment spectra read once (BF16 / FP16
    # pairs: 4 bytes a bin; split: hi and lo, 8 bytes); the template bank stays in L2
    plane_b = cells * (2 if precision == "bf16" else 4)
    in_b = n_seg * S * (8 if precision == "bf16_split" else 4)
    nbytes = plane_b + in_b
    s_ = ms / 1e3
    hbm_peak = MEASURED["hbm_gbs"]
    ten_peak = MEASURED["bf16_tflops"]
    kern = "k3_plane_tc_split" if precision == "bf16_split" else "k3_plane_tc"
    tensor = {"achieved": alg_flops / s_ / 1e12, "peak": ten_peak, "unit": "TFLOP/s",
              "frac": alg_flops / s_ / 1e12 / ten_peak, "flops_per_launch": alg_flops, "flops_per_cell": alg_cell,
              "executed_flops_per_launch": executed, "executed_tflops": executed / s_ / 1e12,
              "executed_frac": executed / s_ / 1e12 / ten_peak,
              "peak_note": "of measured: MEASURED_PEAKS bf16_tflops (burst: the kernel runs well under a "
                           "millisecond inside a step of under a millisecond)"}
    hbm = {"achieved": nbytes / s_ / 1e9, "peak": hbm_peak, "unit": "GB/s", "frac": nbytes / s_ / 1e9 / hbm_peak,
           "bytes_per_launch": nbytes, "peak_note": "of measured: MEASURED_PEAKS hbm_gbs (copy bandwidth)"}
    # the roof that binds is the one with the longer floor time
    if nbytes / (hbm_peak * 1e9) >= alg_flops / (ten_peak * 1e12):
        roof = {"bound": "hbm", **{k: hbm[k] for k in ("achieved", "peak", "unit", "frac")}}
        roof.update(bytes_per_launch=nbytes, peak_note=hbm["peak_note"], tensor=tensor)
    else:
        roof = {"bound": "tensor", **{k: tensor[k] for k in ("achieved", "peak", "unit", "frac")}}
        roof.update(flops_per_launch=alg_flops, peak_note=tensor["peak_note"], hbm=hbm,
                    executed_flops_per_launch=executed)
    roof.update(traffic=_traffic(kern, precision, w.name), kernel=kern, avg_launch_ms=ms,
                floor_ms={"hbm": 1e3 * nbytes / (hbm_peak * 1e9), "tensor": 1e3 * alg_flops / (ten_peak * 1e12)})
    return roof


def _gathers(w, levels):
    """New harmonic terms read for the given harmonic levels: level H (H = 2^l) adds harmonics
    H/2 + 1 .. H for each cell of its region (|H z| <= zmax, H r < Nb)."""
    g = 0
    for l in levels:
        H = 1 << l
        zl = (w.zmax // H) // 2 * 2
        g += (zl + 1) * (w.nb // H) * (H // 2)
    return g


def roofline_peak_kernel(w, precision: str, kernel: str, prof):
    """HBM roofline of one of the two peak-search kernels: k4_level1 reads the plane once;
    k4_levels reads level 2's region of the plane (S_1) and every new harmonic term once."""
    rec = prof["peaks_kernels"][kernel]
    ms = rec["ms"] / max(1, rec["n_timed"])
    eb = 2 if precision in ("bf16", "bf16_direct") else 4
    if kernel == "k4_level1":
        nbytes = w.K * w.nb * eb
    elif kernel == "k4_level1_marked":
        # the unit marks read and the level-1 counts written (the marked units' few cells aside)
        nbytes = w.K * (w.nb // 512) * (1 + 4)
    else:
        zl = (w.zmax // 2) // 2 * 2
        nbytes = ((zl + 1) * (w.nb // 2) + _gathers(w, range(1, 5))) * eb
    ach = nbytes / (ms / 1e3) / 1e9
    peak = MEASURED["hbm_gbs"]
    # the level search runs as k4_levels_ordered (level 2's blocks in ray order)
    kname = "k4_levels_ordered" if kernel == "k4_levels" else kernel
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": _traffic(kname, precision, w.name), "kernel": kname, "avg_launch_ms": ms,
            "bytes_per_launch": nbytes, "peak_note": "of measured: MEASURED_PEAKS hbm_gbs (copy bandwidth)"}


def roofline_stage(w, precision: str, stage: str, prof):
    """HBM roofline of a bandwidth-shaped stage (peak search or the long FFT)."""
    n = max(1, prof["n_timed"][stage])
    ms = prof["ms"][stage] / n
    eb = 2 if precision in ("bf16", "bf16_direct") else 4
    if stage == "peaks":
        # the plane once, plus the H/2 new harmonic terms per cell of each level 2..16
        nbytes = (w.K * w.nb + _gathers(w, range(1, 5))) * eb
        kern = "k4_level1+k4_levels"
    else:
        nbytes = 6 * 8 * (w.nb)                                 # three passes, complex64 in and out
        kern = "k1_spectrum"
    ach = nbytes / (ms / 1e3) / 1e9
    peak = MEASURED["hbm_gbs"]
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": _traffic(kern, precision, w.name), "kernel": kern, "avg_launch_ms": ms, "bytes_per_launch": nbytes,
            "peak_note": "of measured: MEASURED_PEAKS hbm_gbs (copy bandwidth)"}


# ------------------------------------------------------------------------------ oracle timing
def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86 "model name"; Arm implementer and part)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return "unknown"
    for line in info.splitlines():
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "CPU implementer" in fields:
        return f"Arm implementer {fields['CPU implementer']} part {fields.get('CPU part', '?')}"
    return "unknown"


def oracle_sample(w, rows_bins: int = 1 << 15):
    """Time the FP64 oracle on one whole step of the workload: the full-length spectrum, the
    whole plane by direct correlation (all templates, every bin) and the harmonic sums + peaks of
    that plane.  A slice of `rows_bins` bins is timed first and its per-cell cost extrapolated to
    the whole plane, so that the line states how far that extrapolation (the reference arm's
    sampling) lands from the measured full step."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    xhat, _ = oracle.spectrum(w.series)
    t_spec = time.perf_counter() - t0
    T, _ = oracle.templates(w.zmax, w.taps)
    zi = np.repeat(np.arange(w.K, dtype=np.int32), rows_bins)
    r = np.tile(np.arange(rows_bins, dtype=np.int64), w.K)
    t0 = time.perf_counter()
    cells = oracle.plane_cells(xhat, w.zmax, w.taps, T, zi, r).reshape(w.K, rows_bins)
    oracle.peaks_f64(cells, w.zmax, MAX_HARM, THRESHOLDS)
    t_slice = time.perf_counter() - t0
    del cells
    full_cells = w.K * w.nb
    t_extrap = t_spec + t_slice * full_cells / (w.K * rows_bins)
    t0 = time.perf_counter()
    plane = oracle.plane(xhat, w.zmax, w.taps, T)
    t_plane = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.peaks_f64(plane, w.zmax, MAX_HARM, THRESHOLDS)
    t_peaks = time.perf_counter() - t0
    del plane
    t_full = t_spec + t_plane + t_peaks
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {
        "value": full_cells / t_full, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
        "sample": (f"FP64 oracle, one whole step: {w.n}-sample spectrum ({t_spec:.2f} s), direct correlation of "
                   f"all {full_cells} cells ({t_plane:.2f} s), harmonic sums and peaks ({t_peaks:.2f} s); a "
                   f"{w.K} x {rows_bins}-bin slice extrapolated per cell gives {t_extrap:.2f} s "
                   f"({100.0 * (t_extrap / t_full - 1.0):+.1f} % of the measured step)"),
        "ms_full_step": 1e3 * t_full,
        "ms_extrapolated_from_slice": 1e3 * t_extrap,
    }


def reference_arm(args, budget_s: float = 60.0):
    """The FP64 oracle as it stands, on the host cores, on this arm's workload and metric.
    Every warm-up and timed step is a bounded sample of one step of the workload: the direct
    correlation, harmonic sums and peaks of all templates over a slice of bins (a different
    slice each step), plus that slice's share of the full-length spectrum (timed once).  The
    slice is sized from a calibration so that all steps together take about budget_s; the line's
    ms_per_step is the measured time of one such sampled step and value its cells per second."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.build()
    w = workload(0, args.n_log2)
    t0 = time.perf_counter()
    xhat, _ = oracle.spectrum(w.series)
    t_spec = time.perf_counter() - t0
    T, _ = oracle.templates(w.zmax, w.taps)

    def slice_time(bins: int, r0: int) -> float:
        zi = np.repeat(np.arange(w.K, dtype=np.int32), bins)
        r = np.tile(np.arange(r0, r0 + bins, dtype=np.int64), w.K)
        t = time.perf_counter()
        cells = oracle.plane_cells(xhat, w.zmax, w.taps, T, zi, r).reshape(w.K, bins)
        oracle.peaks_f64(cells, w.zmax, MAX_HARM, THRESHOLDS)
        return time.perf_counter() - t

    calib = 1024
    rate = w.K * calib / max(slice_time(calib, 0), 1e-6)
    n_total = max(1, args.steps + args.warmup)
    bins = int(budget_s / n_total * rate / w.K)
    bins = max(256, min(1 << 15, w.nb, bins // 256 * 256))
    ms = []
    for k in range(n_total):
        r0 = (k * bins) % max(1, w.nb - bins)
        t_step = slice_time(bins, r0) + t_spec * bins / w.nb
        if k >= args.warmup:
            ms.append(1e3 * t_step)
    ms_step = statistics.mean(ms)
    value = w.K * bins / (ms_step / 1e3)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"FP64 oracle: each step the direct correlation + harmonic sums + peaks of {w.K} templates x "
              f"{bins} bins ({w.K * bins} of the step's {w.K * w.nb} cells) plus that share of the "
              f"{w.n}-sample spectrum ({t_spec:.2f} s whole, timed once); ms_per_step is one such "
              f"sampled step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_json(w, "fp64-oracle"),
        "cells_per_sampled_step": w.K * bins,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------ refinement
REFINE_STEPS = 20


def refine_peak_split(wl, pts, P):
    """Per truth, the seeds end on the local maxima of that truth's noise realisation.  A truth
    has a dominant peak when at least half its seeds end on its highest maximum; candidates on a
    dominant peak are scored with the joint (Mahalanobis) distance to the truth in Cramer-Rao
    units, chi^2 with 2 degrees of freedom at the bound (the (r, z) errors correlate at -0.968, so
    separate per-axis 3-sigma boxes misjudge points along the degenerate direction)."""
    import numpy as np
    cov = np.array([[48.0, -90.0], [-90.0, 180.0]]) / math.pi ** 2
    on = np.zeros(pts.shape[0], dtype=bool)
    lost = 0
    for t in range(wl.truths.shape[0]):
        sel = np.flatnonzero(wl.truth_index == t)
        top = pts[sel[np.argmax(P[sel])]]
        hit = np.all(np.abs(pts[sel] - top) <= [0.01, 0.02], axis=1)
        if hit.mean() >= 0.5:
            on[sel[hit]] = True
        else:
            lost += 1
    delta = pts - wl.truths[wl.truth_index, :2]
    d2 = np.einsum("ni,ij,nj->n", delta, np.linalg.inv(cov), delta) * P
    return {"on_dominant_peak_fraction": float(on.mean()), "truths_without_dominant_peak": lost,
            "mean_mahalanobis_d2_on_dominant_peaks": float(d2[on].mean()),
            "joint_3sigma_coverage_on_dominant_peaks": float(np.mean(d2[on] <= 11.829))}


def refine_bench(dev, stream, reps: int = 10, warmup: int = 3, cpu_sample: int = 32, cpu: bool = True):
    """Candidate refinement (fdas_refine) on the differentiation workload: the spectrum of the
    series comes from fdas_spectrum; each timed launch refines all candidates; L2 is flushed
    before each.  Accuracy is scored against the injected truths in Cramer-Rao units
    (Var(r, z) = (1/(pi^2 P)) [[48, -90], [-90, 180]] at peak power P, noise mean 2)."""
    import numpy as np
    import torch

    import fdas_synth as synth
    import paper_2206_12205_gb300 as fd

    wl = synth.refine_workload()
    sw = wl.series
    plan = fd.fdas_plan(fd.make_config(sw.n, sw.zmax, sw.taps, sw.seg_len))
    fd.fdas_make_templates(plan, stream)
    ws = torch.empty(plan.info.workspace_bytes, dtype=torch.uint8, device=dev)
    xdev = torch.empty(2 * plan.info.nb, dtype=torch.float32, device=dev)
    fd.fdas_spectrum(plan, torch.from_numpy(sw.series).to(dev), ws, xdev, None, stream)
    seeds = torch.tensor(wl.seeds, dtype=torch.float64, device=dev)
    ncand = int(seeds.shape[0])
    out = torch.empty_like(seeds)
    pw = torch.empty(ncand, 3, dtype=torch.float64, device=dev)
    ev = torch.empty(ncand, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed(steps: int) -> float:
        for _ in range(warmup):
            fd.fdas_refine(plan, xdev, seeds, steps, out, pw, ev, stream)
        ms = []
        for k in range(reps):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fd.fdas_refine(plan, xdev, seeds, steps, out, pw, ev, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    ms_fp64_only = timed(0)
    ms_full = timed(REFINE_STEPS)
    pts, P, evals = out.cpu().numpy(), pw[:, 0].cpu().numpy(), ev.cpu().numpy()
    truth = wl.truths[wl.truth_index, :2]
    sr, sz = np.sqrt(48.0 / (math.pi ** 2 * P)), np.sqrt(180.0 / (math.pi ** 2 * P))
    nr, nz = (pts[:, 0] - truth[:, 0]) / sr, (pts[:, 1] - truth[:, 1]) / sz
    res = {
        "metric": "refined candidates/s (20 FP32 gradient steps + 1 FP64 step each)",
        "value": ncand / (ms_full / 1e3), "unit": "candidates/s", "candidates": ncand,
        "ms_per_launch": ms_full, "ms_final_fp64_step_only": ms_fp64_only,
        "power_evaluations_mean": float(evals.mean()),
        "workload": f"{sw.name}: {wl.truths.shape[0]} injected harmonics with expected P >= 30, "
                    f"seeds within half a bin (uniform) in r and z",
        "vs_truth": {"median_abs_dr": float(np.median(np.abs(pts[:, 0] - truth[:, 0]))),
                     "median_abs_dz": float(np.median(np.abs(pts[:, 1] - truth[:, 1]))),
                     "crb_rms_r": float(np.sqrt(np.mean(nr ** 2))), "crb_rms_z": float(np.sqrt(np.mean(nz ** 2))),
                     "within_3_crb_sigma": float(np.mean((np.abs(nr) <= 3) & (np.abs(nz) <= 3))),
                     **refine_peak_split(wl, pts, P)},
        "gpu_launches_per_step": 1,
    }
    if cpu:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        xh, _ = oracle.spectrum(sw.series)
        t_spec = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.refine(xh, sw.taps, wl.seeds[:cpu_sample], REFINE_STEPS + 1)
        t_ref = time.perf_counter() - t0
        per = t_ref / cpu_sample
        res["cpu_baseline"] = {
            "value": ncand / (t_spec + per * ncand), "unit": "candidates/s", "kind": "oracle",
            "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "sample": (f"FP64 oracle: {sw.n}-sample spectrum ({t_spec:.2f} s) + FP64 ascent of {cpu_sample} of the "
                       f"candidates ({t_ref:.2f} s, threaded over candidates), extrapolated to {ncand}")}
    fd.fdas_destroy(plan)
    return res


# ------------------------------------------------------------------------------ batch of series
BATCH_SERIES = 256


def batch_bench(dev, stream, reps: int = 5, warmup: int = 2, loop_reps: int = 2, lanes=(1, 2, 3, 4)):
    """The batching workload: one fdas_batch_search (a captured graph) over all series, BF16, at
    1 .. 4 concurrent lanes, against per-series loops of fdas_search calls (one plan per distinct
    series shape) in BF16 and in FP32.  The packed series (about 4.8 GB) stay on the device; each
    pass streams far more than L2."""
    import numpy as np
    import torch

    import fdas_synth as synth
    import paper_2206_12205_gb300 as fd
    from paper_2206_12205_gb300 import batch as fbat

    t0 = time.perf_counter()
    wl = synth.batch_workload(n_series=BATCH_SERIES, workers=min(16, os.cpu_count() or 1))
    t_gen = time.perf_counter() - t0
    packed = torch.from_numpy(wl.packed).to(dev)
    cells = wl.total_cells

    def cfg(w, prec, seg=None):
        return fd.make_config(w.n, w.zmax, w.taps, seg or w.seg_len, precision=prec, max_harm=MAX_HARM,
                              thr=THRESHOLDS, max_peaks=4096)

    def timed(fn, n_warm, n_rep):
        for _ in range(n_warm):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(n_rep):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    by_lanes = {}
    npk = None
    for nl in lanes:
        bs = fbat.BatchSearch([cfg(w, "bf16") for w in wl.series], device=dev, stream=stream, lanes=nl)
        by_lanes[nl] = timed(lambda: bs.search(packed, stream), warmup, reps)
        n_ = int(bs.npeaks.sum().item())
        assert npk is None or n_ == npk
        npk = n_
        assert fd.fdas_batch_device_status(bs.batch) == 0
        del bs
    best_lanes = min(by_lanes, key=by_lanes.get)
    ms_batch = by_lanes[best_lanes]

    views = [packed[int(o): int(o) + w.n] for o, w in zip(wl.offsets, wl.series)]

    def loop_ms(prec, seg=None):
        searches = {}
        for w in wl.series:
            key = (w.n, w.zmax, w.taps)
            if key not in searches:
                searches[key] = fd.Search(cfg(w, prec, seg), device=dev, stream=stream)

        def run():
            for w, x in zip(wl.series, views):
                searches[(w.n, w.zmax, w.taps)].search(x, stream)
        out = timed(run, 1, loop_reps)
        del searches
        return out

    ms_bf16_loop = loop_ms("bf16")
    ms_fp32 = loop_ms("fp32", FP32_SEG_LEN)
    del packed
    shapes = sorted({(w.n, w.zmax) for w in wl.series})
    return {
        "metric": "f-z plane cells/s over a batch of series (BF16, one graph launch per batch)",
        "value": cells / (ms_batch / 1e3), "unit": "cells/s", "series": BATCH_SERIES, "cells": cells,
        "ms_per_batch": ms_batch, "lanes": best_lanes, "peaks_found": npk, "gpu_launches_per_batch": 8 * BATCH_SERIES,
        "by_lanes": {str(k): {"value": cells / (v / 1e3), "ms_per_batch": v} for k, v in by_lanes.items()},
        "bf16_loop": {"value": cells / (ms_bf16_loop / 1e3), "unit": "cells/s", "ms_per_batch": ms_bf16_loop,
                      "how": "fdas_search per series from Python, BF16 path, one plan per series shape"},
        "fp32_loop": {"value": cells / (ms_fp32 / 1e3), "unit": "cells/s", "ms_per_batch": ms_fp32,
                      "how": f"fdas_search per series from Python, FP32 path ({FP32_SEG_LEN}-bin segments), "
                             "one plan per series shape"},
        "speedup_vs_bf16_loop": ms_bf16_loop / ms_batch,
        "speedup_vs_fp32_loop": ms_fp32 / ms_batch,
        "workload": (f"{BATCH_SERIES} series, N in {{2^21, 2^22, 2^23}}, zmax in {{20, 50, 84}} (taps 64/128/256), "
                     f"0-2 pulse trains each, {len(shapes)} distinct shapes; synthesised in {t_gen:.1f} s"),
        "l2": "each batch streams about 4.8 GB of series and 33 G cells of planes through HBM (L2 is 129 MB)",
    }


def sharded_batch_bench(dev, stream, dist, rank: int, world: int, reps: int = 5, warmup: int = 2, lanes: int = 3):
    """The batching workload split over the job's GPUs: series dealt by shard_series (largest cost
    first, each to the least loaded rank), each rank synthesising and searching only its share as
    one batch (no exchange during the search), timed between barriers, the max over ranks; then
    the per-series peak lists gathered on rank 0 (the only data that travels)."""
    import torch

    import fdas_synth as synth
    import paper_2206_12205_gb300 as fd
    from paper_2206_12205_gb300 import batch as fbat

    shapes = synth._batch_shapes(2, BATCH_SERIES, synth.BATCH_N, synth.BATCH_ZMAX)
    mine = fbat.shard_series([fbat.series_cost(n, z) for n, z in shapes], world)[rank]
    wl = synth.batch_workload(n_series=BATCH_SERIES, series=mine, workers=min(16, os.cpu_count() or 1))
    packed = torch.from_numpy(wl.packed).to(dev)
    cfgs = [fd.make_config(w.n, w.zmax, w.taps, w.seg_len, precision="bf16", max_harm=MAX_HARM, thr=THRESHOLDS,
                           max_peaks=4096) for w in wl.series]
    bs = fbat.BatchSearch(cfgs, device=dev, stream=stream, lanes=lanes)
    for _ in range(warmup):
        bs.search(packed, stream)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        dist.barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bs.search(packed, stream)
        b.record(stream)
        torch.cuda.synchronize()
        t = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms.append(float(t.item()))
    ms_batch = statistics.median(ms)
    assert fd.fdas_batch_device_status(bs.batch) == 0
    lists = fbat.gather_peak_lists(mine, bs.peak_lists(), BATCH_SERIES, dist)
    cells = [None] * world
    dist.all_gather_object(cells, wl.total_cells)
    del bs, packed
    if rank != 0:
        return None
    total = sum(cells)
    return {
        "metric": "f-z plane cells/s over a batch of series split across GPUs (BF16)",
        "value": total / (ms_batch / 1e3), "unit": "cells/s", "series": BATCH_SERIES, "cells": total,
        "ms_per_batch": ms_batch, "lanes": lanes, "scaling": "strong",
        "cells_per_rank": cells, "peaks_gathered": int(sum(len(x) for x in lists)),
        "how": "series split by batch.shard_series (no data-path collective); per-rank batch timed between "
               "barriers, max over ranks; peak lists gathered on rank 0 with gather_object",
    }


# ------------------------------------------------------------------------------ sensitivity sweep
SENS_FORMS = ("fp32", "bf16", "bf16_split", "fp16_scaled", "bf16_direct", "fp8_direct")
SENS_BANDS = 8


def sensitivity_bench(dev, stream, n_series: int):
    """The sensitivity workload (one binary pulsar per series, N = 2^23) in every precision form:
    band peaks of the fundamental and harmonics (Table harm_bounds) compared with FP32's, the
    noise canopy from noise-only planes, and each form's search throughput."""
    import numpy as np
    import torch

    import fdas_synth as synth
    import paper_2206_12205_gb300 as fd
    from paper_2206_12205_gb300 import sensitivity as se

    base = synth.sensitivity_workload(series_index=0)
    cfgs = {f: fd.make_config(base.n, base.zmax, base.taps, base.seg_len, precision=f, max_harm=MAX_HARM,
                              thr=THRESHOLDS, max_peaks=MAX_PEAKS) for f in SENS_FORMS}
    searches = {f: fd.Search(c, device=dev, stream=stream) for f, c in cfgs.items()}
    rows = {f: [] for f in SENS_FORMS[1:]}
    ms = {f: [] for f in SENS_FORMS}
    widths = []
    t0 = time.perf_counter()
    for sidx in range(n_series):
        w = base if sidx == 0 else synth.sensitivity_workload(series_index=sidx)
        f_bins = w.trains[0].r0
        widths.append(1.5 * f_bins)
        lo, hi = se.harmonic_bands(f_bins, SENS_BANDS, w.nb)
        x = torch.from_numpy(w.series).to(dev)
        peaks = {}
        for f in SENS_FORMS:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            searches[f].search(x, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms[f].append(a.elapsed_time(b))
            peaks[f] = se.band_peaks(searches[f].plan, searches[f].plane_2d(), lo, hi)
        for f in SENS_FORMS[1:]:
            rows[f].append(se.compare(peaks["fp32"], peaks[f]))
    t_sweep = time.perf_counter() - t0
    # noise canopy: noise-only FP32 planes, bands as wide as 1.5 f of each series' pulsar
    rng = np.random.default_rng(7)
    lo_c, hi_c = [], []
    for k in range(2):
        xn = torch.from_numpy(synth.noise(base.n, synth.rng_for(4, 10_000 + k)).astype(np.float32)).to(dev)
        searches["fp32"].search(xn, stream)
        torch.cuda.synchronize()
        a_, b_ = se.noise_canopy(searches["fp32"].plan, searches["fp32"].plane_2d(), widths, rng)
        lo_c.append(a_)
        hi_c.append(b_)
    canopy = (float(min(lo_c)), float(max(hi_c)))
    cells = base.K * base.nb
    out = {
        "workload": (f"{n_series} of the 2000 sensitivity series (N = 2^23, one pulsar each: P 1-20 ms, "
                     f"+-200 m/s^2, duty 2-10 %, SNR 3-40), bands 0..{SENS_BANDS - 1}; host time {t_sweep:.1f} s"),
        "noise_canopy_snr": {"min": canopy[0], "max": canopy[1]},
        "forms": {},
    }
    for f in SENS_FORMS:
        rec = {"cells_per_s": cells / (statistics.median(ms[f]) / 1e3), "ms_per_series": statistics.median(ms[f])}
        if f != "fp32":
            rec.update(se.summarise(rows[f], canopy_hi_snr=canopy[1]))
        out["forms"][f] = rec
    del searches
    return out


# ------------------------------------------------------------------------------ own arm
def own_arm(args):
    import numpy as np
    import torch

    import paper_2206_12205_gb300 as fd

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    fd.load(build_if_missing=True)

    precision = args.precision
    if precision == "auto":
        precision = "fp32"
        try:
            fd.fdas_destroy(fd.fdas_plan(fd.make_config(1 << 12, 4, 16, 1024, precision="bf16")))
            precision = "bf16"
        except fd.FdasError:
            pass

    w = workload(rank, args.n_log2)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    x_host = torch.from_numpy(w.series).pin_memory()
    x_dev = x_host.to(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed_run(prec: str, steps: int, warmup: int, sample_clocks: bool, **variant):
        """Exactly `steps` timed searches, L2 flushed before each, CUDA events per step."""
        cfg_ = fd.make_config(w.n, w.zmax, w.taps, seg_len_run(w, prec) or w.seg_len, precision=prec, max_harm=MAX_HARM,
                              thr=THRESHOLDS, max_peaks=MAX_PEAKS, **variant)
        s_ = fd.Search(cfg_, device=dev)
        for _ in range(warmup):
            s_.search(x_dev, stream)
        torch.cuda.synchronize()
        clocks_ = ClockSampler(local) if sample_clocks else None
        fd.fdas_profile_read(s_.plan, reset=True)        # launch counts of the timed steps only
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if clocks_:
            clocks_.start()
            time.sleep(0.3)
        barrier()
        torch.cuda.synchronize()
        for k in range(steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            s_.search(x_dev, stream)
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier()
        clk_ = clocks_.stop() if clocks_ else None
        launches_ = fd.fdas_profile_read(s_.plan, reset=True)["launches"]
        # the per-stage split comes from separate steps with the library's CUDA events on (the
        # timed steps above run without them)
        fd.fdas_profile_enable(s_.plan, True)
        p_steps = min(steps, 50)
        for k in range(p_steps):
            flush.fill_(k & 0xFF)
            s_.search(x_dev, stream)
        torch.cuda.synchronize()
        prof_ = fd.fdas_profile_read(s_.plan, reset=True)
        fd.fdas_profile_enable(s_.plan, False)
        prof_["launches"] = launches_
        prof_["profiled_steps"] = p_steps
        if prof_.get("level1_fused"):
            # level 1 visited only the units the plane kernel marked: its timed kernel is that one
            pk_ = prof_["peaks_kernels"]
            prof_["peaks_kernels"] = {("k4_level1_marked" if k == "k4_level1" else k): v for k, v in pk_.items()}
        tot = sum(a_.elapsed_time(b_) for a_, b_ in zip(starts, ends))
        t_ = torch.tensor([tot], dtype=torch.float64, device=dev)
        if dist is not None:
            dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        return s_, float(t_.item()), prof_, clk_

    s, total_ms, prof, clk = timed_run(precision, args.steps, args.warmup, not args.quick)
    cells = w.K * w.nb
    value = world * cells * args.steps / (total_ms / 1e3)

    # ---- end to end through the public API: pinned host series in, peak list out
    e2e = None
    if not args.no_e2e and not args.quick:
        # a stream of series: step k's host->device copy (copy stream, into one of two device
        # buffers) overlaps step k-1's search; every step copies its series in and its peak count
        # and list out inside the timed region.  The outputs are double-buffered too (fdas_search
        # into one of two peak buffers), so the read-back runs on a stream of its own while the
        # next series is copied in and searched; a search waits only for the read-back of the
        # buffer it reuses (two steps back).
        peaks_host = torch.empty(16 * MAX_PEAKS, dtype=torch.uint8).pin_memory()
        npk_host = torch.empty(1, dtype=torch.int32).pin_memory()
        e_steps = max(1, min(args.steps, 100))
        x_buf = [torch.empty_like(x_dev), torch.empty_like(x_dev)]
        pk_buf = [s.peaks, torch.empty_like(s.peaks)]
        np_buf = [s.npeaks, torch.empty_like(s.npeaks)]
        copy_stream = torch.cuda.Stream(dev)
        back_stream = torch.cuda.Stream(dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        consumed = [torch.cuda.Event(), torch.cuda.Event()]
        searched = [torch.cuda.Event(), torch.cuda.Event()]
        drained = [torch.cuda.Event(), torch.cuda.Event()]
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        a.record(stream)
        copy_stream.wait_stream(stream)
        back_stream.wait_stream(stream)
        for k in range(e_steps):
            j = k & 1
            with torch.cuda.stream(copy_stream):
                if k >= 2:
                    copy_stream.wait_event(consumed[j])           # step k-2 has read this buffer
                x_buf[j].copy_(x_host, non_blocking=True)
                copied[j].record(copy_stream)
            stream.wait_event(copied[j])
            if k >= 2:
                stream.wait_event(drained[j])                     # step k-2's outputs are read back
            fd.fdas_search(s.plan, x_buf[j], s.workspace, s.plane, pk_buf[j], np_buf[j], stream)
            consumed[j].record(stream)
            searched[j].record(stream)
            with torch.cuda.stream(back_stream):
                back_stream.wait_event(searched[j])
                npk_host.copy_(np_buf[j], non_blocking=True)
                peaks_host.copy_(pk_buf[j][: 16 * MAX_PEAKS], non_blocking=True)
                drained[j].record(back_stream)
        stream.wait_stream(copy_stream)
        stream.wait_stream(back_stream)
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device=dev)
        if dist is not None:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * cells * e_steps / (float(te.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(x_host.numel() * 4), "d2h_bytes_per_step": int(4 + 16 * MAX_PEAKS),
               "steps": e_steps, "how": "pinned host series copied in on a copy stream and each step's peak count "
               "and list copied out on another (series and outputs double-buffered, overlapping the "
               "searches), through fdas_search"}

    # ---- the other precisions on the same GPU and workload (the metric's comparison)
    paths = {}
    if not args.quick and not args.no_compare:
        for prec in ("fp32", "bf16", "bf16_split", "fp16_scaled", "bf16_direct", "fp8_direct"):
            if prec == precision:
                continue
            cmp_steps = max(3, min(args.steps, 100))
            s_c, ms_c, prof_c, _ = timed_run(prec, cmp_steps, args.warmup, False)
            paths[prec] = {"value": world * cells * cmp_steps / (ms_c / 1e3), "unit": UNIT,
                           "ms_per_step": ms_c / cmp_steps, "steps": cmp_steps,
                           "stages_ms_per_step": {k: v / prof_c["profiled_steps"] for k, v in prof_c["ms"].items()},
                           "roofline_correlate": roofline_correlate(w, prec, prof_c)}
            del s_c
        paths[precision] = {"value": value, "unit": UNIT, "ms_per_step": total_ms / args.steps}
        if "fp32" in paths and "bf16" in paths:
            paths["speedup_bf16_over_fp32"] = paths["bf16"]["value"] / paths["fp32"]["value"]

    # ---- the variants of the search (same workload, BF16): robust local normalisation and the
    # highest-harmonic-anchored harmonic sums (the direct correlation is a precision in `paths`)
    variants = None
    if not args.quick and not args.no_compare:
        variants = {}
        for name, kw in (("local_norm_4096", {"norm_block": 4096}), ("harm_anchored", {"harm_mode": 1})):
            v_steps = max(3, min(args.steps, 20))
            s_v, ms_v, prof_v, _ = timed_run("bf16", v_steps, args.warmup, False, **kw)
            variants[name] = {"config": kw, "value": world * cells * v_steps / (ms_v / 1e3), "unit": UNIT,
                              "ms_per_step": ms_v / v_steps, "steps": v_steps,
                              "stages_ms_per_step": {k: v / prof_v["profiled_steps"] for k, v in prof_v["ms"].items()},
                              "peak_kernels_ms_per_step": {k: r["ms"] / prof_v["profiled_steps"]
                                                           for k, r in prof_v["peaks_kernels"].items()}}
            del s_v

    # ---- roofline of the dominant kernel of the step (largest per-launch time): the correlation
    # kernel, one of the two peak-search kernels, or a smaller stage's kernels
    kernel_ms = {k: v / max(1, prof["n_timed"][k]) for k, v in prof["ms"].items() if k != "peaks"}
    for k, rec in prof["peaks_kernels"].items():
        if rec["n_timed"]:
            kernel_ms[k] = rec["ms"] / rec["n_timed"]
    dominant = max(kernel_ms, key=kernel_ms.get)
    roof_corr = roofline_correlate(w, precision, prof)
    if dominant == "correlate":
        roof = roof_corr
    elif dominant in ("k4_level1", "k4_level1_marked", "k4_levels"):
        roof = roofline_peak_kernel(w, precision, dominant, prof)
    else:
        roof = roofline_stage(w, precision, dominant, prof)

    refine = None
    if rank == 0 and world == 1 and not args.no_refine and not args.quick:
        refine = refine_bench(dev, stream, cpu=not args.no_cpu_baseline)
    batch = None
    if rank == 0 and world == 1 and not args.no_batch and not args.quick:
        batch = batch_bench(dev, stream)
    elif world > 1 and not args.no_batch and not args.quick:
        batch = sharded_batch_bench(dev, stream, dist, rank, world)
    sensitivity = None
    if rank == 0 and world == 1 and not args.no_sensitivity and not args.quick:
        sensitivity = sensitivity_bench(dev, stream, args.sensitivity_series)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        import oracle
        oracle.build()
        c = oracle_sample(w)
        cpu = {k: c[k] for k in ("value", "unit", "cores", "kind", "cpu_model", "sample", "ms_full_step",
                                 "ms_extrapolated_from_slice")}

    # the plane generation alone (segment FFTs + correlation, the paper's timed block), from the
    # profiled steps' events
    pg_ms = (prof["ms"]["segments"] + prof["ms"]["correlate"]) / prof["profiled_steps"]
    plane_gen = {"value": world * cells / (pg_ms / 1e3), "unit": UNIT, "ms_per_step": pg_ms,
                 "what": "K2 + K3 CUDA-event time per step (device-resident spectrum), cells per second"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16_split": "bf16-split", "fp16_scaled": "f16-scaled",
                                                    "bf16_direct": "bf16-direct", "fp8_direct": "e4m3-direct"}.get(precision, "bf16"),
            "data": "synthetic: seeded N(0,1) noise + 8 accelerated Gaussian pulse trains (fdas_synth)",
            "config": config_json(w, precision),
            "roofline": roof, "roofline_correlate": roof_corr, "paths": paths or None, "variants": variants,
            "cpu_baseline": cpu, "e2e": e2e, "refine": refine, "batch": batch, "sensitivity": sensitivity,
            "gpu_launches": int(prof["launches"]), "clocks": clk,
            "stages_ms_per_step": {k: v / prof["profiled_steps"] for k, v in prof["ms"].items()},
            "peak_kernels_ms_per_step": {k: r["ms"] / prof["profiled_steps"] for k, r in prof["peaks_kernels"].items()},
            "profiled_steps": prof["profiled_steps"],
            "plane_generation": plane_gen,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return own_arm(args)


if __name__ == "__main__":
    sys.exit(main())
