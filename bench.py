"""Benchmark: f-fdot cells/s of the FDAS correlation on GB300, with roofline and CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload survey|small|batch|zband]

A step is one fdas_convolve_power over the whole plane (segment loads, forward FFTs, template
multiplies, inverse FFTs, overlap discard and power stores: one fused kernel launch).  The
template bank is built once per plan, outside the timed region, and its time is reported
separately.  The default workload is the survey-scale plane: 2^22 bins x 201 templates
(z in [-200, 200] step 2), 512-tap templates, segment length 2048; inputs are seeded synthetic
spectra (Gaussian noise plus 16 injected chirps).

For N > 1 (torchrun) every rank runs an independent replica on its own GPU (the path has no
exchange step): value = cells of all ranks / max over ranks of the timed duration.

--impl reference times the FP64 CPU oracle (the only other implementation of this path) on the
host cores, on a bounded sample of rows of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1711_10855_gb300 import synth  # noqa: E402

METRIC = "f-fdot cells/s on 1 GB300 (2^22 bins x 201 z) and % of HBM roofline"
UNIT = "cells/s"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name: str, n_bins: int | None = None) -> synth.Workload:
    w = synth.survey() if name == "survey" else synth.small()
    if n_bins:
        # same z grid, template span and segment length on a shorter noise-only spectrum
        # (used for profiling captures, not for bench lines)
        w = synth.Workload(f"{w.name}-n{n_bins}", 2 * n_bins, w.zmax, w.zstep, w.tmpl_len, w.seg_len,
                           w.seed, ())
    return w


def algorithmic(w: synth.Workload, nseg: int, group: int = 8) -> dict:
    """Per-launch algorithmic bytes and flops of the correlation kernel, and the two co-limits:
    shared-memory bytes (each inverse transform writes and reads its L points once in the
    exchange and reads its template from the ring; each forward transform one exchange) and
    L2-to-SM template bytes (each group of `group` segments streams the whole bank once)."""
    n, Z, L, m = w.n_bins, w.n_z, w.seg_len, w.tmpl_len
    V = L - m
    bytes_plane = 4 * Z * n
    bytes_spec = 8 * nseg * L          # segments with their m-bin overlap
    bytes_tmpl = 8 * Z * L + 8 * L     # template spectra + twiddle table
    logL = int(np.log2(L))
    fft = 5 * L * logL                 # nominal complex FFT flops
    flops = nseg * Z * (fft + 6 * L + 3 * V) + nseg * fft
    smem = nseg * Z * (2 * 8 * L + 8 * L) + nseg * 2 * 8 * L
    l2_tmpl = -(-nseg // group) * Z * 8 * L
    return {"bytes": bytes_plane + bytes_spec + bytes_tmpl, "bytes_plane": bytes_plane, "flops": flops,
            "smem_bytes": smem, "l2_template_bytes": l2_tmpl}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over all ranks (the replicas' timed durations); identity at N=1."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells_per_rank: int, steps: int, world: int, t_max_s: float) -> float:
    """Whole-job cells/s of N independent replicas: all ranks' cells over the slowest rank's time."""
    return cells_per_rank * steps * world / t_max_s


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rows_rate(spec, w: synth.Workload, seconds: float, max_rows: int | None = None):
    """Time the oracle's row-streamed direct sum on whole rows of the plane, about `seconds` of
    work: returns (cells/s, rows timed, wall seconds)."""
    import oracle
    oracle.build()
    zs = list(range(w.n_z))
    rng = np.random.default_rng(5)
    rng.shuffle(zs)
    t0 = time.perf_counter()
    oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len, zs[0], zs[0] + 1)
    t_row = time.perf_counter() - t0
    rows = max(1, min(len(zs), int(seconds / max(t_row, 1e-3))))
    if max_rows:
        rows = min(rows, max_rows)
    t0 = time.perf_counter()
    for zi in zs[:rows]:
        oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len, zi, zi + 1)
    dt = time.perf_counter() - t0
    return rows * w.n_bins / dt, rows, dt


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, one bounded sample of rows per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = workload(args.workload, args.n_bins)
    spec = synth.spectrum(w)
    cores = cpu_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    rows_per_step = 1
    rng = np.random.default_rng(17)
    order = rng.permutation(w.n_z)
    for i in range(args.warmup):
        zi = int(order[i % w.n_z])
        oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len, zi, zi + 1)
    times = []
    for i in range(args.steps):
        zi = int(order[(args.warmup + i) % w.n_z])
        t0 = time.perf_counter()
        oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len, zi, zi + rows_per_step)
        times.append(time.perf_counter() - t0)
    cells = rows_per_step * w.n_bins
    value = cells * len(times) / sum(times)
    sample = f"{rows_per_step} whole row ({cells} cells) of the {w.n_z}x{w.n_bins} plane per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "n_bins": w.n_bins, "n_z": w.n_z,
                                        "seg_len": w.seg_len, "tmpl_len": w.tmpl_len},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """One persistent CUDA-graph launch over a batch of uneven spectra per step (Gaussian-noise
    time series with 0-4 injected chirps each, synthesised on the device from a seeded generator)."""
    import torch
    from paper_1711_10855_gb300 import build as fdas_build
    from paper_1711_10855_gb300 import fdas
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    fdas_build.build()
    n_bins, zmax = synth.batch_workload(args.batch_count)
    zstep, m = 2, 512
    n_z = 2 * (zmax // zstep) + 1
    specs, _ = synth.batch_spectra(torch, n_bins, zmax, m, dev)
    planes = [torch.empty((int(z), int(n)), dtype=torch.float32, device=dev) for z, n in zip(n_z, n_bins)]
    stream = torch.cuda.current_stream(dev)
    candidates = [1024, 2048, 4096]
    best, tune_ms = fdas.batch_autotune(n_bins, zmax, zstep, m, candidates, specs, planes, stream)
    b = fdas.Batch(n_bins, zmax, zstep, best, m)
    b.build_templates(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        b.convolve_power(specs, planes, use_graph=True, stream=stream)
    b.check(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record(stream)
            b.convolve_power(specs, planes, use_graph=True, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize(dev)
    b.check(stream)
    step_ms = [a.elapsed_time(c) for a, c in evs]
    ms = sum(step_ms) / len(step_ms)
    cells = int(np.sum(n_z.astype(np.int64) * n_bins))
    peaks, peak_src = measured_peaks()
    plane_bytes = 4 * cells
    # nominal flops summed over the spectra, as for the single plane (algorithmic())
    V = best - m
    logL = int(np.log2(best))
    fft = 5 * best * logL
    nseg = -(-n_bins.astype(np.int64) // V)
    flops = int(np.sum(nseg * n_z.astype(np.int64) * (fft + 6 * best + 3 * V) + nseg * fft))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT_GB300 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    alu_achieved = flops / (ms * 1e-3) / 1e12
    line = {
        "metric": "f-fdot cells/s, batched de-dispersion trials (one persistent CUDA-graph launch)",
        "value": cells / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Gaussian-noise series with 0-4 injected chirps each, synthesised on the device)",
        "config": {"workload": f"batch-{args.batch_count}-uneven", "spectra": int(args.batch_count),
                   "n_bins_min": int(n_bins.min()), "n_bins_max": int(n_bins.max()), "cells": cells,
                   "zmax_set": [100, 200], "zstep": zstep, "tmpl_len": m, "seg_len": best,
                   "autotune_candidates": candidates, "autotune_ms": tune_ms,
                   "l2": "512 MiB buffer written between timed steps"},
        "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": alu_achieved / alu_peak, "traffic": None,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (derived)",
                     "flops_per_launch": flops},
        "hbm_roofline": {"achieved": plane_bytes / (ms * 1e-3) / 1e9, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": plane_bytes / (ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"]),
                         "peak_source": f"hbm_gbs ({peak_src})", "bytes_per_launch": plane_bytes},
        # one persistent launch per step at 512 / 2048; one launch per spectrum at the other lengths
        "clocks": clk.summary(),
        "gpu_launches": args.steps * (1 if best in (512, 2048) else int(args.batch_count)),
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
    }
    # parity of this workload at full size: tests/test_gpu_batch_scale.py
    if not args.no_cpu_baseline:
        cores = cpu_cores()
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        import oracle
        i_big = int(np.argmax(n_bins))
        spec_big = specs[i_big].cpu().numpy().view(np.complex64)
        t0, rows = time.time(), 0
        while time.time() - t0 < args.cpu_seconds and rows < int(n_z[i_big]):
            oracle.plane_rows(spec_big, int(zmax[i_big]), zstep, m, rows, rows + 1)
            rows += 1
        dt = time.time() - t0
        line["cpu_baseline"] = {"value": rows * int(n_bins[i_big]) / dt, "unit": UNIT, "cores": cores,
                                "kind": "oracle",
                                "sample": f"{rows} whole rows ({rows * int(n_bins[i_big])} cells) of the largest "
                                          f"spectrum's plane, FP64 direct sum, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def choose_operating_point(points, target: float) -> dict:
    """The calibration rule: of the grid points whose recall reaches `target`, the one with the
    fewest pairs (the first on ties); without any, the highest recall (fewest pairs on ties)."""
    hits = [p for p in points if p["recall"] >= target]
    if hits:
        return min(hits, key=lambda p: p["pair_fraction"])
    return max(points, key=lambda p: (p["recall"], -p["pair_fraction"]))


def run_zband(args):
    """The learned z-band proposal path on the survey plane, measured against the full search.

    The network is first trained, untimed, on windows whose labels the full search produces.  A
    timed step is the whole proposal path through the library, on the device without a host
    synchronisation: fdas_zband_propose over the spectrum (median selection + the fused
    tensor-core inference), the pair list (fdas_zband_work_pairs, its length left on the device)
    and fdas_convolve_power_pairs_device_count over the listed (segment, template) pairs.
    value = cells of the full plane / step time (the plane the full search would compute);
    recall = the fraction of the full search's detections (block maxima >= 20 x the noise power)
    the partial plane holds.  The operating point (threshold, z halo) is calibrated, untimed, on a
    held-out spectrum (a chirp in every 16th block, SNR as in training, its own seed): the point of
    the grid with the fewest pairs whose recall there reaches --zband-recall; the survey spectrum
    and a dense spectrum of the same recipe (another seed) are then measured at that point."""
    import torch
    from paper_1711_10855_gb300 import build as fdas_build
    from paper_1711_10855_gb300 import fdas
    from paper_1711_10855_gb300 import zband as zb
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    fdas_build.build()
    t0 = time.time()
    data = zb.make_training_set(args.zband_windows, snr=tuple(args.zband_snr), snr_dist=args.zband_snr_dist)
    n_windows, n_detected = int(data.windows.shape[0]), int(data.n_detected)
    net = fdas.ZBand(zb.WINDOW, 201, 256)
    net.set_params(zb.init_params(201, seed=1))
    losses = zb.train(net, data, args.zband_steps)
    torch.cuda.synchronize(dev)
    train_s = time.time() - t0
    del data
    w = synth.survey()
    spec = torch.from_numpy(synth.spectrum(w)).to(dev)
    plan = fdas.Plan(w.n_bins, w.zmax, w.zstep, w.seg_len, w.tmpl_len)
    plan.build_templates()
    full = torch.empty((plan.n_z, w.n_bins), dtype=torch.float32, device=dev)
    part = torch.empty_like(full)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    cells = plan.n_z * w.n_bins

    def event_ms(fn, reps):
        out = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    def chirp_spectrum(seed):
        rng = np.random.default_rng(seed)
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        chirps = zb.chirp_blocks(rng, 1, w.n_bins, w.zmax, tuple(args.zband_snr), every=16,
                                 snr_dist=args.zband_snr_dist)
        return zb.chirp_spectra(torch, w.n_bins, chirps, gen, dev)[0], int(chirps["z"].shape[1])

    full_ms = event_ms(lambda: plan.convolve_power(spec, full), 5)
    plan.check()
    searches = {k: zb.ProposalSearch(net, plan, pairs=True, z_halo=k, reach_threshold=args.zband_reach)
                for k in args.zband_halos}
    ps0 = searches[args.zband_halos[0]]
    propose_ms = event_ms(lambda: net.propose(spec, w.n_bins, ps0.logits), 5)
    net.check()

    def grid(s):
        """Recall, pairs and step time (CUDA events, median of 5) at every grid point on spectrum s."""
        plan.convolve_power(s, full)
        plan.check()
        out = []
        for k, ps in searches.items():
            for thr in args.zband_thresholds:
                part.fill_(float("nan"))
                n = ps.search(s, part, thr)
                plan.check()
                rec, n_det, _, _ = zb.recall(torch, full, part, s, w.n_bins)
                point = {"z_halo": k, "threshold": thr, "recall": rec, "detections": n_det,
                         "pair_fraction": ps.unit_fraction, "pairs": int(n)}
                point["ms"] = event_ms(lambda: ps.search_async(s, part, thr, stream), 5)
                out.append(point)
        return out

    calib, n_calib = chirp_spectrum(171110860)
    calib_points = grid(calib)
    del calib
    chosen = choose_operating_point(calib_points, args.zband_recall)
    k, thr = chosen["z_halo"], chosen["threshold"]
    dense, n_dense = chirp_spectrum(171110859)
    dense_points = grid(dense)
    del dense
    survey_points = grid(spec)      # leaves the survey's full plane in `full`
    at = lambda pts: next(p for p in pts if p["z_halo"] == k and p["threshold"] == thr)
    # the group-unit path with segment masks at the same threshold, for comparison (no z halo)
    ps_groups = zb.ProposalSearch(net, plan, pairs=False)
    part.fill_(float("nan"))
    n_units = ps_groups.search(spec, part, thr)
    plan.check()
    g_rec, _, _, _ = zb.recall(torch, full, part, spec, w.n_bins)
    groups_point = {"threshold": thr, "recall": g_rec, "unit_fraction": ps_groups.unit_fraction,
                    "pair_fraction": ps_groups.segment_fraction, "units": int(n_units),
                    "ms": event_ms(lambda: ps_groups.search_async(spec, part, thr, stream), 5)}
    del ps_groups
    ps = searches[k]
    for _ in range(args.warmup):
        ps.search(spec, part, thr)
    plan.check()
    # timed step: the whole path on the device (proposal, pair list, correlation with the list
    # length read on the device), CUDA events on the launching stream; the list length is read
    # back after the timed region
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for _ in range(args.warmup):
        ps.search_async(spec, part, thr, stream)
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        time.sleep(0.3)   # a few clock samples before the short timed region
        torch.cuda.nvtx.range_push("zband_step")   # names the timed launches for profilers
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record(stream)
            ps.search_async(spec, part, thr, stream)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    timed_pairs = ps.device_units()
    plan.check()
    net.check()
    ms = sum(step_ms) / len(step_ms)
    peaks, peak_src = measured_peaks()
    hop = zb.WINDOW // 2
    macs = ps.n_blocks * hop * (9 * 32 + 2 * 9 * 32 * 32) + ps.n_blocks * plan.n_z * 32
    tflops = 2.0 * macs / (propose_ms * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    shape_tflops = 2.0 * 128 * 32 * 16 / 64 * sms * 2.07e9 / 1e12   # at the maximum SM clock
    dense_at = at(dense_points)
    line = {
        "metric": "effective f-fdot cells/s of the learned z-band proposal path (full-plane cells / path time)",
        "value": cells / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16/f32",
        "data": "synthetic (survey spectrum; training windows labelled by the full search)",
        "config": {"workload": w.name + "-zband", "n_bins": w.n_bins, "n_z": plan.n_z, "window": zb.WINDOW,
                   "hop": hop, "threshold": thr, "z_halo": k, "reach_threshold": args.zband_reach,
                   "train_windows": n_windows,
                   "train_detected": n_detected, "train_snr": list(args.zband_snr),
                   "train_snr_dist": args.zband_snr_dist, "train_steps": args.zband_steps, "train_s": train_s,
                   "final_loss": losses[-1][1], "l2": "512 MiB buffer written between timed steps",
                   "timing": "CUDA events around the device-resident path (list length read on the device, "
                             "read back after the timed region)", "timed_pairs": timed_pairs},
        "recall": at(survey_points)["recall"], "pair_fraction": at(survey_points)["pair_fraction"],
        "full_search_ms": full_ms, "full_search_cells_per_s": cells / (full_ms * 1e-3), "propose_ms": propose_ms,
        "calibration": {"spectrum": f"2^22 bins, {n_calib} chirps (one per 16 blocks), held out (seed 171110860)",
                        "target_recall": args.zband_recall, "chosen": chosen, "points": calib_points},
        "dense": {"spectrum": f"2^22 bins, {n_dense} chirps (one per 16 blocks), SNR {args.zband_snr[0]:g}-"
                              f"{args.zband_snr[1]:g} {args.zband_snr_dist}",
                  "recall": dense_at["recall"], "pair_fraction": dense_at["pair_fraction"], "ms": dense_at["ms"],
                  "speedup_vs_full": full_ms / dense_at["ms"], "points": dense_points},
        "operating_points": survey_points,
        "groups_with_segment_masks": groups_point,
        "roofline": {"bound": "tensor", "kernel": "propose_kernel (+ median selection in the timed call)",
                     "achieved": tflops, "peak": float(peaks["bf16_tflops"]), "unit": "TFLOP/s",
                     "frac": tflops / float(peaks["bf16_tflops"]),
                     "peak_source": f"bf16_tflops burst ({peak_src}); FP16 dense rate equals BF16",
                     "flops_per_launch": 2.0 * macs, "traffic": zband_traffic(),
                     # the layers' MMAs are M = 128, N = 32, K = 16: one occupies the tensor pipe ~64
                     # cycles (a per-instruction floor below N = 128), a quarter of the dense rate
                     "shape_peak": {"cycles_per_mma": 64, "tflops": shape_tflops,
                                    "frac": tflops / shape_tflops}},
        # per step: median (init, three histogram passes, three digit kernels) and the fused
        # inference (8), the pair list (3), the list check and the pair correlation (2)
        "clocks": clk.summary(), "gpu_launches": args.steps * 13,
    }
    print(json.dumps(line), flush=True)
    net.close()
    plan.close()
    return 0


def run_ours(args):
    import torch
    from paper_1711_10855_gb300 import fdas

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1711_10855_gb300 import build as fdas_build
    if rank == 0 or world == 1:
        fdas_build.build()
    if world > 1:
        torch.distributed.barrier()
        fdas_build.build()

    w = workload(args.workload, args.n_bins)
    if args.seg_len:
        w = synth.with_seg_len(w, args.seg_len)
    # each rank correlates its own spectrum (independent de-dispersion trials)
    wr = synth.Workload(w.name, w.n_samples, w.zmax, w.zstep, w.tmpl_len, w.seg_len, w.seed + 1000 * rank,
                        w.chirps)
    spec = synth.spectrum(wr)
    plan = fdas.Plan(w.n_bins, w.zmax, w.zstep, w.seg_len, w.tmpl_len)
    stream = torch.cuda.current_stream(dev)
    tb0, tb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tb0.record(stream)
    plan.build_templates(stream)
    tb1.record(stream)
    plan.check(stream)
    template_build_ms = tb0.elapsed_time(tb1)

    d_spec = torch.from_numpy(spec.view(np.float32).copy()).to(dev)
    plane = torch.empty((plan.n_z, w.n_bins), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tc = args.precision != "f32"

    def correlate(out):
        if tc:
            plan.convolve_power_tc(d_spec, out, args.precision, stream)
        else:
            plan.convolve_power(d_spec, out, stream)

    for _ in range(args.warmup):
        correlate(plane)
        flush.fill_(1.0)
    plan.check(stream)

    # ---- device-timed region: K launches, CUDA events on the launching stream -------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        for e0, e1 in evs:
            flush.fill_(1.0)                     # L2 flush between timed steps, outside the events
            e0.record(stream)
            correlate(plane)
            e1.record(stream)
        torch.cuda.synchronize(dev)
    plan.check(stream)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    accuracy = tc_accuracy(torch, plan, w, d_spec, plane, stream) if tc else None
    ms = sum(step_ms) / len(step_ms)
    t_max = max_over_ranks(sum(step_ms) / 1e3, dev)
    cells = plan.n_z * w.n_bins
    value = replica_throughput(cells, args.steps, world, t_max)

    # ---- end to end through the public call with host buffers -----------------------------
    # Each step copies the spectrum from pinned host memory and the kernel stores the plane
    # straight into pinned host memory (the plane crosses the host link inside the kernel,
    # overlapped with the computation; a separate device-to-host copy measured 1.4 ms slower).
    h_spec = torch.from_numpy(spec.view(np.float32).copy()).pin_memory()
    h_plane = torch.empty((plan.n_z, w.n_bins), dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(1):
        d_spec.copy_(h_spec, non_blocking=True)
        correlate(h_plane)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        d_spec.copy_(h_spec, non_blocking=True)
        correlate(h_plane)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plan.check(stream)
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    e2e_value = replica_throughput(cells, e2e_steps, world, e2e_s)

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    peaks, peak_src = measured_peaks()
    alg = algorithmic(w, plan.n_seg, plan.group_segments if w.seg_len <= 2048 else 1)
    hbm_peak = float(peaks["hbm_gbs"])
    hbm_achieved = alg["bytes"] / (ms * 1e-3) / 1e9
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT_GB300 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s, FMA = 2
    alu_achieved = alg["flops"] / (ms * 1e-3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if tj.get("workload") == w.name and tj.get("kernel_rev") == kernel_rev():
            traffic = tj.get("dram_bytes_per_launch")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if not tc else f"{args.precision}x3+f32", "data": "synthetic",
        "config": {"workload": w.name, "n_bins": w.n_bins, "n_z": plan.n_z, "zmax": w.zmax, "zstep": w.zstep,
                   "seg_len": w.seg_len, "tmpl_len": w.tmpl_len, "n_seg": plan.n_seg,
                   "parallelism": f"replicas{world}",
                   "l2": "512 MiB buffer written between timed steps (outside the step events); "
                         "each step also writes a 3.4 GB plane"},
        "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": alu_achieved / alu_peak, "traffic": traffic,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (derived)",
                     "flops_per_launch": alg["flops"]},
        "hbm_roofline": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_achieved / hbm_peak, "peak_source": f"hbm_gbs ({peak_src})",
                         "bytes_per_launch": alg["bytes"]},
        "co_limits": {"note": "shared-memory Stockham kernel (L >= 4096): co-limits not modeled"}
        if w.seg_len > 2048 else {
            "smem_exchange": {"bytes_per_launch": alg["smem_bytes"],
                              "achieved": alg["smem_bytes"] / (ms * 1e-3) / 1e9, "unit": "GB/s",
                              "peak": SM_COUNT_GB300 * 128 * sm_max * 1e6 / 1e9,
                              "frac": alg["smem_bytes"] / (ms * 1e-3) / (SM_COUNT_GB300 * 128 * sm_max * 1e6),
                              "peak_source": f"152 SMs x 128 B/clock x {sm_max:.0f} MHz (nominal)"},
            "l2_template_reads": {"bytes_per_launch": alg["l2_template_bytes"],
                                  "achieved": alg["l2_template_bytes"] / (ms * 1e-3) / 1e9, "unit": "GB/s",
                                  "peak": None, "peak_source": "no measured L2 peak"}},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(d_spec.numel() * 4),
                "d2h_bytes_per_step": int(plane.numel() * 4), "steps": e2e_steps,
                "mode": "spectrum copied from pinned host memory; the kernel stores the plane into pinned host memory"},
        "gpu_launches": args.steps,
        "template_build_ms": template_build_ms,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
    }
    del h_plane
    if tc:
        tc_roofline(torch, plan, w, d_spec, stream, ms, line, peaks, peak_src)
        line["accuracy"] = accuracy
    elif w.seg_len == 2048 and not args.no_variants:
        torch.cuda.empty_cache()
        line["variants"] = tc_variants(torch, plan, w, d_spec, plane, flush, stream, alg["flops"], peaks, peak_src,
                                       alu_peak)
    del plane, flush
    torch.cuda.empty_cache()
    if not args.no_cpu_baseline:
        cores = cpu_cores()
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        rate, rows, dt = oracle_rows_rate(spec, w, seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{rows} whole rows ({rows * w.n_bins} cells) of the plane, "
                                          f"FP64 direct sum, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def tc_accuracy(torch, plan, w, d_spec, plane, stream) -> dict:
    """Per-row error of the tensor-core plane against the FP32 path's (max over the row of the
    absolute difference over the row's peak), and recovery of the injected chirps: the argmax of
    each chirp's +-64-bin window must lie within one zstep and one bin of (z, mean r)."""
    ref = torch.empty_like(plane)
    plan.convolve_power(d_spec, ref, stream)
    plan.check(stream)
    err = ((plane - ref).abs().amax(dim=1) / ref.amax(dim=1)).cpu().numpy()
    zs = np.arange(-w.zmax, w.zmax + 1, w.zstep)
    found = 0
    for c in w.chirps:
        r0 = int(round(c.r_mean))
        lo, hi = max(r0 - 64, 0), min(r0 + 65, w.n_bins)
        win = plane[:, lo:hi].cpu().numpy()
        zi, dr = np.unravel_index(np.argmax(win), win.shape)
        found += int(abs(zs[zi] - c.z) <= w.zstep + 1e-9 and abs(lo + dr - c.r_mean) <= 1.0)
    del ref
    return {"vs": "FP32 path plane (itself within 1e-5 per row of the FP64 oracle in the tests)",
            "max_row_rel_err": float(err.max()), "median_row_rel_err": float(np.median(err)),
            "rows": int(err.size), "chirps_recovered": found, "chirps": len(w.chirps)}


def tc_variants(torch, plan, w, d_spec, plane, flush, stream, method_flops: int, peaks, peak_src, alu_peak):
    """The tensor-core variants of the segment transforms on the same plan and spectrum, beside the
    FP32 line: per precision, the time per plane (CUDA events over 5 launches after 2 warm-ups,
    L2 flushed between), the per-row error against the FP32 plane just computed (`plane`), chirp
    recovery, and two rates: the method's nominal FFT flops (the FP32 line's count) per second,
    and the dense hi + lo DFT-matrix products the kernel executes against the tensor peak."""
    out = {"vs": "FP32 path plane of this run (itself within 1e-5 per row of the FP64 oracle in the tests)"}
    other = torch.empty_like(plane)
    zs = np.arange(-w.zmax, w.zmax + 1, w.zstep)
    for prec in ("bf16", "fp16"):
        for _ in range(2):
            plan.convolve_power_tc(d_spec, other, prec, stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record(stream)
            plan.convolve_power_tc(d_spec, other, prec, stream)
            e1.record(stream)
        torch.cuda.synchronize(d_spec.device)
        plan.check(stream)
        t = [a.elapsed_time(b) for a, b in evs]
        ms = statistics.median(t)
        err = ((other - plane).abs().amax(dim=1) / plane.amax(dim=1)).cpu().numpy()
        found = 0
        for c in w.chirps:
            r0 = int(round(c.r_mean))
            lo, hi = max(r0 - 64, 0), min(r0 + 65, w.n_bins)
            win = other[:, lo:hi].cpu().numpy()
            zi, dr = np.unravel_index(np.argmax(win), win.shape)
            found += int(abs(zs[zi] - c.z) <= w.zstep + 1e-9 and abs(lo + dr - c.r_mean) <= 1.0)
        dense = tc_flops(plan.n_seg, plan.n_z)
        tpk = float(peaks["bf16_tflops"])
        out[prec] = {"ms_per_plane": ms, "cells_per_s": plan.n_z * w.n_bins / (ms * 1e-3),
                     "max_row_rel_err": float(err.max()), "median_row_rel_err": float(np.median(err)),
                     "chirps_recovered": found, "chirps": len(w.chirps),
                     "method_flops_rate": {"achieved": method_flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                                           "flops_per_plane": method_flops,
                                           "frac_of_fp32_peak": method_flops / (ms * 1e-3) / 1e12 / alu_peak},
                     "dense_products_rate": {"achieved": dense / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                                             "flops_per_plane": dense, "peak": tpk,
                                             "frac": dense / (ms * 1e-3) / 1e12 / tpk,
                                             "peak_source": f"bf16_tflops burst ({peak_src})"},
                     "gpu_launches": 2 * (2 + len(evs))}
    del other
    return out


def tc_flops(nseg: int, Z: int) -> int:
    """Tensor flops of the DFT-matrix inverse transforms per call: for each (segment, template) a
    64-point DFT of 32 columns as a real GEMM (32 rows, N = 128, K = 128) and a 32-point DFT of 64
    columns (64 rows, N = 64, K = 64), each as three products (hi hi, hi lo, lo hi)."""
    per = 3 * (2 * 32 * 128 * 128 + 2 * 64 * 64 * 64)
    return nseg * Z * per


def tc_roofline(torch, plan, w, d_spec, stream, step_ms, line, peaks, peak_src):
    """The tensor-core path's line: a step is two launches (the forward segment transforms, then
    the correlation, both on the tensor cores); the forward launch is timed on its own and taken
    off the step to give the correlation kernel's duration."""
    seg = torch.empty((plan.n_seg, w.seg_len * 2), dtype=torch.float32, device=d_spec.device)
    reps = 10
    precision = line["dtype"].split("x")[0]
    plan.segment_spectra_tc(d_spec, seg, precision, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.segment_spectra_tc(d_spec, seg, precision, stream)
    e1.record(stream)
    torch.cuda.synchronize(d_spec.device)
    fwd_ms = e0.elapsed_time(e1) / reps
    kern_ms = max(step_ms - fwd_ms, 1e-6)
    flops = tc_flops(plan.n_seg, plan.n_z)
    peak = float(peaks["bf16_tflops"])
    achieved = flops / (kern_ms * 1e-3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic_tc.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if tj.get("workload") == w.name and tj.get("kernel_rev") == tc_kernel_rev():
            traffic = tj.get("dram_bytes_per_launch")
    line["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": traffic,
                        "peak_source": f"bf16_tflops burst ({peak_src}); FP16 dense rate equals BF16",
                        "flops_per_launch": flops, "kernel_ms": kern_ms, "forward_ms": fwd_ms}
    line["gpu_launches"] = 2 * line["steps"]
    line["config"]["precision"] = f"inverse transforms on tensor cores, {line['dtype']}"
    del seg


def tc_kernel_rev() -> str:
    """Content hash of the tensor-core correlation kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for name in ("fdas_tc.cu", "fdas_umma.cuh", "fdas_device.cuh"):
        with open(os.path.join(ROOT, "paper_1711_10855_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def zband_kernel_rev() -> str:
    """Content hash of the z-band kernel sources (ncu traffic of the inference kernel)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("fdas_zband.cu", "fdas_umma.cuh", "fdas_device.cuh"):
        with open(os.path.join(ROOT, "paper_1711_10855_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def zband_traffic():
    path = os.path.join(ROOT, "profiles", "traffic_zband.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        tj = json.load(f)
    return tj.get("dram_bytes_per_launch") if tj.get("kernel_rev") == zband_kernel_rev() else None


def kernel_rev() -> str:
    """Content hash of the kernel sources; ncu traffic figures are valid only for this hash."""
    import hashlib
    h = hashlib.sha256()
    for name in ("fdas_convolve.cu", "fdas_device.cuh"):
        with open(os.path.join(ROOT, "paper_1711_10855_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["survey", "small", "batch", "zband"], default="survey")
    ap.add_argument("--zband-windows", type=int, default=100_000)
    ap.add_argument("--zband-snr", type=float, nargs=2, default=[5.0, 30.0])
    ap.add_argument("--zband-snr-dist", choices=["uniform", "log-uniform"], default="uniform")
    ap.add_argument("--zband-steps", type=int, default=8000)
    ap.add_argument("--zband-thresholds", type=float, nargs="+", default=[0.05, 0.1, 0.15, 0.2, 0.3, 0.5])
    ap.add_argument("--zband-halos", type=int, nargs="+", default=[0, 4, 8, 12])
    ap.add_argument("--zband-recall", type=float, default=0.97)
    ap.add_argument("--zband-reach", type=float, default=0.5)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the tensor-core variants object")
    ap.add_argument("--n-bins", type=int, default=None, help="profiling only: shorter spectrum, same geometry")
    ap.add_argument("--seg-len", type=int, default=None, help="segment length sweep (default: the workload's)")
    ap.add_argument("--precision", choices=["f32", "bf16", "fp16"], default="f32",
                    help="f32: FP32 FFT path; bf16 / fp16: inverse transforms on the tensor cores (hi + lo split)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "zband":
        return run_zband(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
