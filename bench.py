#!/usr/bin/env python
"""Benchmark of the acquisition search on the realistic workload.

Workload (one step = one full search of one stream, every code x every bin):
1 s of complex64 baseband at 8 MS/s (int16-range Gaussian noise, sigma 2048)
with 40 injected tags at SNR U[-20, 0] dB, 16 codes of 8192 +/-1 chips at 8
samples/chip (L = 65536), windows of N = 131072 overlapping by one code
length (122 windows), 31 carrier-offset bins over +/-15 kHz.  Synthetic,
seeded; it stands in for the paper's recorded 8 MS/s receiver data.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (bounded sample per step).
Multi-GPU (torchrun): every rank searches its own stream (weak scaling,
replicas; no collective on the data path, only a barrier and a max-reduce of
the timings).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "acquisition Msamples/s (full code x freq-bin search); % HBM roofline"
UNIT = "Msamples/s"
WORKLOAD = ("realistic: 1 s complex64 IQ at 8 MS/s, 16 codes x 8192 chips, 8 samples/chip, "
            "N = 131072 (hop 65536, 122 windows), 31 bins over +/-15 kHz, 40 tags at U[-20, 0] dB")
# FP32 FMA lanes per SM of sm_100/sm_103 parts (an architecture constant, not a
# queryable device property); the SM count and the maximum SM clock are read from
# the device (device_fp32_peak) when the benchmark starts.
FP32_LANES_PER_SM = 128
FP32_PEAK_TFLOPS = None   # set by device_fp32_peak()
PEAK_NOTE = ""
L2_FLUSH_BYTES = 256 << 20


def device_fp32_peak(torch, dev) -> float:
    """FP32 FMA peak of the device: SMs x 128 lanes x 2 flop x maximum SM clock.
    The SM count comes from the device properties, the maximum clock from
    nvidia-smi (clocks.max.sm); sets FP32_PEAK_TFLOPS and PEAK_NOTE."""
    global FP32_PEAK_TFLOPS, PEAK_NOTE
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, src = None, "nvidia-smi clocks.max.sm"
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(dev.index or 0)], capture_output=True, text=True, timeout=20).stdout
        mhz = float(out.strip().splitlines()[0])
    except Exception:
        mhz, src = 2070.0, "GB300 maximum SM clock (nvidia-smi unavailable)"
    FP32_PEAK_TFLOPS = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    PEAK_NOTE = (f"FP32 FMA: {sms} SMs (device) x {FP32_LANES_PER_SM} lanes x 2 x {mhz / 1e3:.3f} GHz ({src}); "
                 "derived, not measured")
    return FP32_PEAK_TFLOPS


def flops_per_cell(N: int) -> float:
    """Algorithmic FP32 flops of one (window, code, bin) cell of the correlation
    kernel, in the plain method's terms: inverse FFT of N points (5 N log2 N),
    complex multiply by the code spectrum (6 N), |.|^2 and the floor/argmax
    reduction (4 N)."""
    import math
    return 5.0 * N * math.log2(N) + 6.0 * N + 4.0 * N


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("acq_fft_kernels.cuh", "acq_common.cuh", "fft_block.cuh"):
        with open(os.path.join(ROOT, "paper_2005_10445_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fsk_kernel_source_hash() -> str:
    """sha256 (first 16 hex digits) of the FSK correlation's kernel sources and
    of the host file that sizes its passes."""
    h = hashlib.sha256()
    for f in ("fsk_fft.cu", "acq_fft_kernels.cuh", "acq_common.cuh", "fft_block.cuh", "atlas_fsk_host.cu"):
        with open(os.path.join(ROOT, "paper_2005_10445_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fsk_ncu_traffic_per_cell():
    """DRAM bytes per (window, code) cell of k_fsk_corr from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "k_fsk_corr_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != fsk_kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_cell"])
    except (KeyError, ValueError):
        return None


def ncu_traffic(units_per_launch: float):
    """DRAM bytes of the correlation kernel from the committed ncu summary,
    scaled from the captured full launch to a launch of `units_per_launch`
    cells, if the summary was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "k_corr_realistic_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"]) * units_per_launch / float(vals["cells_per_full_launch"])
    except (KeyError, ValueError, ZeroDivisionError):
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = os.path.join("/tmp", f"atlas_clocks_{os.getpid()}.csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id is not None:
            cmd += ["-i", str(gpu_id)]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "power_w_max": max(pw),
                "samples": len(sm), "reasons": sorted(reasons)}


BATCH_WORKLOAD = ("batching: 8 receiver streams of U[0.5, 2] s at 2, 4 or 8 MS/s (samples/chip = fs / 1 MHz), "
                  "64 codes of 2048-16384 chips, 15-63 bins of 500 Hz per stream, about 5 tags per stream and "
                  "code length at U[-20, 0] dB; one CUDA-graph launch per step; autotuned tile shapes")


def executed_flops(wl) -> float:
    """FP32 flops the polyphase search executes on one stream (5 n log2 n per
    n-point transform; per (window, bin): sps forward transforms of M points;
    per cell: sps inverse transforms plus 10 N for the multiply and epilogue)."""
    import collections
    import math
    tot = 0.0
    for nc, C in collections.Counter(len(c) for c in wl.chips).items():
        L = nc * wl.sps
        N = wl.fft_len or 2 * (1 << (L - 1).bit_length())
        hop, M = N - L, N // wl.sps
        W = max(1, -(-(wl.n_samples - N) // hop) + 1)
        K = len(wl.freqs_hz)
        fft = wl.sps * 5.0 * M * math.log2(M)
        tot += W * K * fft + W * C * K * (fft + 10.0 * N)
    return tot


def unfused_baseline(args, wl, x, st, flush, dev, torch, fused_value):
    """The paper-organised comparison pipeline (cuFFT + element-wise kernels,
    the correlation surface in device memory) timed like the fused search on
    the same resident stream."""
    from paper_2005_10445_gb300 import binding
    S = wl.n_samples
    u = binding.UnfusedSearch(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len)
    cap = args.capacity
    out = torch.empty(cap * 32, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        u.run_ptr(st.cuda_stream, x.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 5))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(st)
        u.run_ptr(st.cuda_stream, x.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())
        evs[i][1].record(st)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    n = int(cnt.item())
    u.close()
    value = S / (ms / 1e3) / 1e6
    return {"value": value, "unit": UNIT, "ms_per_step": ms, "steps": steps, "detections_per_step": n,
            "fused_speedup": fused_value / value,
            "pipeline": "paper-organised: mix kernel, cuFFT forward (windows x bins), multiply kernel for every "
                        "code, cuFFT inverse in place (16 windows x 16 codes x 31 bins per group, the surface in "
                        "HBM), power/floor/argmax kernel reading the surface; same selection and refinement"}


SECONDS = 1.0  # stream length of the realistic workload (--seconds; shorter streams are for profiling runs)


def workload_name() -> str:
    if SECONDS == 1.0:
        return WORKLOAD
    S, N, hop = int(round(8e6 * SECONDS)), 131072, 65536
    W = 1 if S <= N else (S - N + hop - 1) // hop + 1
    return (WORKLOAD.replace("realistic: 1 s", f"realistic, shortened: {SECONDS:g} s")
            .replace("122 windows", f"{W} windows"))


def make_workload(seed: int):
    from paper_2005_10445_gb300 import synth
    return synth.realistic(seed=seed, seconds=SECONDS)


def oracle_pool(wl):
    """The FP64 oracle as it stands, on every host core (spawned worker
    processes, each running the plain search on its share of the pairs)."""
    from oracle import parallel
    return parallel.Pool(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)


def oracle_sample(pool, wl, windows=(1,)):
    """Time the oracle pool on the given windows x every code x every bin:
    returns (seconds, equivalent samples = hop per window: a window holds hop
    new samples for all codes)."""
    from oracle import acq
    L = len(wl.chips[0]) * wl.sps
    W, hop = acq.window_plan(wl.n_samples, wl.fft_len, L)
    pairs = [(w, c) for w in windows for c in range(len(wl.chips))]
    t0 = time.perf_counter()
    pool.search(pairs, chunk=1)
    dt = time.perf_counter() - t0
    return dt, hop * len(windows)


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    wl = make_workload(2)
    with oracle_pool(wl) as pool:
        for _ in range(args.warmup):
            oracle_sample(pool, wl)
        times, samples = [], 0.0
        for _ in range(args.steps):
            dt, s = oracle_sample(pool, wl)
            times.append(dt)
            samples += s
        cores = pool.processes
    total = sum(times)
    value = samples / total / 1e6
    sample = (f"per step: window 1 x 16 codes x 31 bins of the same stream (numpy FP64 oracle, {cores} worker "
              "processes); Msamples/s = hop / time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": f"{cores} host processes"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_batching(dev, torch, steps: int, warmup: int, cap: int, rank: int = 0, world: int = 1, dist=None):
    """The batching workload (8 receiver streams, 64 codes of four lengths,
    per-stream bins) as one graph launch per step: returns (Msamples/s, ms per
    batch, total samples, kernels per graph launch, executed TFLOP/s, clocks,
    per-stream detection counts, tile choices, per-stream correlation timing)."""
    from paper_2005_10445_gb300 import binding, synth
    wls = synth.batch(seed=3 + rank)
    searches = [binding.Search(w.chips, w.sps, w.fs_hz, w.freqs_hz) for w in wls]
    xs = [torch.from_numpy(w.iq().copy()).to(dev) for w in wls]
    st = torch.cuda.current_stream(dev)
    cache = os.environ.get("ATLAS_TUNE_CACHE", os.path.join("/tmp", "atlas_acq_tune.jsonl"))
    for srch, x, w in zip(searches, xs, wls):
        srch.autotune(st.cuda_stream, x.data_ptr(), w.n_samples, cache)
    tiles = sorted({srch.tuning(c) for srch in searches for c in range(len(wls[0].chips))})
    out = torch.zeros(len(wls) * cap * 32, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(len(wls), dtype=torch.int32, device=dev)
    b = binding.Batch(searches, [x.data_ptr() for x in xs], [w.n_samples for w in wls], out.data_ptr(), cap,
                      cnt.data_ptr())
    S = sum(w.n_samples for w in wls)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        b.run(st.cuda_stream)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler() if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(st)
        b.run(st.cuda_stream)
        evs[i][1].record(st)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    t = torch.tensor([sum(a.elapsed_time(c) for a, c in evs)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = S * world * steps / (total_ms / 1e3) / 1e6
    counts = cnt.cpu().numpy().tolist()
    kernels = b.kernels()
    b.close()
    # dominant kernel: per-stream runs outside the graph, timed by the library's events
    corr = {"ms": 0.0, "cells": 0, "launches": 0}
    for srch, x, w in zip(searches, xs, wls):
        srch.profile_begin(65536)
        srch.run_ptr(st.cuda_stream, x.data_ptr(), w.n_samples, out.data_ptr(), cap, cnt.data_ptr())
        pr = srch.profile_end()
        corr["ms"] += pr["corr_ms"]
        corr["cells"] += pr["corr_units"]
        corr["launches"] += pr["corr_launches"]
    fl = sum(executed_flops(w) for w in wls)
    step_tflops = fl / (total_ms / steps / 1e3) / 1e12
    return {"value": value, "ms_per_step": total_ms / steps, "samples": S, "kernels_per_launch": kernels,
            "tflops": step_tflops, "clocks": clocks, "counts": counts, "tiles": tiles, "corr": corr,
            "streams": [w.name for w in wls]}


def run_batching(args, rank: int, world: int, dev, torch, dist) -> None:
    r = measure_batching(dev, torch, args.steps, args.warmup, args.capacity, rank, world, dist)
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "samples_per_step_per_gpu": r["samples"],
                       "streams": r["streams"], "tile_log2_windows_per_launch": r["tiles"],
                       "l2": "flushed before each step (256 MiB write), outside the timed events",
                       "parallelism": "replicas: one independent batch per GPU",
                       "detections_per_stream": r["counts"]},
            "roofline": {"bound": "alu", "achieved": r["tflops"], "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": r["tflops"] / FP32_PEAK_TFLOPS, "traffic": None,
                         "kernel": "whole graph (executed polyphase flops / step time)",
                         "k_corr_ms_per_step_outside_graph": r["corr"]["ms"],
                         "k_corr_launches": r["corr"]["launches"], "k_corr_cells": r["corr"]["cells"]},
            "gpu_launches": r["kernels_per_launch"] * args.steps,
            "clocks": r["clocks"],
        }
        print(json.dumps(line), flush=True)


def run_learned(args, rank: int, world: int, dev, torch, dist) -> None:
    """Learned-proposal row: train on windows labelled by the exhaustive search,
    then report recall and speedup of the proposal search against the
    exhaustive search on held-out windows (64 codes x 63 bins)."""
    from paper_2005_10445_gb300 import binding, learned, synth
    n_train, n_test = args.train_windows, args.test_windows
    cap = max(1 << 16, 4 * n_train)
    t0 = time.perf_counter()
    x_tr, chips, freqs, _ = synth.proposal_stream(5 + 100 * rank, n_train, dev, code_seed=5)
    S_tr = x_tr.shape[0]
    # T = 50: at up to +5 dB over 64 codes, a strong tag's real-valued cross-correlation
    # with the other codes peaks at 25-30 times its floor, so T = 25 would label sidelobes
    search = binding.Search(chips, 8, 8e6, freqs, threshold=50.0)
    W, hop, N = search.windows(0, S_tr)
    dets, n_lab, t_lab = learned.exhaustive(search, x_tr, S_tr, cap, torch)
    code, bin_ = learned.labels_from(dets, W)
    prop = binding.Proposal(len(chips), len(freqs), seed=5)
    prop.set_grid(8e6, freqs)
    feat = learned.features(prop, x_tr, S_tr, W, hop, N, torch)
    hist = learned.train(prop, feat, code, bin_, torch, epochs=args.epochs)
    del x_tr, feat
    torch.cuda.empty_cache()
    x_te, _, _, truth = synth.proposal_stream(6 + 100 * rank, n_test, dev, code_seed=5)
    S_te = x_te.shape[0]
    learned.exhaustive(search, x_te, S_te, cap, torch)  # warm
    exh, n_exh, t_exh = learned.exhaustive(search, x_te, S_te, cap, torch)
    curve = [learned.evaluate(search, prop, x_te, S_te, exh, t_exh, 8, tau, cap, torch)
             for tau in (0.0, 0.3, 0.6, 0.9)]
    curve += [learned.evaluate(search, prop, x_te, S_te, exh, t_exh, nb, tau, cap, torch, bins=True)
              for nb in (1, 2, 4) for tau in (0.0, 0.5, 0.8, 0.9, 0.95, 0.99)]
    ok = [r for r in curve if r["recall"] >= 0.995]
    head = max(ok, key=lambda r: r["speedup"]) if ok else max(curve, key=lambda r: r["recall"])
    if rank == 0:
        line = {
            "metric": "learned proposal: speedup of the proposal search over the exhaustive search at >= 99.5% "
                      "recall (64 codes x 63 bins)",
            "value": head["speedup"], "unit": "x", "n_gpus": world, "higher_is_better": True,
            "recall": head["recall"], "tau_fb": head["tau_fb"], "topk": head["topk"], "mode": head["mode"],
            "max_toa_diff_samples": head["max_toa_diff_samples"], "dtype": "f32 search, f16 weights",
            "data": "synthetic",
            "threshold": 50.0,
            "config": {"workload": f"learned: fs 8 MS/s, N 131072, 64 codes x 8192 chips at sps 8, 63 bins "
                                   f"(-15.5..15.5 kHz, 500 Hz); {n_train} training windows (seed 5), {n_test} "
                                   f"test windows (seed 6); 0-1 tag per window at U[-25, 5] dB, 20% empty",
                       "train_windows": n_train, "test_windows": n_test, "epochs": args.epochs},
            "labels": {"windows_with_detection": int((code >= 0).sum()), "detections": n_lab,
                       "label_search_s": t_lab},
            "train_loss_per_epoch": hist,
            "exhaustive_test_s": t_exh, "exhaustive_test_detections": n_exh,
            "curve": curve,
            "wall_s": time.perf_counter() - t0,
        }
        print(json.dumps(line), flush=True)


def measure_precision(dev, torch, steps: int, warmup: int, cap: int, rank: int = 0):
    """Reduced-precision row: the realistic workload with the per-code inverse
    transforms in FP32 (CUDA cores) and as FP16 / BF16 tensor-core contractions;
    throughput, speedup over FP32, agreement of the detections and scores with
    the FP32 path, and the injected tags' cells found.  The errors against the
    FP64 oracle are asserted by tests/test_gpu_precision.py.  Returns
    ({precision: figures}, number of tag cells)."""
    import math
    from paper_2005_10445_gb300 import binding
    wl = make_workload(2 + rank)
    S = wl.n_samples
    x = torch.from_numpy(wl.iq().copy()).to(dev)
    out = torch.empty(cap * 32, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)
    res, dets = {}, {}
    for prec in (0, 1, 2):
        srch = binding.Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len, precision=prec)
        for _ in range(warmup):
            srch.run_ptr(st.cuda_stream, x.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())
        srch.profile_begin(65536)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(st)
            srch.run_ptr(st.cuda_stream, x.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())
            evs[i][1].record(st)
        torch.cuda.synchronize(dev)
        pr = srch.profile_end()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        n = int(cnt.item())
        d = out.cpu().numpy().view(binding.DETECTION_DTYPE)[: min(n, cap)].copy()
        dets[prec] = d
        res[prec] = {"ms_per_step": ms, "value": S / (ms / 1e3) / 1e6,
                     "k_corr_ms_per_launch": pr["corr_ms"] / max(pr["timed_launches"], 1), "detections": n}
        srch.close()
    key = lambda d: (int(d["code"]), int(d["window"]), int(d["lag"]), int(d["freq_bin"]))
    ref = {key(d): d for d in dets[0]}
    # the injected tags' cells (integer delays, known bins) under the window rule
    N, L = wl.fft_len, len(wl.chips[0]) * wl.sps
    hop = N - L
    W = max(1, math.ceil((S - N) / hop) + 1)
    tag_cells = set()
    for t in wl.tags:
        w = min(int(t.delay) // hop, W - 1)
        tag_cells.add((t.code, w, int(t.delay) - w * hop, t.bin))
    for prec in (0, 1, 2):
        got = {key(d): d for d in dets[prec]}
        common = set(got) & set(ref)
        score_diff = [abs(float(got[k]["score"]) / float(ref[k]["score"]) - 1) for k in common]
        toa_diff = [abs(float(got[k]["toa"]) - float(ref[k]["toa"])) for k in common]
        res[prec].update({
            "speedup_vs_fp32": res[0]["ms_per_step"] / res[prec]["ms_per_step"],
            "fp32_detections_reproduced": len(common) / max(len(ref), 1),
            "extra_vs_fp32": len(set(got) - set(ref)),
            "tag_cells_found": len(tag_cells & set(got)) / max(len(tag_cells), 1),
            "max_score_rel_diff_vs_fp32": max(score_diff or [0.0]),
            "max_toa_diff_vs_fp32": max(toa_diff or [0.0])})
    return res, len(tag_cells)


PRECISION_NAMES = {0: "fp32", 1: "fp16-tc", 2: "bf16-tc"}


def run_precision(args, rank: int, world: int, dev, torch, dist) -> None:
    res, n_tags = measure_precision(dev, torch, args.steps, args.warmup, args.capacity, rank)
    if rank == 0:
        names = PRECISION_NAMES
        line = {"metric": METRIC, "value": res[1]["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res[1]["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f16 tensor-core contractions, f32 accumulate",
                "data": "synthetic",
                "config": {"workload": "precision: " + workload_name(),
                           "l2": "flushed before each step (256 MiB write), outside the timed events",
                           "tag_cells": f"{n_tags} (code, window, lag, bin) cells of the injected tags"},
                "per_precision": {names[p]: r for p, r in res.items()}}
        print(json.dumps(line), flush=True)


def fsk_workload_name(N: int, hop: int, W: int) -> str:
    return ("fsk: 1 s of int16 (I, Q) at 8 MS/s (sigma 2048), 16 codes x 8192 chips at 8 samples/chip on "
            "tones +/-500 kHz, band centre 1 MHz off the receiver's, 200-tap band-pass filter (T = 207), "
            f"N = {N} (n_c = 65742, hop {hop}, {W} windows), 40 tags at U[-15, 0] dB")


def fsk_corr_flops_per_cell(N: int) -> float:
    """Algorithmic FP32 flops of one (window, code) cell of the FSK correlation:
    a real cross-correlation through an N-point transform is half of a complex
    one (2.5 N log2 N; two real windows share one complex transform), plus half
    of the complex spectral product (3 N) and corr^2, its sum and the argmax
    (3 N)."""
    import math
    return 2.5 * N * math.log2(N) + 6.0 * N


def fsk_demod_flops_per_sample(T: int) -> float:
    """FP32 flops per demodulated sample: per 4096-point block, one forward and
    two inverse transforms (5 B log2 B each) and two spectral products (6 B
    each) for B - T + 1 outputs, plus about 12 per output (two magnitudes, d, u)."""
    import math
    B = 4096
    return (3 * 5.0 * B * math.log2(B) + 2 * 6.0 * B) / (B - T + 1) + 12.0


def fsk_oracle_sample(w, windows=(1,)):
    """Time the FP64 oracle on the given windows x every code: (seconds,
    equivalent samples = hop per window)."""
    from oracle import fsk
    N, W, hop, n_c = fsk.plan(w.n_samples, len(w.chips[0]), w.sps, len(w.h_bp) + w.sps - 1, w.fft_len)
    t0 = time.perf_counter()
    fsk.search(w.iq16, w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp, w.fft_len,
               pairs=[(wi, c) for wi in windows for c in range(len(w.chips))])
    return time.perf_counter() - t0, hop * len(windows)


def fsk_codes_in_real_time(args, w, iq, st, flush, dev, torch, n_codes: int = 128) -> dict:
    """The paper's own throughput figure for its FSK search: how many codes can
    be searched in real time when half of the time goes to searching, with
    codes in batches of 128.  Times a 128-code context (8192 chips each; the
    stream's tags use 16 of them) on the same resident 1-s stream."""
    from paper_2005_10445_gb300 import binding, synth
    chips = [synth.random_chips(8192, 2 * 1_000_003 + c) for c in range(n_codes)]
    s = binding.FskSearch(chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp, fft_len=w.fft_len,
                          block_log2=args.fsk_block_log2)
    S = w.n_samples
    cap = 4096
    out = torch.empty(cap * binding.FSK_DETECTION_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        s.run_ptr(st.cuda_stream, iq.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 5))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(st)
        s.run_ptr(st.cuda_stream, iq.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())
        evs[i][1].record(st)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    s.close()
    seconds = S / w.fs_hz
    return {"codes_searchable_in_real_time": n_codes * (seconds / (ms / 1e3)) * 0.5,
            "definition": "codes per batch x (stream seconds / search seconds) x 0.5 (half of the time searching)",
            "codes_per_batch": n_codes, "ms_per_1s_stream": ms,
            "paper_same_metric": {"Titan Xp": 315, "GTX 1050": 77, "Jetson TX2": 26, "i7-8700T 1 core": 6},
            "note": "the paper's figures are for its recorded 8 MS/s data, 8192-bit codes and 100 ms windows "
                    "on its own hardware: context, not a like-for-like target"}


def run_fsk(args, rank: int, world: int, dev, torch, dist) -> None:
    """The FSK front end (Section 3 steps 1-8) on 1 s of int16 samples."""
    from paper_2005_10445_gb300 import binding, synth
    w = synth.fsk_realistic(seed=2 + rank, fft_len=args.fsk_fft_len)
    S = w.n_samples
    s = binding.FskSearch(w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp, fft_len=w.fft_len,
                          block_log2=args.fsk_block_log2)
    Wn, hop, N, n_c = s.windows(0, S)
    logN = N.bit_length() - 1
    M = 1 << (args.fsk_block_log2 or (13 if logN <= 17 else 14)) if logN > 14 else N
    iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).to(dev)
    cap = args.capacity
    rec = binding.FSK_DETECTION_DTYPE.itemsize
    out = torch.empty(cap * rec, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)

    def step():
        s.run_ptr(st.cuda_stream, iq.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    s.profile_begin(65536)
    sampler = ClockSampler() if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(st)
        step()
        evs[i][1].record(st)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    prof = s.profile_end()
    t = torch.tensor([sum(a.elapsed_time(b) for a, b in evs)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = S * world * args.steps / (total_ms / 1e3) / 1e6
    count = int(cnt.item())
    # end to end through the host-buffer entry point (pinned host memory)
    h_iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).pin_memory()
    h_out = torch.empty(cap * rec, dtype=torch.uint8).pin_memory()
    h_cnt = torch.zeros(1, dtype=torch.int32).pin_memory()
    for _ in range(max(2, args.warmup)):
        s.run_host_ptr(st.cuda_stream, h_iq.data_ptr(), S, h_out.data_ptr(), cap, h_cnt.data_ptr())
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    e2e_t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s.run_host_ptr(st.cuda_stream, h_iq.data_ptr(), S, h_out.data_ptr(), cap, h_cnt.data_ptr())
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = torch.tensor([sum(e2e_t)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_s, op=dist.ReduceOp.MAX)
    e2e_value = S * world * args.steps / float(e2e_s.item()) / 1e6
    n_host = int(h_cnt[0])
    if rank != 0:
        return
    T = len(w.h_bp) + w.sps - 1
    corr_avg = prof["corr_ms"] / max(prof["corr_timed"], 1)
    corr_units = prof["corr_units"] / max(prof["corr_launches"], 1)
    corr_tf = corr_units * fsk_corr_flops_per_cell(N) / (corr_avg / 1e3) / 1e12
    demod_avg = prof["demod_ms"] / max(prof["demod_timed"], 1)
    demod_samples = prof["demod_samples"] / max(prof["demod_launches"], 1)
    demod_tf = demod_samples * fsk_demod_flops_per_sample(T) / (demod_avg / 1e3) / 1e12
    corr_share = prof["corr_ms"] / total_ms
    demod_share = prof["demod_ms"] / total_ms
    dom = ("k_fsk_corr_a + k_fsk_corr_b (packed inverse N-point transform per (window pair, code) in two passes: "
           f"{N // M} blocks of {M} points to a device scratch, then the {N // M}-point transform across them, "
           "corr^2, floor, argmax)", corr_units, fsk_corr_flops_per_cell(N), corr_avg, corr_tf, corr_share) \
        if corr_share >= demod_share else \
        ("k_fsk_demod (int16 conversion, LO mix, both composed filters by 4096-point overlap-save transforms, d, u)",
         demod_samples, fsk_demod_flops_per_sample(T), demod_avg, demod_tf, demod_share)
    line = {
        "metric": "FSK acquisition Msamples/s (every code, the paper's FSK front end)", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": fsk_workload_name(N, hop, Wn), "samples_per_step_per_gpu": S, "windows": Wn,
                   "hop": hop, "fft_len": N, "block_points": M,
                   "l2": "flushed before each step (256 MiB write), outside the timed events",
                   "parallelism": "replicas: one independent stream per GPU", "detections_per_step": count},
        "roofline": {"bound": "alu", "achieved": dom[4], "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": dom[4] / FP32_PEAK_TFLOPS,
                     "traffic": (fsk_ncu_traffic_per_cell() * corr_units
                                 if dom[0].startswith("k_fsk_corr_a") and fsk_ncu_traffic_per_cell() else None),
                     "kernel": dom[0],
                     "units_per_launch": dom[1], "flops_per_unit": dom[2], "avg_launch_ms": dom[3],
                     "kernel_share_of_step": dom[5],
                     "peak_note": PEAK_NOTE,
                     "k_fsk_corr": {"avg_launch_ms": corr_avg, "cells_per_launch": corr_units,
                                    "tflops": corr_tf, "share": corr_share},
                     "k_fsk_demod": {"avg_launch_ms": demod_avg, "samples_per_launch": demod_samples,
                                     "tflops": demod_tf, "share": demod_share}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": S * 4,
                "d2h_bytes_per_step": 4 + rec * min(n_host, cap)},
        "gpu_launches": prof["launches"],
        "clocks": clocks,
    }
    line["paper_metric"] = fsk_codes_in_real_time(args, w, iq, st, flush, dev, torch)
    if world == 1 and not args.no_cpu_baseline:
        # about 10 s of CPU work: six windows x every code
        dt, samples = fsk_oracle_sample(w, windows=(1, 2, 3, 4, 5, 6))
        line["cpu_baseline"] = {"value": samples / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"windows 1-6 x 16 codes of the same stream (numpy FP64, single process, "
                                          f"{dt:.1f} s); Msamples/s = 6 hop / time"}
    print(json.dumps(line), flush=True)


STREAM_WORKLOAD = ("stream: 4 s of int16 (I, Q) at 8 MS/s pushed in 10 ms chunks into the device cyclic buffer; "
                   "16 tags x 8192 chips at 8 samples/chip (FSK, tones +/-500 kHz, f_lo 1 MHz), each transmitting "
                   "every U[0.4, 0.6] s at U[-15, 0] dB; scheduler: 100 ms searching blocks with 10 ms overlap, 12 ms "
                   "tracking blocks, half of the work each")


def run_stream(args, rank: int, world: int, dev, torch, dist) -> None:
    """Continuous ingest + scheduler (Section 2.2) on the FSK search: the whole
    stream is pushed chunk by chunk and every ready task is run after each
    push; a step is one pass over the stream with a fresh runtime."""
    from paper_2005_10445_gb300 import binding, synth
    fs = 8e6
    w, periods = synth.fsk_periodic(seed=2 + rank, seconds=4.0, fs_hz=fs, n_codes=16, n_chips=8192, sps=8,
                                    period_s=(0.4, 0.6), snr_range=(-15.0, 0.0), f_lo_hz=1e6, offset_hz=5e3)
    S = w.n_samples
    chunk = int(0.01 * fs)
    fsk_s = binding.FskSearch(w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp,
                              exchange=args.fsk_exchange)
    opts = binding.rt_default_opts(fs)
    iq = np.ascontiguousarray(w.iq16)
    st = torch.cuda.current_stream(dev).cuda_stream

    def one_pass(rt):
        n_ev = 0
        kinds = np.zeros(5, np.int64)
        for a in range(0, S, chunk):
            rt.push(iq[a:a + chunk], st)
            ev = rt.pump(0, 4096, st)
            n_ev += len(ev)
            kinds += np.bincount(ev["kind"], minlength=5)[:5]
        return n_ev, kinds

    for _ in range(args.warmup):
        one_pass(binding.Runtime(fsk_s, periods, opts))
    rts = [binding.Runtime(fsk_s, periods, opts) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    fsk_s.profile_begin(65536)
    sampler = ClockSampler() if rank == 0 else None
    if world > 1:
        dist.barrier()
    times, kinds = [], np.zeros(5, np.int64)
    for rt in rts:
        t0 = time.perf_counter()
        n_ev, k = one_pass(rt)
        times.append(time.perf_counter() - t0)
        kinds += k
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    prof = fsk_s.profile_end()
    stats = rts[-1].stats()
    t = torch.tensor([sum(times)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total = float(t.item())
    value = S * world * args.steps / total / 1e6
    if rank != 0:
        return
    T = len(w.h_bp) + w.sps - 1
    Wn, hop, N, n_c = fsk_s.windows(0, opts.search_block)
    corr_avg = prof["corr_ms"] / max(prof["corr_timed"], 1)
    corr_units = prof["corr_units"] / max(prof["corr_launches"], 1)
    corr_tf = corr_units * fsk_corr_flops_per_cell(N) / (corr_avg / 1e3) / 1e12
    line = {
        "metric": "continuous FSK ingest + scheduler Msamples/s (wall clock, host buffers)", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": STREAM_WORKLOAD, "samples_per_step_per_gpu": S, "chunk_samples": chunk,
                   "real_time_factor": value / (fs / 1e6),
                   "parallelism": "replicas: one independent receiver stream per GPU",
                   "l2": "not flushed: the cyclic buffer is written by every push"},
        "tasks_per_step": {"search": stats["search_tasks"], "track": stats["track_tasks"]},
        "events_per_step": {k: int(v) // args.steps for k, v in zip(
            ["search_detection", "track_detection", "track_miss", "track_lost", "search_skipped"], kinds)},
        "task_latency_ms": {"search": stats["search_ms"] / max(stats["search_tasks"], 1),
                            "track": stats["track_ms"] / max(stats["track_tasks"], 1)},
        "roofline": {"bound": "alu", "achieved": corr_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": corr_tf / FP32_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_fsk_corr inside the searching tasks (tracking tasks run as graphs, untimed)",
                     "units_per_launch": corr_units,
                     "flops_per_unit": fsk_corr_flops_per_cell(N), "avg_launch_ms": corr_avg,
                     "kernel_share_of_step": prof["corr_ms"] / (1e3 * total),
                     "peak_note": PEAK_NOTE},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": S * 4,
                "d2h_bytes_per_step": "per task: the count and its records"},
        # searching tasks' kernels (counted by the library) plus the kernel nodes of the tracking graph launches
        "gpu_launches": prof["launches"] // max(args.steps, 1) + stats["track_kernels"],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-unfused", action="store_true", help="skip the cuFFT comparison pipeline")
    ap.add_argument("--no-batching", action="store_true", help="skip the batching figure of the default line")
    ap.add_argument("--no-precision", action="store_true", help="skip the reduced-precision figure of the default line")
    ap.add_argument("--capacity", type=int, default=4096)
    ap.add_argument("--fsk-fft-len", type=int, default=1 << 18,
                    help="FSK workload: N (0 = the library default, 2 nextpow2(L) = 2^17 here)")
    ap.add_argument("--fsk-block-log2", type=int, default=0, help="FSK workload: log2 points per block (0 = default)")
    ap.add_argument("--fsk-exchange", type=int, default=0,
                    help="stream workload: exchange form of the FSK transforms (0 = default, 1 = cluster, 2 = two passes)")
    ap.add_argument("--workload", default="realistic", choices=["realistic", "batching", "learned", "precision", "fsk", "stream"])
    ap.add_argument("--train-windows", type=int, default=100000)
    ap.add_argument("--test-windows", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--seconds", type=float, default=1.0,
                    help="realistic and precision workloads: stream length in seconds (1.0 = the benchmark; "
                         "shorter streams only for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    global SECONDS
    SECONDS = args.seconds

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_2005_10445_gb300 import binding
    from paper_2005_10445_gb300.build import build

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    device_fp32_peak(torch, dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if not os.path.exists(binding.LIB_PATH):
        build()
    if args.workload in ("batching", "learned", "precision", "fsk", "stream"):
        {"batching": run_batching, "learned": run_learned, "precision": run_precision, "fsk": run_fsk,
         "stream": run_stream}[args.workload](
            args, rank, world, dev, torch, dist)
        if world > 1:
            dist.destroy_process_group()
        return
    wl = make_workload(2 + rank)
    S = wl.n_samples
    s = binding.Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len)
    x = torch.from_numpy(wl.iq().copy()).to(dev)
    cap = args.capacity
    out = torch.empty(cap * 32, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)

    def step():
        s.run_ptr(st.cuda_stream, x.data_ptr(), S, out.data_ptr(), cap, cnt.data_ptr())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # timed region: K steps, L2 flushed before each (outside the events)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    s.profile_begin(max_timed=65536)
    sampler = ClockSampler(gpu_id=None) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(st)
        step()
        evs[i][1].record(st)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    prof = s.profile_end()
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    count = int(cnt.item())
    t = torch.tensor([dev_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = S * world * args.steps / (total_ms / 1e3) / 1e6

    # end to end through the host-buffer entry point (pinned host memory)
    h_x = torch.from_numpy(wl.iq().copy()).pin_memory()
    h_out = torch.empty(cap * 32, dtype=torch.uint8).pin_memory()
    h_cnt = torch.zeros(1, dtype=torch.int32).pin_memory()
    for _ in range(max(2, args.warmup)):
        s.run_host_ptr(st.cuda_stream, h_x.data_ptr(), S, h_out.data_ptr(), cap, h_cnt.data_ptr())
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    e2e_t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s.run_host_ptr(st.cuda_stream, h_x.data_ptr(), S, h_out.data_ptr(), cap, h_cnt.data_ptr())
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = torch.tensor([sum(e2e_t)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_s, op=dist.ReduceOp.MAX)
    e2e_value = S * world * args.steps / float(e2e_s.item()) / 1e6
    n_host = int(h_cnt[0])

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    N = wl.fft_len
    units_per_launch = prof["corr_units"] / max(prof["corr_launches"], 1)
    corr_avg_ms = prof["corr_ms"] / max(prof["timed_launches"], 1)
    achieved = units_per_launch * flops_per_cell(N) / (corr_avg_ms / 1e3) / 1e12
    traffic = ncu_traffic(units_per_launch)
    hbm_bytes_step = S * 8 * (N / (N - len(wl.chips[0]) * wl.sps)) + len(wl.chips) * N * 8
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(), "samples_per_step_per_gpu": S,
                   "l2": "flushed before each step (256 MiB write), outside the timed events",
                   "parallelism": "replicas: one independent stream per GPU",
                   "detections_per_step": count},
        "code_bin_msamples_per_s": value * len(wl.chips) * len(wl.freqs_hz),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "k_corr_dif (inverse FFT + |.|^2 + floor/argmax per (window, code, bin))",
                     "units_per_launch": units_per_launch, "avg_launch_ms": corr_avg_ms,
                     "flops_per_unit": flops_per_cell(N),
                     "peak_note": PEAK_NOTE,
                     "kernel_share_of_step": prof["corr_ms"] / total_ms},
        "hbm": {"algorithmic_bytes_per_step": hbm_bytes_step,
                "achieved_gbs": hbm_bytes_step / (total_ms / args.steps / 1e3) / 1e9,
                "frac_of_measured": hbm_bytes_step / (total_ms / args.steps / 1e3) / 1e9 / 6699.8},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": S * 8,
                "d2h_bytes_per_step": 4 + 32 * min(n_host, cap)},
        "gpu_launches": prof["launches"],
        "clocks": clocks,
    }
    if not args.no_unfused:
        line["unfused_cufft_baseline"] = unfused_baseline(args, wl, x, st, flush, dev, torch, value)
    if world == 1 and not args.no_batching:
        # the batching row, clocked by the same run: 3 timed graph launches after 2 warm-ups
        r = measure_batching(dev, torch, 3, 2, args.capacity)
        line["batching"] = {"workload": BATCH_WORKLOAD, "value": r["value"], "unit": UNIT,
                            "ms_per_batch": r["ms_per_step"], "samples_per_batch": r["samples"],
                            "kernels_per_graph_launch": r["kernels_per_launch"],
                            "executed_tflops": r["tflops"], "frac_of_fp32_peak": r["tflops"] / FP32_PEAK_TFLOPS,
                            "detections_per_stream": r["counts"], "clocks": r["clocks"]}
    if world == 1 and not args.no_precision:
        # the reduced-precision row on the same workload shape: FP32 against the
        # FP16 / BF16 tensor-core correlation (3 timed runs each)
        res, n_tags = measure_precision(dev, torch, 3, 2, args.capacity)
        line["precision"] = {
            "workload": "precision: " + workload_name(), "unit": UNIT,
            "tag_cells": n_tags,
            "per_precision": {PRECISION_NAMES[p]: {k: r[k] for k in (
                "value", "k_corr_ms_per_launch", "speedup_vs_fp32", "detections", "fp32_detections_reproduced",
                "tag_cells_found", "max_score_rel_diff_vs_fp32", "max_toa_diff_vs_fp32")} for p, r in res.items()}}
    if world == 1 and not args.no_cpu_baseline:
        # about 15 s on 16 Arm host cores: 48 windows x every code and bin
        windows = tuple(range(1, 49))
        with oracle_pool(wl) as pool:
            dt, samples = oracle_sample(pool, wl, windows=windows)
            cores = pool.processes
        line["cpu_baseline"] = {"value": samples / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"windows 1-48 x 16 codes x 31 bins of the same stream (numpy FP64 oracle "
                                          f"on {cores} worker processes, {dt:.1f} s); Msamples/s = 48 hop / time"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
