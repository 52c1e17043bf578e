"""Host logic of bench.py, checked without a GPU: the algorithmic work per unit
behind `roofline.achieved`, the source-hash gating and per-launch scaling of the
committed ncu traffic, the name of a shortened stream, and the reference arm's
JSON line (the FP64 oracle on the host cores, printed by rank 0 alone)."""
import json
import os
import subprocess
import sys
import types

import numpy as np
import pytest

import bench
from oracle import acq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_work_per_unit_closed_forms():
    # 5 N log2 N + 6 N + 4 N at N = 2^17: 131072 x (5 x 17 + 10)
    assert bench.flops_per_cell(1 << 17) == 131072 * 95 == 12_451_840
    # half a complex transform plus 6 N at N = 2^18
    assert bench.fsk_corr_flops_per_cell(1 << 18) == 2.5 * 262144 * 18 + 6 * 262144 == 13_369_344
    # per demodulated sample at B = 4096, T = 207: (15 B log2 B + 12 B) / (B - T + 1) + 12
    B = 4096
    assert bench.fsk_demod_flops_per_sample(207) == pytest.approx((15 * B * 12 + 12 * B) / (B - 206) + 12)


def test_executed_flops_of_the_realistic_shape():
    """122 windows x 31 bins of 8 forward transforms of 2^14 points, and per
    (window, code, bin) 8 inverse ones plus 10 N: counted by hand."""
    wl = types.SimpleNamespace(chips=[np.ones(8192)] * 16, sps=8, fft_len=131072, n_samples=8_000_000,
                               freqs_hz=np.zeros(31))
    W, hop = acq.window_plan(8_000_000, 131072, 8192 * 8)
    assert (W, hop) == (122, 65536)
    fft = 8 * 5.0 * 16384 * 14
    assert bench.executed_flops(wl) == W * 31 * fft + W * 16 * 31 * (fft + 10.0 * 131072)


def _fields(path):
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    return vals


def test_search_traffic_scales_per_cell_and_follows_the_sources(monkeypatch):
    vals = _fields(os.path.join(ROOT, "profiles", "k_corr_realistic_traffic.txt"))
    cells = float(vals["cells_per_full_launch"])
    full = float(vals["dram_bytes_per_full_launch"])
    assert full == float(vals["dram_bytes_read_per_full_launch"]) + float(vals["dram_bytes_write_per_full_launch"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: vals["kernel_source_sha256_16"])
    assert bench.ncu_traffic(cells) == full
    assert bench.ncu_traffic(30256) == pytest.approx(full * 30256 / cells)
    # a capture taken on other kernel sources is not reported
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic(cells) is None


def test_fsk_traffic_follows_the_sources(monkeypatch):
    vals = _fields(os.path.join(ROOT, "profiles", "k_fsk_corr_traffic.txt"))
    per_cell = float(vals["dram_bytes_per_captured_launch"]) / float(vals["cells_per_captured_launch"])
    assert float(vals["dram_bytes_per_cell"]) == pytest.approx(per_cell)
    monkeypatch.setattr(bench, "fsk_kernel_source_hash", lambda: vals["kernel_source_sha256_16"])
    assert bench.fsk_ncu_traffic_per_cell() == pytest.approx(per_cell)
    monkeypatch.setattr(bench, "fsk_kernel_source_hash", lambda: "0" * 16)
    assert bench.fsk_ncu_traffic_per_cell() is None


def _cuh_closure(csrc, name, seen=None):
    """name and every .cuh it includes, directly or not."""
    seen = set() if seen is None else seen
    seen.add(name)
    for ln in open(os.path.join(csrc, name)):
        if ln.startswith('#include "'):
            inc = ln.split('"')[1]
            if inc.endswith(".cuh") and inc not in seen:
                _cuh_closure(csrc, inc, seen)
    return seen


def test_source_hashes_cover_the_kernels_they_gate(tmp_path, monkeypatch):
    """An edit of the gated kernel's file or of any .cuh it includes changes
    the hash (on a copy of the sources)."""
    import shutil
    csrc = os.path.join(ROOT, "paper_2005_10445_gb300", "csrc")
    copy = tmp_path / "paper_2005_10445_gb300" / "csrc"
    shutil.copytree(csrc, copy, ignore=shutil.ignore_patterns("*.o"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    for src, f in (("acq_fft_kernels.cuh", bench.kernel_source_hash), ("fsk_fft.cu", bench.fsk_kernel_source_hash)):
        names = _cuh_closure(csrc, src)
        assert len(names) >= 3, names
        h0 = f()
        for name in sorted(names):
            p = copy / name
            orig = p.read_bytes()
            p.write_bytes(orig + b"\n")
            assert f() != h0, (src, name)
            p.write_bytes(orig)
        assert f() == h0


def test_workload_name_of_a_shortened_stream(monkeypatch):
    assert bench.workload_name() == bench.WORKLOAD
    W, _ = acq.window_plan(2_000_000, 131072, 65536)
    monkeypatch.setattr(bench, "SECONDS", 0.25)
    name = bench.workload_name()
    assert "realistic, shortened: 0.25 s" in name and f"(hop 65536, {W} windows)" in name
    assert W == 30


def _run_reference(env_extra, timeout):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def test_reference_arm_json_line():
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1"}, 900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["higher_is_better"]) == (bench.METRIC, bench.UNIT, True)
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["steps"] == 1 and d["warmup"] >= 3  # at least three warm-up steps, whatever is asked
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] == (os.cpu_count() or 1) and cb["sample"]


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2"}, 120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
