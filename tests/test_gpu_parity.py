"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Bar: detections (code, window, lag, freq_bin) identical; ToA within 1e-3
samples; score and peak power within 1e-4 relative (FP32 FFT path against
FP64).  Per-cell statistics: floor and P* within 1e-4 relative, and the lag
identical unless the oracle's own top two lags are within the tolerance (then
the GPU lag must be one of the oracle's near-maximal lags).
"""
import numpy as np
import pytest

from oracle import acq
from paper_2005_10445_gb300 import synth

pytestmark = pytest.mark.gpu

SCORE_RTOL = 1e-4
TOA_ATOL = 1e-3
CELL_RTOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_search(torch, wl, threshold=25.0, capacity=4096, cells=False, **kw):
    from paper_2005_10445_gb300.binding import Search
    s = Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, threshold=threshold, fft_len=wl.fft_len, **kw)
    x = torch.from_numpy(wl.iq().copy()).cuda()
    dets, n, cell = s.run(x, capacity=capacity, cells=cells)
    return s, dets, n, cell


def compare_detections(gpu, ora):
    g_keys = [(int(d["code"]), int(d["window"]), int(d["lag"]), int(d["freq_bin"])) for d in gpu]
    o_keys = [d.key() for d in ora]
    assert sorted(g_keys) == sorted(o_keys)
    by = {d.key(): d for d in ora}
    for d in gpu:
        o = by[(int(d["code"]), int(d["window"]), int(d["lag"]), int(d["freq_bin"]))]
        assert d["score"] == pytest.approx(o.score, rel=SCORE_RTOL)
        assert d["peak_power"] == pytest.approx(o.peak_power, rel=SCORE_RTOL)
        assert abs(d["toa"] - o.toa) <= TOA_ATOL


def compare_cells(torch, wl, gpu_cells, pairs):
    x = wl.x.astype(np.complex128)
    for (w, c) in pairs:
        L = len(wl.chips[c]) * wl.sps
        N = wl.fft_len or acq.default_fft_len(L)
        W, hop = acq.window_plan(wl.n_samples, N, L)
        nv = acq.n_valid_lags(w, W, wl.n_samples, N, L)
        xw = acq.window_samples(x, w, hop, N)
        r = acq.replica(wl.chips[c], wl.sps, N)
        for k, f in enumerate(wl.freqs_hz):
            corr = acq.corr_fft(acq.mix(xw, float(f), wl.fs_hz), r)
            P = np.abs(corr) ** 2
            g = gpu_cells[w, c, k]
            assert g["valid"] == 1
            assert g["floor"] == pytest.approx(P.mean(), rel=CELL_RTOL)
            tau = int(np.argmax(P[:nv]))
            assert g["p_max"] == pytest.approx(P[tau], rel=CELL_RTOL)
            if int(g["lag"]) != tau:
                # only acceptable when the oracle itself cannot separate the two lags
                assert 0 <= int(g["lag"]) < nv
                assert P[int(g["lag"])] >= P[tau] * (1 - CELL_RTOL), (w, c, k, int(g["lag"]), tau)


def test_tiny_parity(torch_cuda):
    wl = synth.tiny()
    s, dets, n, cells = gpu_search(torch_cuda, wl, cells=True)
    ora, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    assert n == len(ora) == 1
    compare_detections(dets, ora)
    compare_cells(torch_cuda, wl, cells, [(0, 0)])
    assert s.device_status() == 0


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_small_parity_all_cells(torch_cuda, seed):
    """Several windows with a ragged, zero-padded last window, 3 codes,
    5 bins, sps 4, N = 8192 (M = 2048)."""
    wl = synth.small(seed=seed)
    s, dets, n, cells = gpu_search(torch_cuda, wl, cells=True)
    ora, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    assert n == len(ora) >= 3
    compare_detections(dets, ora)
    W = cells.shape[0]
    compare_cells(torch_cuda, wl, cells, [(w, c) for w in range(W) for c in range(len(wl.chips))])
    # detections come out ordered by (window, code)
    keys = [(int(d["window"]), int(d["code"])) for d in dets]
    assert keys == sorted(keys)


@pytest.mark.parametrize("n_chips,sps,N", [
    (400, 1, 1024),      # M = 2^10, no box sum
    (500, 2, 2048),      # M = 2^10
    (900, 4, 8192),      # M = 2^11
    (700, 8, 16384),     # M = 2^11, sps 8
    (1500, 2, 8192),     # M = 2^12
    (3000, 4, 32768),    # M = 2^13
    (5000, 2, 32768),    # M = 2^14
    (8192, 8, 131072),   # M = 2^14, sps 8 (the realistic code shape)
    (600, 16, 16384),    # M = 2^10, sps 16
    (16384, 2, 65536),   # M = 2^15: split (two-block) transforms
    (9000, 4, 131072),   # M = 2^15, sps 4
])
def test_sizes_parity(torch_cuda, n_chips, sps, N):
    """Every transform size, both tile shapes (16 and 32 values per thread) and,
    for 2^14 points, both the one-block and the two-block transforms, against
    the oracle cell by cell."""
    L = n_chips * sps
    S = 2 * N + 3 * (N - L) // 2 + 17   # ragged last window
    wl = synth.realistic(seed=n_chips + sps, seconds=S / 4e6, n_codes=2, n_chips=n_chips, sps=sps,
                         fs_hz=4e6, n_tags=2, snr_range=(-8.0, -2.0),
                         freqs_hz=np.array([-2500.0, 0.0, 2500.0]), min_same_code_gap=2 * N, fft_len=N)
    ora, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    shapes = [(5, 0), (4, 0)] + ([(5, 1), (4, 1)] if N // sps == 1 << 14 else [])
    for tile, split in shapes:
        s, dets, n, cells = gpu_search(torch_cuda, wl, cells=True, tile_log2=tile, split=split)
        assert n == len(ora)
        compare_detections(dets, ora)
        W = cells.shape[0]
        pairs = [(w, c) for w in range(W) for c in range(2)]
        if N >= 65536:
            pairs = pairs[:2] + pairs[-2:]
        compare_cells(torch_cuda, wl, cells, pairs)


def test_stream_of_exactly_one_code(torch_cuda):
    """S = L: one window with the single valid lag 0."""
    chips = synth.random_chips(1000, 5)
    sps, N, fs = 2, 4096, 2e6
    x = synth.awgn(2000, 1.0, np.random.default_rng(0))
    tag = synth.Tag(0, 0.0, 0.0, 0, 10.0, 0.0)
    synth.inject(x, chips, sps, fs, tag, 1.0)
    wl = synth.Workload("exact", x, [chips], sps, fs, np.array([0.0, 700.0]), N, [tag], 1.0)
    s, dets, n, cells = gpu_search(torch_cuda, wl, cells=True)
    ora, _ = acq.search(wl.x, wl.chips, sps, fs, wl.freqs_hz, N)
    assert n == len(ora) == 1
    compare_detections(dets, ora)
    assert int(dets[0]["lag"]) == 0 and dets[0]["toa"] == 0.0
    compare_cells(torch_cuda, wl, cells, [(0, 0)])


def test_mixed_code_lengths(torch_cuda):
    """Codes of two lengths form two groups with their own windows."""
    rng = np.random.default_rng(3)
    fs, sps = 4e6, 4
    chips = [synth.random_chips(600, 1), synth.random_chips(1100, 2), synth.random_chips(600, 3)]
    S = 60000
    x = synth.awgn(S, 2048.0, rng)
    tags = [synth.Tag(0, 5000.0, 1500.0, 2, -5.0, 0.1), synth.Tag(1, 21000.0, -1500.0, 0, -6.0, 1.0),
            synth.Tag(2, 40000.0, 0.0, 1, -4.0, 2.0)]
    for t in tags:
        synth.inject(x, chips[t.code], sps, fs, t, 2048.0)
    wl = synth.Workload("mixed", x, chips, sps, fs, np.array([-1500.0, 0.0, 1500.0]), 0, tags, 2048.0)
    s, dets, n, cells = gpu_search(torch_cuda, wl, cells=True)
    ora, _ = acq.search(wl.x, wl.chips, sps, fs, wl.freqs_hz, 0)
    assert n == len(ora) == 3
    compare_detections(dets, ora)


def test_duplicated_bins_tie_to_the_smaller_bin(torch_cuda):
    """Every frequency of the tiny workload listed twice: each pair of bins
    gives identical cells, so every score ties and the detection must name the
    first copy (Section 3 step 8: one argmax, ties to the smaller bin)."""
    wl = synth.tiny()
    f = np.repeat(wl.freqs_hz, 2)
    dup = synth.Workload("tiny, bins doubled", wl.x, wl.chips, wl.sps, wl.fs_hz, f, wl.fft_len, wl.tags, wl.sigma)
    s, dets, n, cells = gpu_search(torch_cuda, dup, cells=True)
    ora, _ = acq.search(dup.x, dup.chips, dup.sps, dup.fs_hz, dup.freqs_hz, dup.fft_len)
    assert n == len(ora) == 1
    compare_detections(dets, ora)
    assert int(dets[0]["freq_bin"]) % 2 == 0
    assert cells[0, 0, 0::2].tobytes() == cells[0, 0, 1::2].tobytes()


def test_capacity_overflow_reports_full_count(torch_cuda):
    wl = synth.small(seed=12)
    s, full, n_full, _ = gpu_search(torch_cuda, wl)
    assert n_full >= 3
    s2, part, n_part, _ = gpu_search(torch_cuda, wl, capacity=2)
    assert n_part == n_full and len(part) == 2
    assert part.tobytes() == full[:2].tobytes()


def test_repeat_runs_bit_identical(torch_cuda):
    wl = synth.small(seed=13)
    from paper_2005_10445_gb300.binding import Search
    s = Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len)
    x = torch_cuda.from_numpy(wl.iq().copy()).cuda()
    a = s.run(x, cells=True)
    b = s.run(x, cells=True)
    assert a[0].tobytes() == b[0].tobytes() and a[2].tobytes() == b[2].tobytes()


@pytest.mark.parametrize("case", ["one group", "groups of one window", "mixed code lengths"])
def test_host_buffer_entry_matches_device(torch_cuda, case):
    """The host-buffer entry copies the first launch group's samples on the
    caller's stream and the rest on a copy stream that the later groups (and
    other code-length groups) wait for: its records equal the device entry's,
    also when the stream spans several launch groups and several code
    lengths, and when it runs twice in a row on the same staging buffer."""
    from paper_2005_10445_gb300.binding import Search
    kw = {}
    if case == "mixed code lengths":
        wl = synth.batch(seed=3)[6]
        wl = synth.Workload(wl.name, wl.x[: 600_000], wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len,
                            [t for t in wl.tags if t.delay + len(wl.chips[t.code]) * wl.sps <= 600_000], wl.sigma)
    else:
        wl = synth.small(seed=11)
        if case == "groups of one window":
            kw["windows_per_launch"] = 1
    s = Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len, **kw)
    x = torch_cuda.from_numpy(wl.iq().copy()).cuda()
    d_dev, n_dev, _ = s.run(x)
    for _ in range(2):
        d_host, n_host = s.run_host(wl.iq())
        assert n_dev == n_host and d_dev.tobytes() == d_host.tobytes()


def test_windows_per_launch_does_not_change_results(torch_cuda):
    wl = synth.small(seed=12)
    _, a, na, ca = gpu_search(torch_cuda, wl, cells=True, windows_per_launch=1)
    _, b, nb, cb = gpu_search(torch_cuda, wl, cells=True, windows_per_launch=3)
    assert na == nb and a.tobytes() == b.tobytes() and ca.tobytes() == cb.tobytes()


def test_selection_forms_agree(torch_cuda):
    """Launch groups of one window (pairs selected by the one-block kernel)
    and of every window (the many-block kernel and the ordered compaction):
    the same records in (window, code) order, at threshold 0 (every pair)."""
    wl = synth.small(seed=14)
    _, a, na, _ = gpu_search(torch_cuda, wl, threshold=0.0, windows_per_launch=1)
    _, b, nb, _ = gpu_search(torch_cuda, wl, threshold=0.0)
    assert na == nb > 16 and a.tobytes() == b.tobytes()
    keys = [(int(d["window"]), int(d["code"])) for d in b]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_short_stream_rejected(torch_cuda):
    from paper_2005_10445_gb300.binding import AtlasError, Search
    wl = synth.small()
    s = Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len)
    x = torch_cuda.zeros((100, 2), dtype=torch_cuda.float32, device="cuda")
    with pytest.raises(AtlasError):
        s.run(x)


def compare_all_cells(wl, gpu_cells, ora_cells):
    """Every (window, code, bin) cell the oracle computed: floor and P* within
    CELL_RTOL; the lag identical, or (checked by the caller with
    near_tie_ok) one the oracle itself cannot separate from its own."""
    differ = []
    for (w, c), cells in ora_cells.items():
        for k, o in enumerate(cells):
            g = gpu_cells[w, c, k]
            assert g["valid"] == 1, (w, c, k)
            assert g["floor"] == pytest.approx(o.floor, rel=CELL_RTOL), (w, c, k)
            assert g["p_max"] == pytest.approx(o.p_max, rel=CELL_RTOL), (w, c, k)
            if int(g["lag"]) != o.lag:
                differ.append((w, c, k, int(g["lag"]), o))
    return differ


def near_tie_ok(wl, differ):
    """A GPU lag that differs from the oracle's must be a valid lag whose FP64
    power is within CELL_RTOL of the oracle's maximum."""
    x = wl.x.astype(np.complex128)
    for (w, c, k, g_lag, o) in differ:
        L = len(wl.chips[c]) * wl.sps
        N = wl.fft_len or acq.default_fft_len(L)
        W, hop = acq.window_plan(wl.n_samples, N, L)
        nv = acq.n_valid_lags(w, W, wl.n_samples, N, L)
        corr = acq.corr_fft(acq.mix(acq.window_samples(x, w, hop, N), float(wl.freqs_hz[k]), wl.fs_hz),
                            acq.replica(wl.chips[c], wl.sps, N))
        P = np.abs(corr) ** 2
        assert 0 <= g_lag < nv
        assert P[g_lag] >= o.p_max * (1 - CELL_RTOL), (w, c, k, g_lag, o.lag)


def test_realistic_full_size_all_pairs(torch_cuda):
    """1 s at 8 MS/s, 16 codes x 8192 chips at sps 8, 31 bins, 40 tags -- the
    benchmark's workload and launch configuration.  The oracle (on every host
    core) searches all 1952 (window, code) pairs; every detection and every one
    of the 60,512 (window, code, bin) cells is compared."""
    from oracle import parallel
    wl = synth.realistic()
    s, dets, n, cells = gpu_search(torch_cuda, wl, cells=True)
    assert n == len(dets)
    W, hop, N = s.windows(0, wl.n_samples)
    ora, ora_cells, procs = parallel.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    assert len(ora_cells) == W * len(wl.chips) == 1952
    compare_detections(dets, ora)
    near_tie_ok(wl, compare_all_cells(wl, cells, ora_cells))
    # every injected tag is found
    found = {(int(d["code"]), int(d["window"]) * hop + int(d["lag"])) for d in dets}
    for t in wl.tags:
        assert (t.code, int(t.delay)) in found
    print(f"all pairs: {len(ora)} detections, {len(ora_cells) * len(wl.freqs_hz)} cells, oracle on {procs} processes")


def test_all_zero_stream_has_no_detections(torch_cuda):
    """Degenerate input: every power and floor is zero; the score is defined as
    0 (no division by zero), nothing is detected, every cell is finite."""
    from paper_2005_10445_gb300.binding import Search
    wl = synth.small(seed=11)
    s = Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len)
    x = torch_cuda.zeros((wl.n_samples, 2), dtype=torch_cuda.float32, device="cuda")
    dets, n, cells = s.run(x, cells=True)
    assert n == 0
    assert np.isfinite(cells["floor"]).all() and (cells["floor"] == 0).all()
    assert (cells["valid"] == 1).all()


def test_outputs_stay_inside_caller_buffers(torch_cuda):
    """Canary bytes after the detection buffer and after the cell buffer are
    untouched when the detections overflow the capacity."""
    from paper_2005_10445_gb300.binding import Search
    wl = synth.small(seed=12)
    s = Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len)
    x = torch_cuda.from_numpy(wl.iq().copy()).cuda()
    cap = 1
    canary = 4096
    out = torch_cuda.full((cap * 32 + canary,), 0xA5, dtype=torch_cuda.uint8, device="cuda")
    nw = s.max_windows(wl.n_samples)
    ncell = nw * len(wl.chips) * len(wl.freqs_hz) * 16
    cells = torch_cuda.full((ncell + canary,), 0x5A, dtype=torch_cuda.uint8, device="cuda")
    cnt = torch_cuda.zeros(1, dtype=torch_cuda.int32, device="cuda")
    st = torch_cuda.cuda.current_stream()
    s.run_cells_ptr(st.cuda_stream, x.data_ptr(), wl.n_samples, cells.data_ptr(), out.data_ptr(), cap, cnt.data_ptr())
    st.synchronize()
    assert int(cnt.item()) >= 3
    assert (out[cap * 32:].cpu().numpy() == 0xA5).all()
    assert (cells[ncell:].cpu().numpy() == 0x5A).all()
