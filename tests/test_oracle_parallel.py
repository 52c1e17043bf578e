"""The oracle's process-pool search gives exactly the single-process search:
the same detections in the same order and the same cells (CPU only)."""
from oracle import acq, parallel
from paper_2005_10445_gb300 import synth


def test_pool_equals_single_process():
    wl = synth.small(seed=12)
    want, want_cells = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len, keep_cells=True)
    got, cells, procs = parallel.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len, processes=2,
                                        chunk=2)
    assert procs == 2
    assert got == want and len(got) >= 3
    assert cells == want_cells


def test_all_pairs_order_and_ragged_code_lengths():
    chips = [synth.random_chips(600, 1), synth.random_chips(1100, 2)]
    pairs = parallel.all_pairs(60000, chips, 4)
    assert pairs == sorted(pairs)
    for c, ch in enumerate(chips):
        L = len(ch) * 4
        W, _ = acq.window_plan(60000, acq.default_fft_len(L), L)
        assert sorted(w for w, cc in pairs if cc == c) == list(range(W))
