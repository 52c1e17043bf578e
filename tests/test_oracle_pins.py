"""Pins for the FP64 oracle against facts fixed outside it: a hand-worked
example, closed forms, textbook identities, a library routine the oracle does
not use, brute force on tiny inputs, and planted mistakes that must be caught.
CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import acq
from paper_2005_10445_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = [float(t) for t in v]
    return out


# --- hand-worked example (tests/golden/hand_worked_example.txt) -------------

def test_hand_worked_example():
    g = _read_fixture("hand_worked_example.txt")
    N = int(g["N"][0])
    chips = np.array(g["chips"], dtype=np.int8)
    x = np.array(g["x_re"]) + 1j * np.array(g["x_im"])
    r = acq.replica(chips, int(g["sps"][0]), N)
    y = acq.mix(x, g["freqs"][0], g["fs"][0])
    want = np.array(g["corr_re"]) + 1j * np.array(g["corr_im"])
    np.testing.assert_allclose(acq.corr_direct(y, r, len(chips)), want, atol=1e-12)
    np.testing.assert_allclose(acq.corr_fft(y, r), want, atol=1e-12)
    dets, cells = acq.search(x, [chips], 1, g["fs"][0], g["freqs"], fft_len=N, threshold=2.0,
                             keep_cells=True)
    c = cells[(0, 0)][0]
    assert c.floor == pytest.approx(g["floor"][0], rel=1e-12)
    assert c.lag == int(g["lag"][0])
    assert len(dets) == 1
    d = dets[0]
    assert (d.code, d.window, d.lag, d.freq_bin) == (0, 0, 2, 0)
    assert d.score == pytest.approx(g["score"][0], rel=1e-12)
    assert d.toa == pytest.approx(g["toa"][0], abs=1e-12)
    assert d.peak_power == pytest.approx(g["peak_power"][0], rel=1e-12)


# --- bin selection ties (tests/golden/select_ties.txt) ----------------------

def test_select_ties_golden():
    g = _read_fixture("select_ties.txt")
    for case in "abc":
        v = g["case_" + case]
        cells = [acq.Cell(v[i], int(v[i + 1]), v[i + 2]) for i in range(0, len(v), 3)]
        k, s = acq.select(cells)
        want_k, want_s = g["want_" + case]
        assert k == int(want_k), case
        assert s == want_s, case


def test_duplicated_bins_select_the_first():
    """Two identical frequencies give identical cells; the search reports the
    smaller bin index (the hand-worked example's detection, at bin 0 of 2)."""
    g = _read_fixture("hand_worked_example.txt")
    chips = np.array(g["chips"], dtype=np.int8)
    x = np.array(g["x_re"]) + 1j * np.array(g["x_im"])
    dets, cells = acq.search(x, [chips], 1, g["fs"][0], [0.0, 0.0], fft_len=int(g["N"][0]), threshold=2.0,
                             keep_cells=True)
    assert len(dets) == 1 and dets[0].freq_bin == 0
    assert cells[(0, 0)][0] == cells[(0, 0)][1]


# --- refinement at the stream ends (tests/golden/refine_stream_end.txt) ------

def test_refine_stream_ends_golden():
    g = _read_fixture("refine_stream_end.txt")
    N, fs = int(g["N"][0]), g["fs"][0]
    chips = np.array(g["chips"], dtype=np.int8)
    for end in ("upper", "lower"):
        x = np.array(g[end + "_x"], dtype=np.complex128)
        dets, _ = acq.search(x, [chips], 1, fs, g["freqs"], fft_len=N, threshold=1.0)
        assert len(dets) == 1, end
        d = dets[0]
        assert d.lag == int(g[end + "_lag"][0]), end
        assert d.toa == g[end + "_toa"][0], end
    x = np.array(g["upper_x"], dtype=np.complex128)
    d = acq.search(x, [chips], 1, fs, g["freqs"], fft_len=N, threshold=1.0)[0][0]
    assert d.score == pytest.approx(g["upper_score"][0], rel=1e-15)
    assert d.peak_power == pytest.approx(g["upper_peak_power"][0], rel=1e-15)
    assert acq.parabolic_offset(*g["interior_p"]) == pytest.approx(g["interior_delta"][0], rel=1e-15)


# --- windowing: every start lag searched exactly once (Section 2.1) --------

@pytest.mark.parametrize("S,N,L", [(16384, 16384, 2046), (8_000_000, 131072, 65536), (40000, 8192, 2400),
                                   (5000, 4096, 1000), (4096, 4096, 1000), (1000, 4096, 1000),
                                   (1001, 4096, 1000), (7000, 4096, 3000), (9, 8, 3)])
def test_every_lag_once(S, N, L):
    W, hop = acq.window_plan(S, N, L)
    seen = np.zeros(S - L + 1, dtype=np.int64)
    for w in range(W):
        nv = acq.n_valid_lags(w, W, S, N, L)
        assert 1 <= nv <= hop + 1
        a = w * hop + np.arange(nv)
        assert a.max() + L - 1 < w * hop + N  # the code fits in the window
        seen[a] += 1
    assert (seen == 1).all()


def test_window_plan_workload_sizes():
    assert acq.window_plan(16384, 16384, 2046) == (1, 14338)
    assert acq.n_valid_lags(0, 1, 16384, 16384, 2046) == 14339
    W, hop = acq.window_plan(8_000_000, 131072, 65536)
    assert (W, hop) == (122, 65536)
    assert acq.n_valid_lags(121, W, 8_000_000, 131072, 65536) == 4609


# --- closed forms -----------------------------------------------------------

def test_autocorrelation_peak_equals_code_length():
    """A noise-free unit code at lag d, f = 0: corr[d] = L exactly; all other
    valid lags are smaller in magnitude."""
    chips = synth.random_chips(300, 7)
    sps, N = 4, 4096
    L = 300 * sps
    d = 517
    x = np.zeros(N, dtype=np.complex128)
    x[d:d + L] = np.repeat(chips.astype(np.float64), sps)
    c = acq.corr_fft(acq.mix(x, 0.0, 1e6), acq.replica(chips, sps, N))
    assert c[d] == pytest.approx(L, abs=1e-9)
    others = np.delete(np.abs(c[: N - L + 1]), d)
    assert others.max() < L - sps / 2
    # mainlobe: one sample off the peak the overlap loses 1/sps of each chip
    assert abs(c[d + 1]) == pytest.approx(L * (1 - 1 / sps), abs=1e-6 * L) or \
        abs(c[d + 1]) < L * (1 - 1 / sps) + 1e-6 * L


def test_m_sequence_periodic_autocorrelation():
    """The LFSR stand-in code is an m-sequence: periodic autocorrelation 1023
    at shift 0 and -1 at every other shift (textbook property)."""
    c = synth.lfsr_chips(1).astype(np.int64)
    ac = np.array([int(np.dot(c, np.roll(c, k))) for k in range(1023)])
    assert ac[0] == 1023 and (ac[1:] == -1).all()


@pytest.mark.parametrize("f", [0.0, 1250.0, -3000.0])
def test_delta_input_gives_reversed_code(f):
    """x = delta at p: corr[tau] = exp(-j 2 pi f p / fs) * r[(p - tau) mod N].
    Catches correlation-vs-convolution, lag direction and the mix sign."""
    chips = np.array([1, -1, -1, 1, 1, 1, -1], dtype=np.int8)
    sps, N, fs, p = 3, 64, 48000.0, 40
    x = np.zeros(N, dtype=np.complex128)
    x[p] = 1.0
    r = acq.replica(chips, sps, N)
    want = np.exp(-2j * np.pi * f * p / fs) * r[(p - np.arange(N)) % N]
    y = acq.mix(x, f, fs)
    np.testing.assert_allclose(acq.corr_fft(y, r), want, atol=1e-12)
    np.testing.assert_allclose(acq.corr_direct(y, r, len(chips) * sps), want, atol=1e-12)


def test_dft_textbook_delta_and_tone():
    N = 256
    d = np.zeros(N, complex)
    d[0] = 1
    np.testing.assert_allclose(np.fft.fft(d), np.ones(N), atol=1e-13)
    k0 = 37
    tone = np.exp(2j * np.pi * k0 * np.arange(N) / N)
    X = np.fft.fft(tone)
    assert abs(X[k0] - N) < 1e-9 and np.abs(np.delete(X, k0)).max() < 1e-9


def test_tag_on_bin_closed_form_power():
    """A noise-free tag of amplitude A exactly on bin b of an asymmetric grid:
    detected at (code, lag, bin b) with P* = (A L)^2.  A flipped mix sign would
    pull the tag to -f, which is not on this grid."""
    chips = synth.random_chips(256, 3)
    sps, N, fs = 2, 2048, 1e6
    L = 512
    freqs = np.array([-4000.0, 0.0, 1500.0, 6000.0])
    x = np.zeros(N, dtype=np.complex64)
    tag = synth.Tag(code=0, delay=700.0, freq_hz=1500.0, bin=2, snr_db=0.0, phase=0.3)
    A = 3.0
    synth.inject(x, chips, sps, fs, tag, 1.0, amplitude=A)
    dets, cells = acq.search(x, [chips], sps, fs, freqs, fft_len=N, keep_cells=True)
    assert [d.key() for d in dets] == [(0, 0, 700, 2)]
    assert cells[(0, 0)][2].p_max == pytest.approx((A * L) ** 2, rel=1e-6)
    assert dets[0].toa == pytest.approx(700.0, abs=1e-6)


def test_parseval_floor():
    """mean_tau |corr|^2 = sum_m |Y_m|^2 |R_m|^2 / N^2 (Parseval), and the FFT
    keeps energy: sum|x|^2 = sum|X|^2 / N."""
    rng = np.random.default_rng(5)
    N = 1024
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    assert np.sum(np.abs(x) ** 2) == pytest.approx(np.sum(np.abs(np.fft.fft(x)) ** 2) / N, rel=1e-12)
    chips = synth.random_chips(50, 9)
    r = acq.replica(chips, 4, N)
    y = acq.mix(x, 777.0, 1e5)
    _, _, floor = acq.cell_stats(acq.corr_fft(y, r), 10)
    Y, R = np.fft.fft(y), np.fft.fft(r)
    assert floor == pytest.approx(np.sum(np.abs(Y) ** 2 * np.abs(R) ** 2) / N ** 2, rel=1e-12)


def test_library_correlate_special_case():
    """f = 0 and lags whose code span does not wrap: corr equals
    numpy.correlate(x, r, 'valid') (a routine the oracle does not use)."""
    rng = np.random.default_rng(8)
    N, sps = 512, 3
    chips = synth.random_chips(40, 1)
    L = 40 * sps
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    c = acq.corr_fft(acq.mix(x, 0.0, 1.0), acq.replica(chips, sps, N))
    want = np.correlate(x, np.repeat(chips.astype(float), sps), "valid")
    np.testing.assert_allclose(c[: N - L + 1], want, rtol=1e-11, atol=1e-9)


def test_brute_force_tiny_search():
    """Pure-Python loops over every (window, code, bin, lag) on a tiny ragged
    stream give the same detections as the oracle's FFT route."""
    rng = np.random.default_rng(21)
    sps, N, fs = 2, 32, 1000.0
    chip_sets = [np.array([1, -1, 1, 1, -1], np.int8), np.array([-1, -1, 1, -1, 1, 1], np.int8)]
    freqs = [-60.0, 0.0, 45.0]
    S = 75
    x = (rng.standard_normal(S) + 1j * rng.standard_normal(S)) * 0.3
    x[9:19] += np.repeat(chip_sets[0], sps) * np.exp(2j * np.pi * 45.0 * np.arange(9, 19) / fs)
    x[50:62] += np.repeat(chip_sets[1], sps) * np.exp(-2j * np.pi * 60.0 * np.arange(50, 62) / fs)
    got, _ = acq.search(x, chip_sets, sps, fs, freqs, fft_len=N, threshold=3.0)
    # brute force
    want = []
    for c, ch in enumerate(chip_sets):
        L = len(ch) * sps
        hop = N - L
        W = max(1, math.ceil((S - N) / hop) + 1)
        rep = [float(ch[n // sps]) for n in range(L)]
        for w in range(W):
            nv = hop if w < W - 1 else min(hop, S - L - w * hop) + 1
            best = None
            for k, f in enumerate(freqs):
                P = []
                for tau in range(N):
                    acc = 0j
                    for n in range(L):
                        m = (tau + n) % N
                        xm = x[w * hop + m] if w * hop + m < S else 0j
                        acc += xm * complex(math.cos(-2 * math.pi * f * m / fs),
                                            math.sin(-2 * math.pi * f * m / fs)) * rep[n]
                    P.append(abs(acc) ** 2)
                floor = sum(P) / N
                t = max(range(nv), key=lambda i: (P[i], -i))
                s = P[t] / floor
                if best is None or s > best[0]:
                    best = (s, k, t)
            if best[0] >= 3.0:
                want.append((c, w, best[2], best[1], best[0]))
    want.sort(key=lambda t: (t[1], t[0]))
    assert [d.key() for d in got] == [t[:4] for t in want]
    for d, t in zip(got, want):
        assert d.score == pytest.approx(t[4], rel=1e-10)
    assert len(got) >= 2


# --- interpolation -----------------------------------------------------------

@pytest.mark.parametrize("t0", [-0.5, -0.31, 0.0, 0.12, 0.49])
def test_parabolic_vertex_exact(t0):
    P = [7.0 - 2.5 * (t - t0) ** 2 for t in (-1, 0, 1)]
    assert acq.parabolic_offset(*P) == pytest.approx(t0, abs=1e-12)


def test_parabolic_degenerate_cases():
    assert acq.parabolic_offset(1.0, 1.0, 1.0) == 0.0      # flat
    assert acq.parabolic_offset(2.0, 1.0, 2.0) == 0.0      # a minimum
    assert acq.parabolic_offset(0.0, 1.0, 1.5) == 0.5      # vertex past +1/2: clamp
    assert acq.parabolic_offset(1.5, 1.0, 0.0) == -0.5


def test_fractional_delay_toa_direction():
    """A noise-free tag at a fractional delay: the refined ToA moves toward
    the truth from the integer peak and lands within 0.15 samples (the
    parabola on |corr|^2 of a rectangular-chip code is a biased estimator)."""
    chips = synth.random_chips(500, 4)
    sps, N, fs = 8, 8192, 8e6
    for frac in (0.2, 0.35, 0.65):
        x = np.zeros(N, dtype=np.complex64)
        tag = synth.Tag(0, 1000 + frac, 0.0, 0, 0.0, 0.0)
        synth.inject(x, chips, sps, fs, tag, 1.0, amplitude=1.0)
        dets, _ = acq.search(x, [chips], sps, fs, [0.0], fft_len=N)
        assert len(dets) == 1
        assert abs(dets[0].toa - (1000 + frac)) < 0.15
        assert abs(dets[0].toa - (1000 + frac)) < abs(dets[0].lag - (1000 + frac))


def test_direct_power_equals_window_peak():
    wl = synth.small()
    dets, cells = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len, keep_cells=True)
    for d in dets:
        c = cells[(d.window, d.code)][d.freq_bin]
        assert d.peak_power == pytest.approx(c.p_max, rel=1e-9)


# --- injected tags ----------------------------------------------------------

def _expected_keys(wl):
    out = []
    for t in wl.tags:
        L = len(wl.chips[t.code]) * wl.sps
        N = wl.fft_len or acq.default_fft_len(L)
        W, hop = acq.window_plan(wl.n_samples, N, L)
        d = int(t.delay)
        w = min(d // hop, W - 1)
        out.append((t.code, w, d - w * hop, t.bin))
    return sorted(out, key=lambda k: (k[1], k[0]))


@pytest.mark.parametrize("maker", [synth.tiny, synth.small])
def test_injected_tags_recovered(maker):
    wl = maker()
    dets, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    assert [d.key() for d in dets] == _expected_keys(wl)
    for d in dets:
        t = [t for t in wl.tags if t.code == d.code and abs(t.delay - d.toa) < 1][0]
        assert abs(d.toa - t.delay) < 0.1
        L = len(wl.chips[d.code]) * wl.sps
        assert d.score > 0.3 * (L * 10 ** (t.snr_db / 10))


def test_noise_free_tags_exact_toa():
    """One code, noise-free integer-delay tags: exact keys and toa = delay.
    On a bin centre the peak is symmetric and delta = 0 exactly (see
    test_tag_on_bin_closed_form_power); the +/-20 Hz carrier jitter here makes
    it slightly asymmetric, a few thousandths of a sample."""
    wl = synth.small(n_codes=1, n_tags=3, snr_range=(0.0, 0.0), sigma=1e-9)
    dets, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    assert [d.key() for d in dets] == _expected_keys(wl)
    for d in dets:
        t = [t for t in wl.tags if t.code == d.code and abs(t.delay - d.toa) < 1][0]
        assert d.toa == pytest.approx(t.delay, abs=0.02)


def test_score_is_scale_invariant():
    wl = synth.small()
    a, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    b, _ = acq.search(wl.x * np.float32(32.0), wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    assert [d.key() for d in a] == [d.key() for d in b]
    for p, q in zip(a, b):
        assert p.score == pytest.approx(q.score, rel=1e-9)
        assert p.toa == pytest.approx(q.toa, abs=1e-9)


# --- planted mistakes: each one must trip a pin above -----------------------

def _mutants():
    def no_conj(y, r):
        return np.fft.ifft(np.fft.fft(y) * np.fft.fft(r))

    def mix_plus(xw, f, fs):
        m = np.arange(xw.shape[0], dtype=np.float64)
        return xw * np.exp(2j * np.pi * (f / fs) * m)

    def floor_valid_only(corr, nv):
        P = np.abs(corr) ** 2
        t = int(np.argmax(P[:nv]))
        return float(P[t]), t, float(P[:nv].mean())

    def last_tie(corr, nv):
        P = np.abs(corr) ** 2
        t = nv - 1 - int(np.argmax(P[:nv][::-1]))
        return float(P[t]), t, float(P.mean())

    def drop_last_chip(chips, sps, N):
        r = np.zeros(N)
        L = len(chips) * sps
        r[: L - sps] = np.repeat(np.asarray(chips[:-1], float), sps)
        return r

    def sign_flipped_vertex(pm, p0, pp):
        den = pm - 2 * p0 + pp
        if not den < 0:
            return 0.0
        return min(0.5, max(-0.5, 0.5 * (pp - pm) / den))

    def larger_bin_on_ties(cells):
        best_k, best_s = 0, -1.0
        for k, c in enumerate(cells):
            s = c.p_max / c.floor if c.floor > 0 else 0.0
            if s >= best_s:
                best_k, best_s = k, s
        return best_k, best_s

    def no_upper_stream_end(x, chips, sps, f_hz, fs_hz, a):
        p0 = acq.direct_power(x, chips, sps, f_hz, fs_hz, a)
        if a - 1 < 0:
            return float(a), p0
        pm = acq.direct_power(x, chips, sps, f_hz, fs_hz, a - 1)
        pp = acq.direct_power(x, chips, sps, f_hz, fs_hz, a + 1)
        return float(a) + acq.parabolic_offset(pm, p0, pp), p0

    return [("corr_fft", no_conj), ("mix", mix_plus), ("cell_stats", floor_valid_only),
            ("cell_stats", last_tie), ("replica", drop_last_chip),
            ("parabolic_offset", sign_flipped_vertex), ("select", larger_bin_on_ties),
            ("refine", no_upper_stream_end)]


PINS = [test_hand_worked_example,
        lambda: test_delta_input_gives_reversed_code(1250.0),
        test_tag_on_bin_closed_form_power, test_parseval_floor,
        test_autocorrelation_peak_equals_code_length, test_brute_force_tiny_search,
        lambda: test_parabolic_vertex_exact(0.12), test_fractional_delay_toa_direction,
        test_select_ties_golden, test_duplicated_bins_select_the_first, test_refine_stream_ends_golden]


@pytest.mark.parametrize("name,fn", _mutants(), ids=[f"{n}:{f.__name__}" for n, f in _mutants()])
def test_planted_mistake_is_caught(monkeypatch, name, fn):
    if name == "parabolic_offset":
        monkeypatch.setattr(acq, name, fn)
        with pytest.raises(AssertionError):
            test_parabolic_vertex_exact(0.12)
        return
    monkeypatch.setattr(acq, name, fn)
    failed = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1
