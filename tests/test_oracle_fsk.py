"""Pins for the FP64 FSK oracle against facts fixed outside it: a hand-worked
example, closed forms of the matched filters and of a noise-free tag,
invariants (amplitude, Parseval), brute force on a tiny stream, and planted
mistakes that must be caught.  CPU only."""
import cmath
import math
import os

import numpy as np
import pytest

from oracle import acq, fsk
from paper_2005_10445_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fixture(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, *v = line.split()
                out[k] = [float(t) for t in v]
    return out


# --- hand-worked example (tests/golden/fsk_hand_worked.txt) -----------------

def test_hand_worked_example():
    g = _fixture("fsk_hand_worked.txt")
    fs, sps, f1, f0 = g["fs"][0], int(g["sps"][0]), g["f1"][0], g["f0"][0]
    g1, g0 = fsk.filters(np.array(g["h_bp"]), f1, f0, sps, fs)
    np.testing.assert_allclose(g1, np.array(g["g1_re"]) + 1j * np.array(g["g1_im"]), atol=1e-15)
    np.testing.assert_allclose(g0, np.array(g["g0_re"]) + 1j * np.array(g["g0_im"]), atol=1e-15)
    x = np.array(g["x_re"]) + 1j * np.array(g["x_im"])
    d, u = fsk.demod_range(x, g1, g0, 0, 4)
    np.testing.assert_allclose(d, g["d"], atol=1e-14)
    np.testing.assert_allclose(u, g["u"], atol=1e-14)
    dc, _ = fsk.code_demod(np.array(g["chips"], np.int8), sps, f1, f0, fs, g1, g0)
    np.testing.assert_allclose(dc, g["dc"], atol=1e-14)


# --- steps 1-2 ---------------------------------------------------------------

def test_int16_conversion_exact():
    iq = np.array([[-32768, 32767], [0, -1], [5, 7]], dtype=np.int16)
    x = fsk.iq_to_complex(iq)
    assert list(x) == [complex(-32768, 32767), complex(0, -1), complex(5, 7)]


@pytest.mark.parametrize("start", [0, 12345])
def test_lo_mix_brings_the_band_centre_to_zero(start):
    fs, f_lo = 8e6, 1.25e6
    i = start + np.arange(64)
    x = np.exp(2j * np.pi * f_lo * i / fs)
    np.testing.assert_allclose(fsk.lo_mix(x, f_lo, fs, start), np.ones(64), atol=1e-9)


# --- steps 3-5: matched filters ------------------------------------------------

@pytest.mark.parametrize("sps,fs", [(2, 2e6), (4, 4e6), (8, 8e6)])
def test_matched_filter_closed_form(sps, fs):
    """One chip of tone f1 (identity band-pass filter): at the chip's last
    sample |f1| = sps and |f0| = 0, since the tones +/-500 kHz are orthogonal
    over a chip of 1 us; so d = 1 and u = sps.  Chip -1 gives d = -1."""
    f1, f0 = 5e5, -5e5
    g1, g0 = fsk.filters(np.array([1.0]), f1, f0, sps, fs)
    for f, sign in ((f1, 1.0), (f0, -1.0)):
        x = np.exp(2j * np.pi * f * np.arange(sps) / fs) * cmath.exp(0.7j) * 3.0
        d, u = fsk.demod_range(x, g1, g0, 0, sps)
        assert d[-1] == pytest.approx(sign, abs=1e-12)
        assert u[-1] == pytest.approx(sign * 3.0 * sps, abs=1e-9)


def test_composition_equals_filters_in_sequence():
    """Section 4.1 composes H_BP with H_b: filtering with the composed taps
    equals the band-pass filter followed by the matched filter (explicit loops)."""
    rng = np.random.default_rng(3)
    h = rng.standard_normal(7)
    sps, fs, f = 4, 4e6, 5e5
    x = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    m = [cmath.exp(-2j * math.pi * f * (sps - 1 - t) / fs) for t in range(sps)]
    y = [sum(h[t] * x[i - t] for t in range(len(h)) if i - t >= 0) for i in range(40)]
    z = [sum(m[t] * y[i - t] for t in range(sps) if i - t >= 0) for i in range(40)]
    g1, _ = fsk.filters(h, f, -f, sps, fs)
    np.testing.assert_allclose(fsk.filter_range(x, g1, 0, 40), z, atol=1e-12)
    np.testing.assert_allclose(fsk.filter_range(x, g1, 13, 29), z[13:29], atol=1e-12)


def test_demod_normalisation():
    d, u = fsk.demod_values(np.array([3.0, 1j, 0.0, -2.0]), np.array([1.0, 1.0, 0.0, 0.0]))
    np.testing.assert_allclose(d, [0.5, 0.0, 0.0, 1.0])
    np.testing.assert_allclose(u, [2.0, 0.0, 0.0, 2.0])


def test_amplitude_invariance():
    """d is a ratio of magnitudes: a complex gain leaves it unchanged and
    scales u by its modulus."""
    w = synth.fsk_small(seed=4)
    x = fsk.iq_to_complex(w.iq16)
    g1, g0 = fsk.filters(w.h_bp, w.f1_hz, w.f0_hz, w.sps, w.fs_hz)
    d, u = fsk.demod_range(x, g1, g0, 1000, 3000)
    d2, u2 = fsk.demod_range(x * (7.0 * cmath.exp(1.1j)), g1, g0, 1000, 3000)
    np.testing.assert_allclose(d2, d, atol=1e-12)
    np.testing.assert_allclose(u2, 7.0 * u, rtol=1e-12)


# --- step 6: replica -----------------------------------------------------------

def test_replica_phase_continuity():
    chips = synth.random_chips(50, 9)
    sps, fs, f1, f0 = 4, 4e6, 5e5, -5e5
    r = fsk.replica(chips, sps, f1, f0, fs)
    assert r.shape == (200,) and r[0] == 1.0
    np.testing.assert_allclose(np.abs(r), 1.0, atol=1e-13)
    f = np.where(np.repeat(chips > 0, sps), f1, f0)[:-1]
    np.testing.assert_allclose(r[1:] / r[:-1], np.exp(2j * np.pi * f / fs), atol=1e-12)


def test_replica_support_length():
    g1, g0 = fsk.filters(np.ones(5) / 5, 5e5, -5e5, 2, 2e6)
    dc, uc = fsk.code_demod(np.array([1, -1, 1], np.int8), 2, 5e5, -5e5, 2e6, g1, g0)
    assert dc.shape == (6 + 6 - 1,) and uc.shape == dc.shape
    assert np.any(np.abs(dc[6:]) > 0)   # the filter tail past the packet carries signal


# --- step 7 ----------------------------------------------------------------------

def test_correlation_direct_equals_fft():
    rng = np.random.default_rng(5)
    dw = rng.uniform(-1, 1, 256)
    dc = rng.uniform(-1, 1, 100)
    np.testing.assert_allclose(fsk.corr_fft(dw, dc), fsk.corr_direct(dw, dc), atol=1e-10)


def test_correlation_of_shifted_code_peaks_at_the_shift():
    rng = np.random.default_rng(6)
    dc = rng.uniform(-1, 1, 60)
    dw = np.zeros(128)
    dw[37:97] = dc
    c = fsk.corr_fft(dw, dc)
    assert int(np.argmax(np.abs(c))) == 37
    assert c[37] == pytest.approx(float(np.dot(dc, dc)), rel=1e-12)


def test_floor_by_parseval():
    """mean over all N lags of corr^2 = sum_k |D_w[k] C[k]|^2 / N^2 (Parseval)."""
    rng = np.random.default_rng(7)
    dw = rng.uniform(-1, 1, 512)
    dc = rng.uniform(-1, 1, 200)
    _, _, fl = fsk.cell_stats(fsk.corr_direct(dw, dc), 300)
    pad = np.zeros(512)
    pad[:200] = dc
    want = np.sum(np.abs(np.fft.fft(dw) * np.fft.fft(pad)) ** 2) / 512 ** 2
    assert fl == pytest.approx(want, rel=1e-10)


def test_ties_take_the_smallest_lag():
    c = np.array([0.0, -3.0, 1.0, 3.0, 0.5])
    p, j, _ = fsk.cell_stats(c, 5)
    assert (p, j) == (9.0, 1)


# --- step 8 and the whole search ----------------------------------------------

def _noise_free(f_lo, delay, amp=900.0, phase=0.4, S=20000):
    chips = synth.random_chips(400, 21)
    sps, fs, f1, f0 = 4, 4e6, 5e5, -5e5
    h = synth.bandpass_taps(40, 7.5e5, fs)
    s = synth.fsk_transmission(chips, sps, f1, f0, fs)
    x = np.zeros(S, np.complex128)
    t = delay + np.arange(s.shape[0])
    x[t] = amp * s * np.exp(1j * (2 * np.pi * f_lo * t / fs + phase))
    return x, chips, sps, fs, f1, f0, h


@pytest.mark.parametrize("f_lo,delay", [(0.0, 5000), (3e5, 7777), (-1.1e6, 12001)])
def test_noise_free_tag_closed_forms(f_lo, delay):
    """A lone noise-free tag: d on its support equals d_c exactly (d is
    invariant to the complex gain), so the peak is at the true delay, w_c = q =
    sum d_c^2 and p_c = A sum d_c u_c (u_c of the unit replica)."""
    amp = 900.0
    x, chips, sps, fs, f1, f0, h = _noise_free(f_lo, delay, amp)
    dets, _ = fsk.search_samples(x, [chips], sps, fs, f1, f0, f_lo, h, threshold=10.0)
    g1, g0 = fsk.filters(h, f1, f0, sps, fs)
    dc, uc = fsk.code_demod(chips, sps, f1, f0, fs, g1, g0)
    e = float(np.dot(dc, dc))
    hit = [d for d in dets if d.window * (acq.default_fft_len(len(chips) * sps) - len(dc)) + d.lag == delay]
    assert len(hit) == 1
    d = hit[0]
    assert d.w_c == pytest.approx(e, rel=1e-9)
    assert d.q == pytest.approx(e, rel=1e-9)
    assert d.p_c == pytest.approx(amp * float(np.dot(dc, uc)), rel=1e-9)
    assert abs(d.toa - delay) <= 0.5


def test_stream_end_offset_golden():
    """The interpolation offset is 0 when a neighbour of the peak lies past the
    last searched lag S - n_c (tests/golden/refine_stream_end.txt: correlation
    values -1.5, 3, -2 at lags 4, 5, 6 of an 8-sample stream, n_c = 3)."""
    g = _fixture("refine_stream_end.txt")
    cm, c0, cp = g["upper_corr"]
    assert fsk.interp_offset(cm, c0, cp, 5, 8, 3) == 0.0
    assert fsk.interp_offset(cm, c0, cp, 0, 8, 3) == 0.0
    assert fsk.interp_offset(cm, c0, cp, 4, 8, 3) == pytest.approx(g["interior_delta"][0], rel=1e-15)


def test_peak_at_the_last_lag_is_not_interpolated():
    """A tag whose peak is the stream's last searched lag a = S - n_c (the last
    window's last valid lag, Section 2.1): toa = a exactly.  The seeded noise
    makes the two neighbours unequal, so ignoring the stream end would move it."""
    S = 20000
    x, chips, sps, fs, f1, f0, h = _noise_free(0.0, 0, S=S)
    g1, g0 = fsk.filters(h, f1, f0, sps, fs)
    n_c = len(chips) * sps + g1.shape[0] - 1
    a = S - n_c
    x, *_ = _noise_free(0.0, a, S=S)
    rng = np.random.default_rng(31)
    x = x + 20.0 * (rng.standard_normal(S) + 1j * rng.standard_normal(S))
    dets, _ = fsk.search_samples(x, [chips], sps, fs, f1, f0, 0.0, h, threshold=10.0)
    N, W, hop, _ = fsk.plan(S, len(chips), sps, g1.shape[0])
    hit = [d for d in dets if d.window * hop + d.lag == a]
    assert len(hit) == 1 and hit[0].window == W - 1
    assert hit[0].toa == float(a)
    cm, c0, cp, _, _ = fsk.lag_sums(fsk.lo_mix(x, 0.0, fs), g1, g0,
                                    fsk.code_demod(chips, sps, f1, f0, fs, g1, g0)[0], a)
    assert abs(acq.parabolic_offset(cm * cm, c0 * c0, cp * cp)) > 1e-6


def test_noisy_sums_obey_cauchy_schwarz():
    w = synth.fsk_small(seed=8)
    dets, _ = fsk.search(w.iq16, w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp)
    assert dets
    g1, g0 = fsk.filters(w.h_bp, w.f1_hz, w.f0_hz, w.sps, w.fs_hz)
    for d in dets:
        dc, _ = fsk.code_demod(w.chips[d.code], w.sps, w.f1_hz, w.f0_hz, w.fs_hz, g1, g0)
        e = float(np.dot(dc, dc))
        assert d.w_c ** 2 <= d.q * e * (1 + 1e-12)
        assert d.q != pytest.approx(e, rel=1e-6)


def test_tags_recovered_at_their_delays():
    w = synth.fsk_small(seed=11)
    dets, _ = fsk.search(w.iq16, w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp)
    g1, _ = fsk.filters(w.h_bp, w.f1_hz, w.f0_hz, w.sps, w.fs_hz)
    found = {}
    for d in dets:
        N, W, hop, n_c = fsk.plan(w.n_samples, len(w.chips[d.code]), w.sps, g1.shape[0])
        found[(d.code, d.window * hop + d.lag)] = d
    for t in w.tags:
        assert (t.code, int(t.delay)) in found
        assert abs(found[(t.code, int(t.delay))].toa - t.delay) < 0.5


def _brute_force(x, chips, sps, fs, f1, f0, f_lo, h, N, threshold):
    """Every step by explicit loops over samples, taps and lags."""
    S = len(x)
    xm = [x[i] * cmath.exp(-2j * math.pi * f_lo * i / fs) for i in range(S)]
    taps = []
    for f in (f1, f0):
        m = [cmath.exp(-2j * math.pi * f * (sps - 1 - t) / fs) for t in range(sps)]
        taps.append([sum(h[s] * m[t - s] for s in range(len(h)) if 0 <= t - s < sps)
                     for t in range(len(h) + sps - 1)])
    T = len(taps[0])

    def demod(sig, i):
        if i < 0 or i >= len(sig):
            return 0.0, 0.0
        a = [abs(sum(g[t] * sig[i - t] for t in range(T) if i - t >= 0)) for g in taps]
        return ((a[0] - a[1]) / (a[0] + a[1]) if a[0] + a[1] > 0 else 0.0), a[0] - a[1]

    L = len(chips) * sps
    ph, r = 0.0, []
    for n in range(L):
        r.append(cmath.exp(1j * ph))
        ph += 2 * math.pi * (f1 if chips[n // sps] > 0 else f0) / fs
    n_c = L + T - 1
    r += [0.0] * (T - 1)              # the replica is zero padded, its filter tail kept
    dc = [demod(r, n)[0] for n in range(n_c)]
    d = [demod(xm, i) for i in range(S)]
    dd = lambda i: d[i][0] if 0 <= i < S else 0.0
    hop = N - n_c
    W = max(1, -(-(S - N) // hop) + 1)
    out = []
    for w in range(W):
        corr = [sum(dc[n] * dd(w * hop + (t + n) % N) for n in range(n_c)) for t in range(N)]
        nv = hop if w < W - 1 else min(hop, S - n_c - w * hop) + 1
        P = [c * c for c in corr]
        j = max(range(nv), key=lambda t: (P[t], -t))
        fl = sum(P) / N
        if P[j] / fl >= threshold:
            a = w * hop + j
            cs = [sum(dc[n] * dd(a + k + n) for n in range(n_c)) for k in (-1, 0, 1)]
            q = sum(dd(a + n) ** 2 for n in range(n_c))
            p = sum(dc[n] * (d[a + n][1] if a + n < S else 0.0) for n in range(n_c))
            delta = 0.0
            if a - 1 >= 0 and a + 1 <= S - n_c:
                den = cs[0] ** 2 - 2 * cs[1] ** 2 + cs[2] ** 2
                if den < 0:
                    delta = min(0.5, max(-0.5, 0.5 * (cs[0] ** 2 - cs[2] ** 2) / den))
            out.append((w, j, P[j] / fl, a + delta, cs[1], q, p))
    return out


def test_brute_force_tiny_search():
    rng = np.random.default_rng(12)
    chips = synth.random_chips(20, 4)
    sps, fs, f1, f0, f_lo = 2, 2e6, 5e5, -5e5, 1e5
    h = synth.bandpass_taps(5, 7e5, fs)
    S, N = 300, 128
    x = rng.standard_normal(S) * 150 + 1j * rng.standard_normal(S) * 150
    s = synth.fsk_transmission(chips, sps, f1, f0, fs)
    t = 100 + np.arange(40)
    x[t] += 900 * s * np.exp(2j * np.pi * f_lo * t / fs)
    iq = synth.quantise_iq(x)
    want = _brute_force(list(fsk.iq_to_complex(iq)), chips, sps, fs, f1, f0, f_lo, h, N, 3.0)
    for method in ("fft", "direct"):
        got, _ = fsk.search(iq, [chips], sps, fs, f1, f0, f_lo, h, fft_len=N, threshold=3.0, method=method)
        assert len(got) == len(want) >= 2
        for g, b in zip(got, want):
            assert (g.window, g.lag) == b[:2]
            np.testing.assert_allclose([g.score, g.toa, g.w_c, g.q, g.p_c], b[2:], rtol=1e-9, atol=1e-9)


def test_default_threshold_quiet_on_noise():
    """No detection on a noise-only stream at the default threshold."""
    w = synth.fsk_small(seed=13, n_tags=0)
    dets, _ = fsk.search(w.iq16, w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp)
    assert dets == []


# --- planted mistakes: each one must trip a pin above --------------------------

def _mutants():
    def typo_denominator(f1, f0):
        a1, a0 = np.abs(f1), np.abs(f0)
        s = a0 + a0
        return np.where(s > 0, (a1 - a0) / np.where(s > 0, s, 1.0), 0.0), a1 - a0

    def unreversed_chip_filter(f, sps, fs):
        return np.exp(-2j * np.pi * (f / fs) * np.arange(sps, dtype=np.float64))

    def lo_plus(x, f_lo, fs, start=0):
        i = start + np.arange(x.shape[0], dtype=np.float64)
        return x * np.exp(2j * np.pi * (f_lo / fs) * i)

    def phase_reset_per_chip(chips, sps, f1, f0, fs):
        f = np.where(np.repeat(np.asarray(chips) > 0, sps), f1, f0)
        n = np.tile(np.arange(sps), len(chips))
        return np.exp(2j * np.pi * f * n / fs)

    def convolution_not_correlation(dw, dc):
        pad = np.zeros(dw.shape[0])
        pad[:dc.shape[0]] = dc
        return np.fft.ifft(np.fft.fft(dw) * np.fft.fft(pad)).real

    def floor_valid_only(corr, nv):
        P = corr * corr
        j = int(np.argmax(P[:nv]))
        return float(P[j]), j, float(P[:nv].mean())

    def no_upper_stream_end(cm, c0, cp, a, S, n_c):
        if a - 1 < 0:
            return 0.0
        return acq.parabolic_offset(cm * cm, c0 * c0, cp * cp)

    def q_of_the_code(x, g1, g0, dc, a):
        cm, c0, cp, q, p = fsk_lag_sums(x, g1, g0, dc, a)
        return cm, c0, cp, float(np.dot(dc, dc)), p

    return [("demod_values", typo_denominator), ("chip_filter", unreversed_chip_filter),
            ("lo_mix", lo_plus), ("replica", phase_reset_per_chip),
            ("corr_fft", convolution_not_correlation), ("cell_stats", floor_valid_only),
            ("lag_sums", q_of_the_code), ("interp_offset", no_upper_stream_end)]


fsk_lag_sums = fsk.lag_sums

PINS = [test_hand_worked_example,
        lambda: test_matched_filter_closed_form(4, 4e6),
        test_replica_phase_continuity,
        lambda: test_noise_free_tag_closed_forms(3e5, 7777),
        test_correlation_of_shifted_code_peaks_at_the_shift,
        test_floor_by_parseval,
        test_noisy_sums_obey_cauchy_schwarz,
        test_brute_force_tiny_search,
        test_stream_end_offset_golden,
        test_peak_at_the_last_lag_is_not_interpolated]


@pytest.mark.parametrize("name,fn", _mutants(), ids=[f"{n}:{f.__name__}" for n, f in _mutants()])
def test_planted_mistake_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(fsk, name, fn)
    failed = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1
