"""FP64 CPU oracle for the FSK acquisition front end.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The product path
(the CUDA library and its binding) never calls it and shares no code with it.

What it computes, in the order of Section 3 (steps 1-8, stated there for
frequency-shift keying) with the filter composition and cross-correlation
identity of Section 4.1:

1. int16 (I, Q) pairs become complex samples x[i] = I[i] + j Q[i];
2. the local-oscillator mix x[i] <- x[i] * exp(-j 2 pi f_lo i / fs), i the
   absolute sample index of the stream;
3.-4. the band-pass filter and the two one-chip matched filters, applied as
   the composed filters g_b = h_bp * m_b (Section 4.1 composes H_BP H_1 and
   H_BP H_0), f_b[i] = sum_{t<T} g_b[t] x[i-t] with x[i<0] = 0 (a causal
   linear convolution over the stream; the paper's circulant matrices are the
   block form of it).  m_b is the time-reversed conjugate of one chip of tone
   f_b: m_b[t] = exp(-j 2 pi f_b (sps-1-t) / fs), t < sps;
5. a_b = |f_b|, d = (a_1 - a_0) / (a_1 + a_0) (0 where a_1 + a_0 = 0) and
   u = a_1 - a_0.  The paper prints |f0| + |f0| as the denominator; the sum of
   the two magnitudes is read instead (the normalisation the text describes);
6. the replica of code c: a continuous-phase FSK packet with the same
   parameters, r[n] = exp(j phi[n]) with phi[0] = 0 and phi[n+1] = phi[n] +
   2 pi f_{b(n)} / fs (chip +1 -> tone f_1, chip -1 -> tone f_0), n < L =
   chips * sps, zero elsewhere.  Steps 3-5 without the LO mix give d_c, which
   is nonzero on its first n_c = L + T - 1 samples;
7. per overlapping window (the rule of the coherent search with the code
   length L replaced by n_c: hop = N - n_c, window w covers [w hop, w hop + N),
   the demodulated stream reads as zero at and past its end)
   corr[tau] = sum_{n < n_c} d_c[n] d[w hop + (tau + n) mod N], every circular
   lag; by Section 4.1 this is the real part of ifft(fft(d_w) conj(fft(d_c)));
8. j = argmax of |corr| over the window's valid lags (smallest lag on ties),
   P = corr^2, floor = mean of P over all N lags, score = P[j] / floor, a
   detection when score >= threshold.  At the absolute lag a = w hop + j the
   sums of step 8 are taken directly in FP64 over n < n_c (the paper's upper
   limit i = n is read as the n_c terms of the support):
   w_c = sum d_c[n] d[a+n], q = sum d[a+n]^2, p_c = sum d_c[n] u[a+n];
   the arrival time is a plus the vertex of the parabola through corr^2 at
   a-1, a, a+1 (0 at the stream ends, as in the coherent search).

Every function is plain numpy in float64/complex128; ``np.convolve`` and
``np.fft`` serve as library steps.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from oracle import acq

DEFAULT_THRESHOLD = 49.0


# ---------------------------------------------------------------------------
# steps 1-2: conversion and local-oscillator mix
# ---------------------------------------------------------------------------

def iq_to_complex(iq16: np.ndarray) -> np.ndarray:
    """Interleaved int16 (I, Q) pairs -> complex128 (Section 3 step 1)."""
    a = np.asarray(iq16, dtype=np.int16).reshape(-1).astype(np.float64)
    return a[0::2] + 1j * a[1::2]


def lo_mix(x: np.ndarray, f_lo_hz: float, fs_hz: float, start: int = 0) -> np.ndarray:
    """x[i] * exp(-j 2 pi f_lo (start + i) / fs) (Section 3 step 2)."""
    i = start + np.arange(x.shape[0], dtype=np.float64)
    return x * np.exp(-2j * np.pi * (f_lo_hz / fs_hz) * i)


# ---------------------------------------------------------------------------
# steps 3-5: filters and demodulation
# ---------------------------------------------------------------------------

def chip_filter(f_hz: float, sps: int, fs_hz: float) -> np.ndarray:
    """Matched filter of one chip of tone f: m[t] = exp(-j 2 pi f (sps-1-t)/fs)."""
    t = np.arange(sps, dtype=np.float64)
    return np.exp(-2j * np.pi * (f_hz / fs_hz) * (sps - 1 - t))


def compose(h_bp: np.ndarray, m: np.ndarray) -> np.ndarray:
    """The filter that applies h_bp and then m (Section 4.1): their full
    convolution, T = len(h_bp) + len(m) - 1 taps."""
    return np.convolve(np.asarray(h_bp, dtype=np.complex128), np.asarray(m, dtype=np.complex128))


def filters(h_bp: np.ndarray, f1_hz: float, f0_hz: float, sps: int, fs_hz: float):
    """(g_1, g_0): the composed filters H_BP H_1 and H_BP H_0."""
    return (compose(h_bp, chip_filter(f1_hz, sps, fs_hz)),
            compose(h_bp, chip_filter(f0_hz, sps, fs_hz)))


def filter_range(x: np.ndarray, g: np.ndarray, start: int, stop: int) -> np.ndarray:
    """y[i] = sum_{t<T} g[t] x[i-t] for i in [start, stop); x reads as zero
    outside [0, len(x))."""
    T = g.shape[0]
    lo = start - (T - 1)
    seg = np.zeros(stop - lo, dtype=np.complex128)
    a, b = max(lo, 0), min(stop, x.shape[0])
    if b > a:
        seg[a - lo:b - lo] = x[a:b]
    full = np.convolve(seg, g)          # full[k] = sum_t g[t] seg[k - t]
    return full[T - 1:stop - lo]


def demod_values(f1: np.ndarray, f0: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(d, u) of Section 3 step 5 from the two matched-filter outputs."""
    a1, a0 = np.abs(f1), np.abs(f0)
    s = a1 + a0
    d = np.where(s > 0, (a1 - a0) / np.where(s > 0, s, 1.0), 0.0)
    return d, a1 - a0


def demod_range(x: np.ndarray, g1: np.ndarray, g0: np.ndarray, start: int,
                stop: int) -> Tuple[np.ndarray, np.ndarray]:
    """d[i], u[i] of the (mixed) stream x for i in [start, stop); zero for
    i < 0 and i >= len(x): the demodulated stream has the stream's length."""
    n = stop - start
    d = np.zeros(n)
    u = np.zeros(n)
    a, b = max(start, 0), min(stop, x.shape[0])
    if b > a:
        dd, uu = demod_values(filter_range(x, g1, a, b), filter_range(x, g0, a, b))
        d[a - start:b - start] = dd
        u[a - start:b - start] = uu
    return d, u


# ---------------------------------------------------------------------------
# step 6: the replica
# ---------------------------------------------------------------------------

def replica(chips: np.ndarray, sps: int, f1_hz: float, f0_hz: float, fs_hz: float) -> np.ndarray:
    """Continuous-phase FSK packet of L = chips * sps samples.  The phase at
    sample n is 2 pi (n_1(n) f_1 + n_0(n) f_0) / fs, n_b(n) the number of
    earlier samples sent on tone b."""
    ones = np.repeat(np.asarray(chips) > 0, sps).astype(np.int64)
    L = ones.shape[0]
    n1 = np.concatenate(([0], np.cumsum(ones)[:-1]))
    n0 = np.arange(L, dtype=np.int64) - n1
    phi = 2.0 * np.pi * (n1.astype(np.float64) * (f1_hz / fs_hz) + n0.astype(np.float64) * (f0_hz / fs_hz))
    return np.exp(1j * phi)


def code_demod(chips: np.ndarray, sps: int, f1_hz: float, f0_hz: float, fs_hz: float,
               g1: np.ndarray, g0: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(d_c, u_c) over the support n < n_c = L + T - 1 (steps 3-5 on the
    zero-padded replica, no LO mix)."""
    r = replica(chips, sps, f1_hz, f0_hz, fs_hz)
    n_c = r.shape[0] + g1.shape[0] - 1
    return demod_values(filter_range(r, g1, 0, n_c), filter_range(r, g0, 0, n_c))


# ---------------------------------------------------------------------------
# step 7: correlation
# ---------------------------------------------------------------------------

def corr_direct(dw: np.ndarray, dc: np.ndarray, chunk: int = 256) -> np.ndarray:
    """The definition: corr[tau] = sum_{n<n_c} dc[n] dw[(tau+n) mod N], every tau."""
    N = dw.shape[0]
    n = np.arange(dc.shape[0])
    out = np.empty(N)
    for t0 in range(0, N, chunk):
        tau = np.arange(t0, min(t0 + chunk, N))
        out[tau] = dw[(tau[:, None] + n[None, :]) % N] @ dc
    return out


def corr_fft(dw: np.ndarray, dc: np.ndarray) -> np.ndarray:
    """Section 4.1: the real part of ifft(fft(d_w) * conj(fft(d_c padded)))."""
    N = dw.shape[0]
    pad = np.zeros(N)
    pad[:dc.shape[0]] = dc
    return np.fft.ifft(np.fft.fft(dw) * np.conj(np.fft.fft(pad))).real


def cell_stats(corr: np.ndarray, n_valid: int) -> Tuple[float, int, float]:
    """(P*, j, floor): P = corr^2, its max over lags [0, n_valid) (smallest lag
    on ties), and its mean over all N lags."""
    P = corr * corr
    j = int(np.argmax(P[:n_valid]))
    return float(P[j]), j, float(P.mean())


# ---------------------------------------------------------------------------
# step 8: sums at the peak and interpolation
# ---------------------------------------------------------------------------

def lag_sums(x: np.ndarray, g1: np.ndarray, g0: np.ndarray, dc: np.ndarray,
             a: int) -> Tuple[float, float, float, float, float]:
    """(corr[a-1], w_c = corr[a], corr[a+1], q, p_c) at absolute lag a,
    non-circular, directly in FP64."""
    n_c = dc.shape[0]
    d, u = demod_range(x, g1, g0, a - 1, a + n_c + 1)
    cm = float(np.dot(dc, d[0:n_c]))
    c0 = float(np.dot(dc, d[1:n_c + 1]))
    cp = float(np.dot(dc, d[2:n_c + 2]))
    q = float(np.dot(d[1:n_c + 1], d[1:n_c + 1]))
    p = float(np.dot(dc, u[1:n_c + 1]))
    return cm, c0, cp, q, p


def interp_offset(cm: float, c0: float, cp: float, a: int, S: int, n_c: int) -> float:
    """Sub-sample offset of the peak at absolute lag a (step 8, "interpolated"):
    the parabola vertex through the squared correlations at a-1, a, a+1, and 0
    at the stream ends, where a neighbour lag is not a searched lag
    (a-1 < 0 or a+1 > S - n_c)."""
    if a - 1 < 0 or a + 1 > S - n_c:
        return 0.0
    return acq.parabolic_offset(cm * cm, c0 * c0, cp * cp)


@dataclasses.dataclass
class FskDetection:
    code: int
    window: int
    lag: int        # window-relative
    score: float    # P* / floor
    toa: float      # samples from stream start
    w_c: float
    q: float
    p_c: float

    def key(self) -> Tuple[int, int, int]:
        return (self.code, self.window, self.lag)


@dataclasses.dataclass
class FskCell:
    p_max: float
    lag: int
    floor: float


def plan(S: int, n_chips: int, sps: int, T: int, fft_len: int = 0) -> Tuple[int, int, int, int]:
    """(N, W, hop, n_c) of a code: N = fft_len or 2 nextpow2(L), n_c = L + T - 1."""
    L = n_chips * sps
    n_c = L + T - 1
    N = fft_len if fft_len else acq.default_fft_len(L)
    W, hop = acq.window_plan(S, N, n_c)
    return N, W, hop, n_c


def search(iq16: np.ndarray, chips_list: Sequence[np.ndarray], sps: int, fs_hz: float,
           f1_hz: float, f0_hz: float, f_lo_hz: float, h_bp: np.ndarray, fft_len: int = 0,
           threshold: float = DEFAULT_THRESHOLD, method: str = "fft",
           pairs: Optional[Sequence[Tuple[int, int]]] = None, keep_cells: bool = False):
    """Every (window, code), or only ``pairs``, of an int16 (I, Q) stream.
    Returns (detections ordered by (window, code), {(w, c): FskCell} when
    keep_cells)."""
    return search_samples(iq_to_complex(iq16), chips_list, sps, fs_hz, f1_hz, f0_hz, f_lo_hz, h_bp,
                          fft_len, threshold, method, pairs, keep_cells)


def search_samples(x: np.ndarray, chips_list: Sequence[np.ndarray], sps: int, fs_hz: float,
                   f1_hz: float, f0_hz: float, f_lo_hz: float, h_bp: np.ndarray, fft_len: int = 0,
                   threshold: float = DEFAULT_THRESHOLD, method: str = "fft",
                   pairs: Optional[Sequence[Tuple[int, int]]] = None, keep_cells: bool = False):
    """The search from step 2 on, for complex samples x."""
    x = lo_mix(np.asarray(x, dtype=np.complex128), f_lo_hz, fs_hz)
    S = x.shape[0]
    g1, g0 = filters(h_bp, f1_hz, f0_hz, sps, fs_hz)
    T = g1.shape[0]
    plans = [plan(S, len(ch), sps, T, fft_len) for ch in chips_list]
    dcs = [code_demod(ch, sps, f1_hz, f0_hz, fs_hz, g1, g0)[0] for ch in chips_list]
    if pairs is None:
        maxW = max(p[1] for p in plans)
        pairs = [(w, c) for w in range(maxW) for c in range(len(chips_list)) if w < plans[c][1]]
    dets: List[FskDetection] = []
    cells: Dict[Tuple[int, int], FskCell] = {}
    for (w, c) in sorted(pairs):
        N, W, hop, n_c = plans[c]
        dw, _ = demod_range(x, g1, g0, w * hop, w * hop + N)
        corr = corr_fft(dw, dcs[c]) if method == "fft" else corr_direct(dw, dcs[c])
        nv = acq.n_valid_lags(w, W, S, N, n_c)
        pmax, j, fl = cell_stats(corr, nv)
        if keep_cells:
            cells[(w, c)] = FskCell(pmax, j, fl)
        score = pmax / fl if fl > 0 else 0.0
        if score >= threshold:
            a = w * hop + j
            cm, c0, cp, q, p = lag_sums(x, g1, g0, dcs[c], a)
            delta = interp_offset(cm, c0, cp, a, S, n_c)
            dets.append(FskDetection(c, w, j, score, a + delta, c0, q, p))
    return dets, cells
