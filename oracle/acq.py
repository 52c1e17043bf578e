"""FP64 CPU oracle for the acquisition-mode time-of-arrival search.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The product path
(the CUDA library and its binding) never calls it and shares no code with it.

What it computes, in the paper's order (Section 3, steps 2 and 6-8, and the
cross-correlation identity of Section 4.1), for the coherent complex-baseband
search over codes and carrier-frequency offsets:

* overlapping windows (Section 2.1: search blocks overlap so that every
  transmission lies entirely inside one block).  For a code of L samples and
  an FFT/window length N, hop = N - L; window w covers samples
  [w*hop, w*hop + N), samples at or past the stream end read as zero;
* the replica (Section 3 step 6): r[n] = chip[floor(n/sps)] for n < L, zero
  padded to N;
* the local-oscillator mix (Section 3 step 2) generalised to one mix per
  frequency bin: y[m] = x_w[m] * exp(-j 2 pi f_k m / fs), m window-relative;
* cross-correlation (Section 3 step 7): corr[tau] = sum_{n<L} y[(tau+n) mod N] r[n]
  for every circular lag tau in [0, N); by Section 4.1 this equals
  ifft(fft(y) * conj(fft(r))) (the conjugate is required for a correlation);
* peak search (Section 3 step 8): P = |corr|^2, the argmax over the window's
  valid lags (smallest lag on ties), and the noise floor = mean of P over all N
  lags; score = P* / floor; per (window, code) the bin with the largest score
  (smallest bin on ties) is a detection when score >= threshold;
* interpolation around the peak (Section 3 step 8, method not stated): the
  correlation is recomputed directly in FP64 at the absolute lags a-1, a, a+1
  and the vertex of the parabola through the three powers gives the
  sub-sample offset.

Every function is plain numpy in float64/complex128.  ``corr_direct`` is the
definition written out; ``corr_fft`` uses numpy's FFT as a library step.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


# ---------------------------------------------------------------------------
# windowing (Section 2.1, overlapping search blocks)
# ---------------------------------------------------------------------------

def default_fft_len(code_len: int) -> int:
    """N = 2 * nextpow2(L): the window holds one full code plus a hop of at
    least one code length."""
    return 2 * (1 << (int(code_len) - 1).bit_length())


def window_plan(n_samples: int, N: int, L: int) -> Tuple[int, int]:
    """(W, hop) with hop = N - L and W = max(1, ceil((S - N) / hop) + 1)."""
    if L < 1 or N <= L:
        raise ValueError("need 1 <= L < N")
    if n_samples < L:
        raise ValueError("stream shorter than one code")
    hop = N - L
    W = max(1, -(-(n_samples - N) // hop) + 1)
    return W, hop


def n_valid_lags(w: int, W: int, n_samples: int, N: int, L: int) -> int:
    """Number of valid lags (0 .. n-1) in window w.

    Windows before the last own lags [0, hop); the last owns
    [0, min(hop, S - L - w*hop)] inclusive, so every absolute start lag
    0 .. S-L is searched by exactly one window."""
    hop = N - L
    if w < W - 1:
        return hop
    return min(hop, n_samples - L - w * hop) + 1


def window_samples(x: np.ndarray, w: int, hop: int, N: int) -> np.ndarray:
    out = np.zeros(N, dtype=np.complex128)
    a = w * hop
    b = min(a + N, x.shape[0])
    if b > a:
        out[: b - a] = x[a:b]
    return out


# ---------------------------------------------------------------------------
# replica and mix (Section 3 steps 2 and 6)
# ---------------------------------------------------------------------------

def replica(chips: np.ndarray, sps: int, N: int) -> np.ndarray:
    L = len(chips) * sps
    if L > N:
        raise ValueError("code longer than the window")
    r = np.zeros(N, dtype=np.float64)
    r[:L] = np.repeat(np.asarray(chips, dtype=np.float64), sps)
    return r


def mix(xw: np.ndarray, f_hz: float, fs_hz: float) -> np.ndarray:
    """y[m] = x_w[m] * exp(-j 2 pi f m / fs) for window-relative m."""
    m = np.arange(xw.shape[0], dtype=np.float64)
    return xw * np.exp(-2j * np.pi * (f_hz / fs_hz) * m)


# ---------------------------------------------------------------------------
# cross-correlation (Section 3 step 7; Section 4.1 identity)
# ---------------------------------------------------------------------------

def corr_direct(y: np.ndarray, r: np.ndarray, L: int, chunk: int = 256) -> np.ndarray:
    """The definition: corr[tau] = sum_{n<L} y[(tau+n) mod N] * r[n], every tau."""
    N = y.shape[0]
    n = np.arange(L)
    out = np.empty(N, dtype=np.complex128)
    rL = r[:L]
    for t0 in range(0, N, chunk):
        tau = np.arange(t0, min(t0 + chunk, N))
        idx = (tau[:, None] + n[None, :]) % N
        out[tau] = y[idx] @ rL
    return out


def corr_fft(y: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Section 4.1: xcorr = ifft(fft(y) * conj(fft(r))) (circular, length N)."""
    return np.fft.ifft(np.fft.fft(y) * np.conj(np.fft.fft(r)))


# ---------------------------------------------------------------------------
# peak, floor, score (Section 3 step 8)
# ---------------------------------------------------------------------------

def cell_stats(corr: np.ndarray, n_valid: int) -> Tuple[float, int, float]:
    """(P*, tau*, floor): max of |corr|^2 over lags [0, n_valid) with the
    smallest lag on ties, and the mean of |corr|^2 over all N lags."""
    P = corr.real ** 2 + corr.imag ** 2
    tau = int(np.argmax(P[:n_valid]))
    return float(P[tau]), tau, float(P.mean())


# ---------------------------------------------------------------------------
# interpolation (Section 3 step 8, "interpolated"; 3-point parabola on P)
# ---------------------------------------------------------------------------

def direct_power(x: np.ndarray, chips: np.ndarray, sps: int, f_hz: float, fs_hz: float,
                 a: int) -> float:
    """|sum_{n<L} x[a+n] exp(-j 2 pi f (a+n)/fs) r[n]|^2 at absolute lag a,
    non-circular, samples past the stream end read as zero (FP64)."""
    L = len(chips) * sps
    S = x.shape[0]
    seg = np.zeros(L, dtype=np.complex128)
    hi = min(a + L, S)
    if hi > a:
        seg[: hi - a] = x[a:hi]
    t = a + np.arange(L, dtype=np.float64)
    y = seg * np.exp(-2j * np.pi * (f_hz / fs_hz) * t)
    r = np.repeat(np.asarray(chips, dtype=np.float64), sps)
    c = np.dot(y, r)
    return float(c.real ** 2 + c.imag ** 2)


def parabolic_offset(p_minus: float, p0: float, p_plus: float) -> float:
    """Vertex of the parabola through (-1, P-), (0, P0), (1, P+), clamped to
    [-1/2, 1/2]; 0 when the three points do not bend downward."""
    den = p_minus - 2.0 * p0 + p_plus
    if not den < 0.0:
        return 0.0
    d = 0.5 * (p_minus - p_plus) / den
    return min(0.5, max(-0.5, d))


def refine(x: np.ndarray, chips: np.ndarray, sps: int, f_hz: float, fs_hz: float,
           a: int) -> Tuple[float, float]:
    """(toa, P0): sub-sample arrival time a + delta (samples) and the direct
    peak power.  delta = 0 at the stream ends (a-1 < 0 or a+1 > S-L)."""
    L = len(chips) * sps
    S = x.shape[0]
    p0 = direct_power(x, chips, sps, f_hz, fs_hz, a)
    if a - 1 < 0 or a + 1 > S - L:
        return float(a), p0
    pm = direct_power(x, chips, sps, f_hz, fs_hz, a - 1)
    pp = direct_power(x, chips, sps, f_hz, fs_hz, a + 1)
    return float(a) + parabolic_offset(pm, p0, pp), p0


# ---------------------------------------------------------------------------
# the whole search
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Detection:
    code: int
    window: int
    lag: int          # window-relative
    freq_bin: int
    score: float
    peak_power: float  # direct FP64 |corr|^2 at the absolute lag
    toa: float        # samples from stream start

    def key(self) -> Tuple[int, int, int, int]:
        return (self.code, self.window, self.lag, self.freq_bin)


@dataclasses.dataclass
class Cell:
    """Per (window, code, bin): peak power, its lag, and the floor."""
    p_max: float
    lag: int
    floor: float


def search_window_code(x: np.ndarray, chips: np.ndarray, sps: int, fs_hz: float,
                       freqs_hz: Sequence[float], N: int, w: int,
                       method: str = "fft") -> List[Cell]:
    """All K cells of one (window, code)."""
    L = len(chips) * sps
    W, hop = window_plan(x.shape[0], N, L)
    nv = n_valid_lags(w, W, x.shape[0], N, L)
    xw = window_samples(x, w, hop, N)
    r = replica(chips, sps, N)
    cells = []
    for f in freqs_hz:
        y = mix(xw, float(f), fs_hz)
        c = corr_fft(y, r) if method == "fft" else corr_direct(y, r, L)
        p, t, fl = cell_stats(c, nv)
        cells.append(Cell(p, t, fl))
    return cells


def select(cells: List[Cell]) -> Tuple[int, float]:
    """(k*, score): the bin with the largest P*/floor, smallest bin on ties."""
    best_k, best_s = 0, -1.0
    for k, c in enumerate(cells):
        s = c.p_max / c.floor if c.floor > 0 else 0.0
        if s > best_s:
            best_k, best_s = k, s
    return best_k, best_s


def search(x: np.ndarray, chips_list: Sequence[np.ndarray], sps: int, fs_hz: float,
           freqs_hz: Sequence[float], fft_len: int = 0, threshold: float = 25.0,
           method: str = "fft", pairs: Optional[Sequence[Tuple[int, int]]] = None,
           keep_cells: bool = False):
    """Run the search over every (window, code), or only over ``pairs``
    ((window, code) tuples).  Returns (detections ordered by (window, code),
    cells dict {(w, c): [Cell]*K} when keep_cells)."""
    x = np.asarray(x).astype(np.complex128)
    S = x.shape[0]
    dets: List[Detection] = []
    cells_out: Dict[Tuple[int, int], List[Cell]] = {}
    plans = []
    for c, ch in enumerate(chips_list):
        L = len(ch) * sps
        N = fft_len if fft_len else default_fft_len(L)
        W, hop = window_plan(S, N, L)
        plans.append((N, W, hop))
    if pairs is None:
        maxW = max(p[1] for p in plans)
        pairs = [(w, c) for w in range(maxW) for c in range(len(chips_list)) if w < plans[c][1]]
    for (w, c) in sorted(pairs):
        N, W, hop = plans[c]
        cells = search_window_code(x, chips_list[c], sps, fs_hz, freqs_hz, N, w, method)
        if keep_cells:
            cells_out[(w, c)] = cells
        k, s = select(cells)
        if s >= threshold:
            a = w * hop + cells[k].lag
            toa, p0 = refine(x, chips_list[c], sps, float(freqs_hz[k]), fs_hz, a)
            dets.append(Detection(c, w, cells[k].lag, k, s, p0, toa))
    return dets, cells_out
