"""Seeded synthetic inputs for the acquisition search.

This module only *makes* inputs: tag codes, complex baseband streams with
additive white Gaussian noise, and tag transmissions injected at a known
delay, carrier offset, phase and SNR.  It contains none of the search's
arithmetic (no correlation, no FFT, no peak search), so that both the CUDA
path and the FP64 oracle can be fed from it without sharing method code.

Signal model (Section 2: packets of pseudorandom bits at about 1 Mb/s,
received as complex samples at 8 MS/s; Section 3 step 6: the replica is a
noise-free copy of the transmission):

* a tag code is a sequence of +/-1 chips; a transmission of code ``c`` at
  integer delay ``d`` occupies samples ``d .. d + chips*sps - 1`` and holds
  chip ``i`` for ``sps`` consecutive samples;
* the transmission is rotated by a carrier offset ``f`` (Hz) and a phase,
  ``A * exp(j(2*pi*f*t/fs + phi)) * chip[(t-d)//sps]`` for absolute sample ``t``;
* noise is complex AWGN with standard deviation ``sigma`` per component
  (int16-range, sigma = 2048 by default) and the amplitude follows the
  per-complex-sample SNR, ``A = sqrt(2 sigma^2 10^(snr_db/10))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(state: int, n: int) -> np.ndarray:
    """``n`` outputs of Vigna's splitmix64 generator started at ``state``.

    Published definition: state += 0x9E3779B97F4A7C15; z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) *
    0x94D049BB133111EB; return z ^ (z >> 31)  (all mod 2^64).
    """
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(state & MASK64)
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = s + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        out[:] = z ^ (z >> np.uint64(31))
    return out


def random_chips(n_chips: int, seed: int) -> np.ndarray:
    """+/-1 chips (int8) from the low bit of splitmix64 outputs."""
    bits = splitmix64(seed, n_chips) & np.uint64(1)
    return (1 - 2 * bits.astype(np.int8)).astype(np.int8)


def lfsr_chips(seed: int = 1, degree: int = 10, taps: Sequence[int] = (10, 7)) -> np.ndarray:
    """One period (2^degree - 1 chips) of a Fibonacci LFSR as +/-1 int8.

    The default polynomial x^10 + x^7 + 1 is primitive, so the sequence is a
    maximal-length (m-)sequence of 1023 chips.  ``seed`` is the nonzero initial
    register state.
    """
    n = (1 << degree) - 1
    reg = seed & n
    if reg == 0:
        raise ValueError("LFSR seed must be nonzero")
    out = np.empty(n, dtype=np.int8)
    for i in range(n):
        bit = 0
        for t in taps:
            bit ^= (reg >> (degree - t)) & 1
        out[i] = 1 - 2 * (reg & 1)
        reg = (reg >> 1) | (bit << (degree - 1))
    return out


@dataclasses.dataclass
class Tag:
    code: int
    delay: float          # samples from stream start (integer for parity configs)
    freq_hz: float        # carrier offset actually injected
    bin: int              # nearest grid bin index (for bookkeeping)
    snr_db: float
    phase: float


@dataclasses.dataclass
class Workload:
    name: str
    x: np.ndarray                 # complex64 [S]
    chips: List[np.ndarray]       # list of int8 +/-1 arrays
    sps: int
    fs_hz: float
    freqs_hz: np.ndarray          # float64 [K]
    fft_len: int                  # N (0 = library default per code)
    tags: List[Tag]
    sigma: float

    @property
    def n_samples(self) -> int:
        return int(self.x.shape[0])

    @property
    def chips_concat(self) -> np.ndarray:
        return np.concatenate(self.chips).astype(np.int8)

    @property
    def chips_per_code(self) -> np.ndarray:
        return np.array([len(c) for c in self.chips], dtype=np.int32)

    def iq(self) -> np.ndarray:
        """Interleaved float32 (re, im) view, shape [S, 2]."""
        return self.x.view(np.float32).reshape(-1, 2)


def awgn(n: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    z = rng.standard_normal(2 * n, dtype=np.float64) * sigma
    return (z[0::2] + 1j * z[1::2]).astype(np.complex64)


def tag_amplitude(snr_db: float, sigma: float) -> float:
    return math.sqrt(2.0 * sigma * sigma * 10.0 ** (snr_db / 10.0))


def inject(x: np.ndarray, chips: np.ndarray, sps: int, fs_hz: float, tag: Tag, sigma: float,
           amplitude: Optional[float] = None) -> None:
    """Add one transmission of ``chips`` to ``x`` in place (float64 arithmetic).

    The receiver's sample ``t`` is modelled as the average of the chip
    waveform over the sample interval [t, t+1) (an integrate-and-dump front
    end), so a fractional delay produces a partial sample at each chip edge
    and carries sub-sample timing.  For an integer delay every interval lies
    inside one chip and sample ``t`` holds chip ``(t - delay) // sps`` exactly.
    The carrier is evaluated at the sample instant ``t``.
    """
    S = x.shape[0]
    L = len(chips) * sps
    A = tag_amplitude(tag.snr_db, sigma) if amplitude is None else amplitude
    t0 = int(math.floor(tag.delay))
    t = np.arange(max(t0, 0), min(t0 + L + 1, S), dtype=np.int64)
    if t.size == 0:
        return
    ch = np.asarray(chips, dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(ch)]) * sps   # integral at chip edges

    def integral(u):
        u = np.clip(u, 0.0, float(L))
        i = np.minimum(np.floor(u / sps).astype(np.int64), len(ch) - 1)
        return cum[i] + (u - i * sps) * ch[i]

    rel = t.astype(np.float64) - tag.delay
    val = integral(rel + 1.0) - integral(rel)
    ph = 2.0 * math.pi * tag.freq_hz * t.astype(np.float64) / fs_hz + tag.phase
    x[t] += (A * val * np.exp(1j * ph)).astype(np.complex64)


def freq_grid(lo_hz: float, hi_hz: float, step_hz: float) -> np.ndarray:
    k = int(round((hi_hz - lo_hz) / step_hz)) + 1
    return lo_hz + step_hz * np.arange(k, dtype=np.float64)


def tiny(seed: int = 1, snr_db: float = -10.0, sigma: float = 2048.0) -> Workload:
    """One 16384-sample window, one 1023-chip LFSR code at 2 samples/chip,
    5 bins of 500 Hz at 2 MS/s, one tag at -10 dB."""
    rng = np.random.default_rng(seed)
    fs, sps, N = 2e6, 2, 16384
    chips = lfsr_chips(seed=seed if seed > 0 else 1)
    L = len(chips) * sps
    freqs = freq_grid(-1000.0, 1000.0, 500.0)
    x = awgn(N, sigma, rng)
    hop = N - L
    delay = int(rng.integers(0, hop + 1))
    b = int(rng.integers(0, len(freqs)))
    f = float(freqs[b] + rng.uniform(-50.0, 50.0))
    tag = Tag(code=0, delay=float(delay), freq_hz=f, bin=b, snr_db=snr_db,
              phase=float(rng.uniform(0, 2 * math.pi)))
    inject(x, chips, sps, fs, tag, sigma)
    return Workload("tiny: 1 window x 16384, 1 code x 1023 chips, sps 2, 5 bins",
                    x, [chips], sps, fs, freqs, N, [tag], sigma)


def realistic(seed: int = 2, seconds: float = 1.0, n_codes: int = 16, n_chips: int = 8192,
              sps: int = 8, fs_hz: float = 8e6, n_tags: int = 40, snr_range=(-20.0, 0.0),
              freqs_hz: Optional[np.ndarray] = None, sigma: float = 2048.0,
              jitter_hz: float = 12.0, min_same_code_gap: Optional[int] = None,
              fft_len: int = 0) -> Workload:
    """1 s of 8 MS/s complex noise, 16 codes x 8192 chips at 8 samples/chip,
    31 bins of 1 kHz over +/-15 kHz, 40 tags with SNR U[-20, 0] dB."""
    rng = np.random.default_rng(seed)
    S = int(round(seconds * fs_hz))
    L = n_chips * sps
    N = fft_len if fft_len else 2 * (1 << (L - 1).bit_length())
    freqs = freq_grid(-15000.0, 15000.0, 1000.0) if freqs_hz is None else np.asarray(freqs_hz, np.float64)
    chips = [random_chips(n_chips, seed * 1_000_003 + c) for c in range(n_codes)]
    x = awgn(S, sigma, rng)
    gap = 2 * N if min_same_code_gap is None else min_same_code_gap
    tags: List[Tag] = []
    placed = {c: [] for c in range(n_codes)}
    tries = 0
    while len(tags) < n_tags and tries < 100000:
        tries += 1
        c = int(rng.integers(0, n_codes))
        d = int(rng.integers(0, S - L + 1))
        if any(abs(d - p) < gap for p in placed[c]):
            continue
        b = int(rng.integers(0, len(freqs)))
        f = float(freqs[b] + rng.uniform(-jitter_hz, jitter_hz))
        snr = float(rng.uniform(*snr_range))
        tg = Tag(code=c, delay=float(d), freq_hz=f, bin=b, snr_db=snr,
                 phase=float(rng.uniform(0, 2 * math.pi)))
        placed[c].append(d)
        tags.append(tg)
        inject(x, chips[c], sps, fs_hz, tg, sigma)
    return Workload(f"realistic: {S} samples at {fs_hz/1e6:g} MS/s, {n_codes} codes x {n_chips} chips, "
                    f"sps {sps}, {len(freqs)} bins, {len(tags)} tags", x, chips, sps, fs_hz, freqs, N,
                    tags, sigma)


def small(seed: int = 11, S: int = 40000, n_codes: int = 3, n_chips: int = 600, sps: int = 4,
          fs_hz: float = 4e6, N: int = 8192, freqs_hz: Optional[np.ndarray] = None, n_tags: int = 4,
          snr_range=(-12.0, -3.0), sigma: float = 2048.0) -> Workload:
    """A few ragged windows (S not a multiple of the hop), several codes, an odd
    bin count; small enough that the oracle finishes in well under a second."""
    freqs = freq_grid(-3000.0, 3000.0, 1500.0) if freqs_hz is None else np.asarray(freqs_hz, np.float64)
    return realistic(seed=seed, seconds=S / fs_hz, n_codes=n_codes, n_chips=n_chips, sps=sps,
                     fs_hz=fs_hz, n_tags=n_tags, snr_range=snr_range, freqs_hz=freqs,
                     sigma=sigma, jitter_hz=20.0, min_same_code_gap=2 * N, fft_len=N)


def batch(seed: int = 3, n_streams: int = 8, duration_s=(0.5, 2.0), fs_choices=(2e6, 4e6, 8e6),
          n_codes: int = 64, chip_choices=(2048, 4096, 8192, 16384), bins=(15, 63), bin_step_hz: float = 500.0,
          tags_per_group: int = 5, snr_range=(-20.0, 0.0), sigma: float = 2048.0,
          chip_rate_hz: float = 1e6) -> List[Workload]:
    """Several receiver streams for one batched search: each stream draws its
    sample rate from fs_choices (samples/chip = fs / chip rate) and its duration
    from duration_s, and has its own odd number of bins in [bins], spaced
    bin_step_hz and centred on 0.  All streams search the same codes, whose
    lengths are drawn from chip_choices.  About tags_per_group tags per stream
    and code-length group, with SNR uniform in snr_range, integer delays,
    on-grid carrier offsets plus a jitter of at most a tenth of a bin step."""
    rng = np.random.default_rng(seed)
    lengths = [int(rng.choice(chip_choices)) for _ in range(n_codes)]
    chips = [random_chips(n, seed * 7_919 + c) for c, n in enumerate(lengths)]
    out: List[Workload] = []
    for s in range(n_streams):
        fs = float(rng.choice(fs_choices))
        sps = int(round(fs / chip_rate_hz))
        S = int(round(rng.uniform(*duration_s) * fs))
        lo, hi = bins
        K = int(rng.integers(lo // 2, hi // 2 + 1)) * 2 + 1
        freqs = (np.arange(K, dtype=np.float64) - (K - 1) / 2) * bin_step_hz
        x = awgn(S, sigma, rng)
        tags: List[Tag] = []
        for n_chips in sorted(set(lengths)):
            group = [c for c in range(n_codes) if lengths[c] == n_chips]
            L = n_chips * sps
            if L >= S:
                continue
            gap = 4 * (1 << (L - 1).bit_length())
            placed: dict = {}
            for _ in range(tags_per_group):
                for _try in range(100):
                    c = int(rng.choice(group))
                    d = int(rng.integers(0, S - L + 1))
                    if all(abs(d - p) >= gap for p in placed.get(c, [])):
                        break
                else:
                    continue
                placed.setdefault(c, []).append(d)
                b = int(rng.integers(0, K))
                tg = Tag(code=c, delay=float(d), freq_hz=float(freqs[b] + rng.uniform(-0.1, 0.1) * bin_step_hz),
                         bin=b, snr_db=float(rng.uniform(*snr_range)), phase=float(rng.uniform(0, 2 * math.pi)))
                inject(x, chips[c], sps, fs, tg, sigma)
                tags.append(tg)
        out.append(Workload(f"batch stream {s}: {S} samples at {fs/1e6:g} MS/s, sps {sps}, {K} bins", x, chips,
                            sps, fs, freqs, 0, tags, sigma))
    return out


def proposal_stream(seed: int, n_windows: int, device, n_codes: int = 64, n_chips: int = 8192, sps: int = 8,
                    fs_hz: float = 8e6, n_bins: int = 63, bin_step_hz: float = 500.0, snr_range=(-25.0, 5.0),
                    p_empty: float = 0.2, sigma: float = 2048.0, chunk: int = 512, code_seed: Optional[int] = None):
    """A device-resident stream laid out as n_windows search windows of
    N = 2 * chips * sps samples (hop = chips * sps): each hop period holds one
    transmission with probability 1 - p_empty (code, bin, SNR, phase and an
    integer start inside the period all uniform; carrier = bin centre plus a
    jitter of at most a tenth of a step).  Noise from torch's seeded generator
    on `device`; tag parameters from a seeded numpy generator; the codes from
    code_seed (default: seed), so training and test streams can share a bank.  Returns
    (x [S, 2] float32 tensor, chips, freqs, truth) with truth[w] = (code, bin)
    or (-1, -1)."""
    import torch
    L = n_chips * sps
    N = 2 * L
    hop = N - L
    S = N + (n_windows - 1) * hop
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    x = torch.randn((S, 2), generator=gen, device=device, dtype=torch.float32) * sigma
    cs = seed if code_seed is None else code_seed
    chips = [random_chips(n_chips, cs * 1_000_003 + c) for c in range(n_codes)]
    chips_t = torch.from_numpy(np.stack(chips).astype(np.float32)).to(device)
    freqs = (np.arange(n_bins, dtype=np.float64) - (n_bins - 1) / 2) * bin_step_hz
    rng = np.random.default_rng(seed)
    truth = []
    tags = []
    for w in range(n_windows):
        if rng.uniform() < p_empty:
            truth.append((-1, -1))
            continue
        c = int(rng.integers(0, n_codes))
        b = int(rng.integers(0, n_bins))
        f = float(freqs[b] + rng.uniform(-0.1, 0.1) * bin_step_hz)
        snr = float(rng.uniform(*snr_range))
        d = w * hop + int(rng.integers(0, hop))
        tags.append((d, c, f, tag_amplitude(snr, sigma), float(rng.uniform(0, 2 * math.pi))))
        truth.append((c, b))
    t = torch.arange(L, device=device, dtype=torch.int64)
    xc = torch.view_as_complex(x)
    for i0 in range(0, len(tags), chunk):
        part = tags[i0:i0 + chunk]
        d = torch.tensor([p[0] for p in part], device=device, dtype=torch.int64)
        code = torch.tensor([p[1] for p in part], device=device, dtype=torch.int64)
        f = torch.tensor([p[2] for p in part], device=device, dtype=torch.float64)
        amp = torch.tensor([p[3] for p in part], device=device, dtype=torch.float64)
        ph0 = torch.tensor([p[4] for p in part], device=device, dtype=torch.float64)
        idx = d[:, None] + t[None, :]                                       # [n, L]
        wave = chips_t[code][:, t // sps].to(torch.float64)                 # [n, L]
        ph = 2 * math.pi * f[:, None] * idx.to(torch.float64) / fs_hz + ph0[:, None]
        sig = (amp[:, None] * wave * torch.exp(1j * ph)).to(torch.complex64)
        ok = idx < S
        xc.index_add_(0, idx[ok], sig[ok])
    return x, chips, freqs, truth


# ---------------------------------------------------------------------------
# FSK streams (Section 3: the frequency-shift-keyed transmissions of the tags,
# received as int16 (I, Q) pairs)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class FskWorkload:
    name: str
    iq16: np.ndarray              # int16 [S, 2] (I, Q) pairs
    chips: List[np.ndarray]       # +/-1 int8 per code
    sps: int
    fs_hz: float
    f1_hz: float                  # tone of chip +1, relative to the band centre
    f0_hz: float                  # tone of chip -1
    f_lo_hz: float                # band centre relative to the receiver's centre
    h_bp: np.ndarray              # band-pass taps (float64), an input of the search
    fft_len: int                  # N (0 = library default per code)
    tags: List[Tag]
    sigma: float

    @property
    def n_samples(self) -> int:
        return int(self.iq16.shape[0])

    @property
    def chips_concat(self) -> np.ndarray:
        return np.concatenate(self.chips).astype(np.int8)

    @property
    def chips_per_code(self) -> np.ndarray:
        return np.array([len(c) for c in self.chips], dtype=np.int32)


def bandpass_taps(n_taps: int = 200, cutoff_hz: float = 1.5e6, fs_hz: float = 8e6) -> np.ndarray:
    """A Hamming-windowed sinc low-pass of n_taps real taps: after the LO shift
    the transmissions' band is centred at zero, so the band-pass filter of the
    front end is a low-pass at baseband.  Unit gain at DC."""
    if n_taps == 1:
        return np.ones(1)
    n = np.arange(n_taps, dtype=np.float64)
    t = n - (n_taps - 1) / 2.0
    h = np.sinc(2.0 * cutoff_hz / fs_hz * t) * (0.54 - 0.46 * np.cos(2.0 * math.pi * n / (n_taps - 1)))
    return h / h.sum()


def fsk_transmission(chips: np.ndarray, sps: int, f1_hz: float, f0_hz: float, fs_hz: float) -> np.ndarray:
    """Unit-amplitude continuous-phase FSK packet: chip +1 on tone f1, chip -1
    on tone f0, sps samples per chip, phase 0 at the first sample and advanced
    by 2 pi f / fs after each sample."""
    f = np.where(np.repeat(np.asarray(chips) > 0, sps), f1_hz, f0_hz)
    step = 2.0 * math.pi * f / fs_hz
    return np.exp(1j * (np.cumsum(step) - step))


def inject_fsk(x: np.ndarray, w: "FskWorkload", tag: Tag, amplitude: Optional[float] = None) -> None:
    """Add one transmission at integer delay tag.delay to the complex128 stream
    x: A exp(j(2 pi (f_lo + f_tag) t / fs + phase)) s[t - delay]."""
    S = x.shape[0]
    s = fsk_transmission(w.chips[tag.code], w.sps, w.f1_hz, w.f0_hz, w.fs_hz)
    d = int(tag.delay)
    n = min(s.shape[0], S - d)
    if n <= 0:
        return
    t = d + np.arange(n, dtype=np.float64)
    A = tag_amplitude(tag.snr_db, w.sigma) if amplitude is None else amplitude
    x[d:d + n] += A * s[:n] * np.exp(1j * (2.0 * math.pi * (w.f_lo_hz + tag.freq_hz) * t / w.fs_hz + tag.phase))


def quantise_iq(x: np.ndarray) -> np.ndarray:
    """Round to the nearest integer and saturate to int16, as [S, 2] (I, Q)."""
    out = np.empty((x.shape[0], 2), dtype=np.int16)
    out[:, 0] = np.clip(np.rint(x.real), -32768, 32767)
    out[:, 1] = np.clip(np.rint(x.imag), -32768, 32767)
    return out


def fsk_stream(seed: int, S: int, chips: List[np.ndarray], sps: int, fs_hz: float, f1_hz: float, f0_hz: float,
               f_lo_hz: float, n_tags: int, snr_range, offset_hz: float = 5e3, sigma: float = 2048.0,
               n_taps: int = 200, cutoff_hz: Optional[float] = None, fft_len: int = 0,
               min_same_code_gap: Optional[int] = None, name: str = "fsk") -> FskWorkload:
    """Complex AWGN (sigma per component) plus n_tags FSK transmissions (code,
    integer delay, carrier offset within +/-offset_hz of the band centre,
    phase and SNR drawn from a seeded generator; transmissions of one code at
    least min_same_code_gap samples apart, by default twice the window),
    quantised to int16."""
    rng = np.random.default_rng(seed)
    cut = cutoff_hz if cutoff_hz is not None else 1.5 * max(abs(f1_hz), abs(f0_hz))
    w = FskWorkload(name, np.zeros((0, 2), np.int16), chips, sps, fs_hz, f1_hz, f0_hz, f_lo_hz,
                    bandpass_taps(n_taps, cut, fs_hz), fft_len, [], sigma)
    z = rng.standard_normal(2 * S) * sigma
    x = z[0::2] + 1j * z[1::2]
    L = max(len(c) for c in chips) * sps
    N = fft_len if fft_len else 2 * (1 << (L - 1).bit_length())
    gap = 2 * N if min_same_code_gap is None else min_same_code_gap
    placed: dict = {}
    tries = 0
    while len(w.tags) < n_tags and tries < 100000:
        tries += 1
        c = int(rng.integers(0, len(chips)))
        Lc = len(chips[c]) * sps
        if Lc > S:
            continue
        d = int(rng.integers(0, S - Lc + 1))
        if any(abs(d - p) < gap for p in placed.get(c, [])):
            continue
        placed.setdefault(c, []).append(d)
        tg = Tag(code=c, delay=float(d), freq_hz=float(rng.uniform(-offset_hz, offset_hz)), bin=-1,
                 snr_db=float(rng.uniform(*snr_range)), phase=float(rng.uniform(0, 2 * math.pi)))
        inject_fsk(x, w, tg)
        w.tags.append(tg)
    w.iq16 = quantise_iq(x)
    return w


def fsk_tiny(seed: int = 1) -> FskWorkload:
    """16384 samples at 2 MS/s, one 1023-chip LFSR code at 2 samples/chip on
    tones +/-500 kHz, a 200-tap band-pass filter, one tag at -5 dB."""
    return fsk_stream(seed, 16384, [lfsr_chips(seed=seed if seed > 0 else 1)], 2, 2e6, 5e5, -5e5, 0.0, 1,
                      (-5.0, -5.0), cutoff_hz=0.75e6, name="fsk tiny: 16384 samples, 1 code x 1023 chips, sps 2")


def fsk_small(seed: int = 11, S: int = 40000, n_codes: int = 3, n_chips: int = 600, sps: int = 4,
              fs_hz: float = 4e6, f_lo_hz: float = 250e3, n_tags: int = 4, fft_len: int = 0,
              snr_range=(-8.0, 0.0)) -> FskWorkload:
    """A few ragged windows, several codes, an LO offset."""
    chips = [random_chips(n_chips, seed * 1_000_003 + c) for c in range(n_codes)]
    return fsk_stream(seed, S, chips, sps, fs_hz, 5e5, -5e5, f_lo_hz, n_tags, snr_range, fft_len=fft_len,
                      name=f"fsk small: {S} samples, {n_codes} codes x {n_chips} chips, sps {sps}")


def fsk_realistic(seed: int = 2, seconds: float = 1.0, n_codes: int = 16, n_chips: int = 8192, sps: int = 8,
                  fs_hz: float = 8e6, f_lo_hz: float = 1e6, n_tags: int = 40, snr_range=(-15.0, 0.0),
                  chip_lengths: Optional[Sequence[int]] = None, fft_len: int = 0) -> FskWorkload:
    """1 s at 8 MS/s of int16 samples, 16 codes x 8192 chips at 8 samples/chip
    on tones +/-500 kHz around a band centre 1 MHz off the receiver's, a
    200-tap band-pass filter, 40 tags with SNR U[-15, 0] dB.  chip_lengths
    (optional) gives each code its own length; fft_len (optional) the window
    N, which also sets the smallest gap between transmissions of one code
    (2 N)."""
    S = int(round(seconds * fs_hz))
    lens = list(chip_lengths) if chip_lengths is not None else [n_chips] * n_codes
    chips = [random_chips(n, seed * 1_000_003 + c) for c, n in enumerate(lens)]
    return fsk_stream(seed, S, chips, sps, fs_hz, 5e5, -5e5, f_lo_hz, n_tags, snr_range, fft_len=fft_len,
                      name=f"fsk realistic: {S} samples at {fs_hz/1e6:g} MS/s, {len(chips)} codes, sps {sps}")


def fsk_periodic(seed: int = 7, seconds: float = 1.0, fs_hz: float = 4e6, n_codes: int = 4, n_chips: int = 1024,
                 sps: int = 4, period_s=(0.04, 0.06), snr_range=(-5.0, -2.0), f_lo_hz: float = 250e3,
                 offset_hz: float = 2e3, sigma: float = 2048.0):
    """A stream for the scheduler: every tag transmits its code periodically
    (Section 2.2: tracked tags are predicted one period ahead).  Tag c's period
    is drawn from period_s (seconds, rounded to whole samples) and its first
    transmission from [0, period); each transmission has its own phase, a
    carrier offset within +/-offset_hz and an SNR from snr_range.  Returns
    (FskWorkload, periods in samples)."""
    rng = np.random.default_rng(seed)
    S = int(round(seconds * fs_hz))
    chips = [random_chips(n_chips, seed * 1_000_003 + c) for c in range(n_codes)]
    w = FskWorkload(f"fsk periodic: {S} samples at {fs_hz/1e6:g} MS/s, {n_codes} codes x {n_chips} chips, sps {sps}",
                    np.zeros((0, 2), np.int16), chips, sps, fs_hz, 5e5, -5e5, f_lo_hz,
                    bandpass_taps(200, 7.5e5, fs_hz), 0, [], sigma)
    z = rng.standard_normal(2 * S) * sigma
    x = z[0::2] + 1j * z[1::2]
    L = n_chips * sps
    periods = []
    for c in range(n_codes):
        per = int(round(rng.uniform(*period_s) * fs_hz))
        periods.append(float(per))
        d = int(rng.integers(0, per))
        while d + L <= S:
            tg = Tag(code=c, delay=float(d), freq_hz=float(rng.uniform(-offset_hz, offset_hz)), bin=-1,
                     snr_db=float(rng.uniform(*snr_range)), phase=float(rng.uniform(0, 2 * math.pi)))
            inject_fsk(x, w, tg)
            w.tags.append(tg)
            d += per
    w.iq16 = quantise_iq(x)
    return w, periods
