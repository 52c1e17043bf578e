"""FSK front end: CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Bar:
* demodulation (steps 1-5): the GPU filters by FP32 4096-point transforms,
  the oracle by FP64 direct convolution.  A relative FP32 transform error of
  order 1e-6 on |f_b| is allowed ten times over: |delta a_b| <= eta =
  1e-5 * rms(a_b), so |delta u| <= 2 eta and |delta d| <= 4 eta / (a_1 + a_0)
  (the quotient's sensitivity), plus 1e-6 absolute;
* detections: (code, window, lag) identical; score within 1e-4 relative; the
  FP64 peak sums w_c, q, p_c within 1e-4 relative (FP32 d against FP64 d);
  arrival time within 1e-3 samples, the bar of the coherent search.  The
  parabola's offset moves by about (sps / 4) sqrt(2) rho / sqrt(score) for a
  relative error rho of d (correlation errors are a fixed fraction rho of
  sqrt(floor); the peak is c0 = sqrt(score floor) with a mainlobe one chip
  wide), far inside 1e-3 for rho near 1e-6.
* cells searched below the default threshold (tests that lower it): the same
  absolute correlation error is a larger fraction of a smaller peak, so the
  score, w_c, p_c and ToA bars widen by sqrt(49 / score), the ratio of the
  peak at the default threshold to the peak at the cell's score.
"""
import numpy as np
import pytest

from oracle import fsk
from paper_2005_10445_gb300 import synth

pytestmark = pytest.mark.gpu

SCORE_RTOL = 1e-4
SUM_RTOL = 1e-4
TOA_ATOL = 1e-3
MAX_TOA_ERR = [0.0]   # largest |GPU - oracle| ToA / widening seen (printed by the last test)


@pytest.fixture(scope="module")
def torch_cuda(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make(w, **kw):
    from paper_2005_10445_gb300.binding import FskSearch
    return FskSearch(w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp, fft_len=w.fft_len, **kw)


def gpu_run(torch, w, capacity=4096, **kw):
    s = make(w, **kw)
    iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).cuda()
    dets, n = s.run(iq, capacity=capacity)
    return s, dets, n


def oracle(w, pairs=None, threshold=fsk.DEFAULT_THRESHOLD):
    dets, _ = fsk.search(w.iq16, w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp, w.fft_len,
                         threshold=threshold, pairs=pairs)
    return dets


def compare(gpu, ora):
    """Detections equal.  Below the default threshold (cells searched with a
    lower one) a correlation value is closer to the noise: with an absolute
    error that stays a fixed fraction of the r.m.s. correlation, the relative
    error of the score and of the sums grows as sqrt(49 / score)."""
    g_keys = [(int(d["code"]), int(d["window"]), int(d["lag"])) for d in gpu]
    assert sorted(g_keys) == sorted(o.key() for o in ora)
    by = {o.key(): o for o in ora}
    for d in gpu:
        o = by[(int(d["code"]), int(d["window"]), int(d["lag"]))]
        k = max(1.0, (fsk.DEFAULT_THRESHOLD / max(o.score, 1e-6)) ** 0.5)
        assert d["score"] == pytest.approx(o.score, rel=SCORE_RTOL * k)
        assert d["w_c"] == pytest.approx(o.w_c, rel=SUM_RTOL * k)
        assert d["q"] == pytest.approx(o.q, rel=SUM_RTOL)
        assert d["p_c"] == pytest.approx(o.p_c, rel=SUM_RTOL * k)
        err = abs(d["toa"] - o.toa)
        MAX_TOA_ERR[0] = max(MAX_TOA_ERR[0], err / k)
        assert err <= TOA_ATOL * k, (o.key(), err, k)


def demod_bound(x, g1, g0, start, stop):
    a1 = np.abs(fsk.filter_range(x, g1, start, stop))
    a0 = np.abs(fsk.filter_range(x, g0, start, stop))
    eta = 1e-5 * max(np.sqrt(np.mean(a1 ** 2)), np.sqrt(np.mean(a0 ** 2)))
    s = np.maximum(a1 + a0, 1e-30)
    return 4 * eta / s + 1e-6, 2 * eta + 1e-6


def test_demod_matches_oracle(torch_cuda):
    torch = torch_cuda
    w = synth.fsk_small(seed=4)
    s = make(w)
    iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).cuda()
    S = w.n_samples
    start, count = -5, S + 17    # reaches before the stream and past its end
    d = torch.empty(count, device="cuda")
    u = torch.empty(count, device="cuda")
    st = torch.cuda.current_stream()
    s.demod_ptr(st.cuda_stream, iq.data_ptr(), S, start, count, d.data_ptr(), u.data_ptr())
    st.synchronize()
    gd, gu = d.cpu().numpy().astype(np.float64), u.cpu().numpy().astype(np.float64)
    x = fsk.lo_mix(fsk.iq_to_complex(w.iq16), w.f_lo_hz, w.fs_hz)
    g1, g0 = fsk.filters(w.h_bp, w.f1_hz, w.f0_hz, w.sps, w.fs_hz)
    od, ou = fsk.demod_range(x, g1, g0, start, start + count)
    assert np.all(gd[:5] == 0) and np.all(gd[5 + S:] == 0) and np.all(gu[5 + S:] == 0)
    bd, bu = demod_bound(x, g1, g0, 0, S)
    assert np.all(np.abs(gd[5:5 + S] - od[5:5 + S]) <= bd), np.max(np.abs(gd[5:5 + S] - od[5:5 + S]) / bd)
    assert np.all(np.abs(gu[5:5 + S] - ou[5:5 + S]) <= bu), np.max(np.abs(gu[5:5 + S] - ou[5:5 + S]) / bu)


def test_code_demod_matches_oracle(torch_cuda):
    w = synth.fsk_small(seed=5)
    s = make(w)
    g1, g0 = fsk.filters(w.h_bp, w.f1_hz, w.f0_hz, w.sps, w.fs_hz)
    for c, ch in enumerate(w.chips):
        got = s.code_demod(c).astype(np.float64)
        want, _ = fsk.code_demod(ch, w.sps, w.f1_hz, w.f0_hz, w.fs_hz, g1, g0)
        assert got.shape == want.shape
        r = np.zeros(want.shape[0], np.complex128)
        r[: len(ch) * w.sps] = fsk.replica(ch, w.sps, w.f1_hz, w.f0_hz, w.fs_hz)
        bd, _ = demod_bound(r, g1, g0, 0, want.shape[0])
        assert np.all(np.abs(got - want) <= bd), np.max(np.abs(got - want) / bd)


def test_tiny_parity(torch_cuda):
    w = synth.fsk_tiny()
    s, dets, n = gpu_run(torch_cuda, w)
    ora = oracle(w)
    assert n == len(ora) >= 1
    compare(dets, ora)
    t = w.tags[0]
    assert any(abs(d["toa"] - t.delay) < 0.5 for d in dets)


def test_small_parity_and_tags(torch_cuda):
    w = synth.fsk_small(seed=11)
    s, dets, n = gpu_run(torch_cuda, w)
    ora = oracle(w)
    assert n == len(ora) >= len(w.tags)
    compare(dets, ora)


@pytest.mark.parametrize("n_chips", [1024, 2048, 4096, 8192])
def test_transform_sizes(torch_cuda, n_chips):
    """N = 2^14 (one block), 2^15, 2^16, 2^17 (4, 8 and 16 blocks of 2^13
    points, two passes); about 2.7 windows of stream, ragged tail, two codes."""
    L = n_chips * 8
    S = int(2.7 * 2 * L) + 1234
    w = synth.fsk_realistic(seed=20 + n_chips, seconds=S / 8e6, n_codes=2, n_chips=n_chips, n_tags=3,
                            snr_range=(-12.0, -3.0))
    s, dets, n = gpu_run(torch_cuda, w)
    Wn, hop, N, n_c = s.windows(0, w.n_samples)
    assert N == 2 * L and Wn >= 3
    ora = oracle(w)
    assert n == len(ora) >= 1
    compare(dets, ora)


@pytest.mark.parametrize("fft_len,block_log2,seconds", [(1 << 18, 0, 0.075), (1 << 18, 13, 0.075),
                                                        (1 << 18, 14, 0.075), (1 << 17, 14, 0.045)])
def test_two_pass_only_plans(torch_cuda, fft_len, block_log2, seconds):
    """Plans with no cluster form: N = 2^18 as 32 blocks of 2^13 points or 16
    of 2^14 (and the default there), N = 2^17 as 8 blocks of 2^14; about 2.7
    windows of stream, ragged tail, two codes."""
    w = synth.fsk_realistic(seed=23, seconds=seconds, n_codes=2, n_tags=3, snr_range=(-12.0, -3.0),
                            fft_len=fft_len)
    s, dets, n = gpu_run(torch_cuda, w, block_log2=block_log2)
    Wn, hop, N, n_c = s.windows(0, w.n_samples)
    assert N == fft_len and Wn >= 3
    ora = oracle(w)
    assert n == len(ora) >= 1
    compare(dets, ora)


def test_launch_groups_at_2_18_do_not_change_results(torch_cuda):
    """N = 2^18 in launch groups of 2 windows (several passes of the two-pass
    forms, each with its own scratch fill) against one group: bit-identical."""
    w = synth.fsk_realistic(seed=26, seconds=0.2, n_codes=3, n_tags=4, snr_range=(-12.0, -3.0),
                            fft_len=1 << 18)
    _, ref, n_ref = gpu_run(torch_cuda, w, threshold=0.0)
    _, got, n = gpu_run(torch_cuda, w, threshold=0.0, windows_per_launch=2)
    assert n == n_ref >= 3 * 7 and got.tobytes() == ref.tobytes()


def test_block_sizes_agree_at_2_17(torch_cuda):
    """N = 2^17 as sixteen blocks of 2^13 points or eight of 2^14: different
    factorisations of the same transform, the same detections with scores and
    sums within FP32 rounding of each other."""
    w = synth.fsk_realistic(seed=24, seconds=0.06, n_codes=4, n_tags=5, snr_range=(-12.0, -3.0))
    _, a, na = gpu_run(torch_cuda, w, block_log2=13)
    _, b, nb = gpu_run(torch_cuda, w, block_log2=14)
    assert na == nb >= 1
    assert [(int(d["code"]), int(d["window"]), int(d["lag"])) for d in a] == \
        [(int(d["code"]), int(d["window"]), int(d["lag"])) for d in b]
    for x, y in zip(a, b):
        assert x["score"] == pytest.approx(y["score"], rel=SCORE_RTOL)
        assert x["w_c"] == y["w_c"] and x["q"] == y["q"] and x["toa"] == y["toa"]


def test_mixed_code_lengths(torch_cuda):
    w = synth.fsk_realistic(seed=31, seconds=0.03, chip_lengths=[2048, 4096, 2048], n_tags=4,
                            snr_range=(-10.0, -3.0))
    s, dets, n = gpu_run(torch_cuda, w)
    ora = oracle(w)
    assert n == len(ora) >= 1
    compare(dets, ora)


@pytest.mark.parametrize("wpl", [1, 3])
def test_launch_groups_do_not_change_results(torch_cuda, wpl):
    w = synth.fsk_small(seed=11)
    _, ref, n_ref = gpu_run(torch_cuda, w)
    _, got, n = gpu_run(torch_cuda, w, windows_per_launch=wpl)
    assert n == n_ref and got.tobytes() == ref.tobytes()


def test_repeat_is_bit_identical_and_host_entry(torch_cuda):
    torch = torch_cuda
    w = synth.fsk_small(seed=12)
    s = make(w)
    iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).cuda()
    a, na = s.run(iq)
    b, nb = s.run(iq)
    h, nh = s.run_host(w.iq16)
    assert na == nb == nh and a.tobytes() == b.tobytes() == h.tobytes()


def test_host_entry_many_records(torch_cuda):
    """The host-buffer entry with more records than its eager read-back (64):
    every (window, code) cell reported at threshold 0, equal to the device
    entry's records; a capacity below the count gives its first records."""
    torch = torch_cuda
    w = synth.fsk_realistic(seed=25, seconds=0.05, n_codes=16, n_chips=1024, n_tags=4, snr_range=(-6.0, 0.0))
    s = make(w, threshold=0.0)
    iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).cuda()
    dev, nd = s.run(iq, capacity=8192)
    host, nh = s.run_host(w.iq16, capacity=8192)
    Wn = s.windows(0, w.n_samples)[0]
    assert nd == nh == Wn * 16 > 64 and host.tobytes() == dev.tobytes()
    part, np_ = s.run_host(w.iq16, capacity=100)
    assert np_ == nd and part.tobytes() == dev[:100].tobytes()


@pytest.mark.parametrize("extra", [0, 1000, 11000, 37400])
def test_host_entry_equals_device_entry(torch_cuda, extra):
    """Streams from one support long (one copy chunk) to many demodulation
    blocks (eight chunks): the host entry's chunked copy and demodulation give
    the device entry's records bit for bit (threshold 0: every cell)."""
    torch = torch_cuda
    w0 = synth.fsk_small(seed=16, n_tags=0)
    n_c = make(w0).windows(0, w0.n_samples)[3]
    w = synth.fsk_stream(16, n_c + extra, w0.chips, w0.sps, w0.fs_hz, w0.f1_hz, w0.f0_hz, w0.f_lo_hz, 2,
                         (-3.0, 0.0))
    s = make(w, threshold=0.0)
    iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).cuda()
    dev, nd = s.run(iq, capacity=4096)
    host, nh = s.run_host(w.iq16, capacity=4096)
    assert nd == nh >= 1 and host.tobytes() == dev.tobytes()


def test_capacity_overflow_reports_required_count(torch_cuda):
    w = synth.fsk_small(seed=11)
    s, full, n = gpu_run(torch_cuda, w)
    assert n >= 3
    _, part, n2 = gpu_run(torch_cuda, w, capacity=2)
    assert n2 == n and part.tobytes() == full[:2].tobytes()


def test_noise_only_stream(torch_cuda):
    w = synth.fsk_small(seed=13, n_tags=0)
    _, dets, n = gpu_run(torch_cuda, w)
    assert n == 0 == len(oracle(w))


def test_stream_of_exactly_one_support(torch_cuda):
    """S = n_c: one window with the single lag 0."""
    w0 = synth.fsk_small(seed=14, n_tags=0)
    s = make(w0)
    _, _, N, n_c = s.windows(0, w0.n_samples)
    w = synth.fsk_stream(14, n_c, w0.chips[:1], w0.sps, w0.fs_hz, w0.f1_hz, w0.f0_hz, w0.f_lo_hz, 1,
                         (-3.0, -3.0))
    _, dets, n = gpu_run(torch_cuda, w, threshold=0.0)
    ora = oracle(w, threshold=0.0)
    assert n == len(ora) == 1 and int(dets[0]["lag"]) == 0
    compare(dets, ora)


@pytest.mark.parametrize("fft_len", [0, 1 << 18])
def test_realistic_full_size_sampled(torch_cuda, fft_len):
    """1 s at 8 MS/s, 16 codes x 8192 chips (N = 2^17, sixteen blocks of 2^13
    points; N = 2^18, sixteen blocks of 2^14): every injected tag found at its
    delay; the oracle recomputes the cells of two detections and of one tag."""
    w = synth.fsk_realistic(fft_len=fft_len)
    s, dets, n = gpu_run(torch_cuda, w)
    assert n == len(dets) >= len(w.tags)
    Wn, hop, N, n_c = s.windows(0, w.n_samples)
    # at -15 dB the broad (about one chip wide) correlation peak of a tag can
    # sit a sample or two from its delay: the tag counts as found when a
    # detection of its code has its ToA within two samples
    for t in w.tags:
        near = [d for d in dets if int(d["code"]) == t.code and abs(d["toa"] - t.delay) <= 2.0]
        assert len(near) == 1, (t, [(int(d["window"]) * hop + int(d["lag"]), float(d["toa"])) for d in dets
                                    if int(d["code"]) == t.code])
    rng = np.random.default_rng(3)
    pick = [dets[i] for i in rng.choice(len(dets), size=2, replace=False)]
    t = w.tags[int(rng.integers(0, len(w.tags)))]
    pairs = {(int(d["window"]), int(d["code"])) for d in pick}
    pairs.add((min(int(t.delay) // hop, Wn - 1), t.code))
    ora = oracle(w, pairs=sorted(pairs))
    sel = np.array([d for d in dets if (int(d["window"]), int(d["code"])) in pairs], dtype=dets.dtype)
    compare(sel, ora)


@pytest.mark.parametrize("sps,fs,f1,f0,n_taps,fft_len,n_chips", [
    (3, 3e6, 5e5, -5e5, 60, 0, 150),        # odd samples per chip
    (2, 2e6, 3.5e5, -3.5e5, 30, 0, 400),    # tones that are not orthogonal over a chip
    (4, 4e6, 5e5, -5e5, 1, 0, 150),         # a one-tap band-pass filter: T = sps
    (4, 4e6, 5e5, -5e5, 40, 1024, 100),     # the smallest transform, 2^10
])
def test_fsk_shapes(torch_cuda, sps, fs, f1, f0, n_taps, fft_len, n_chips):
    chips = [synth.random_chips(n_chips, 40 + c) for c in range(2)]
    w = synth.fsk_stream(41, 30000, chips, sps, fs, f1, f0, -1.5e5, 3, (-6.0, 0.0), n_taps=n_taps,
                         cutoff_hz=0.45 * fs, fft_len=fft_len)
    _, dets, n = gpu_run(torch_cuda, w)
    ora = oracle(w)
    assert n == len(ora) >= 1
    compare(dets, ora)


def test_fsk_saturated_samples_and_zero_capacity(torch_cuda):
    """Tags strong enough to clip the int16 range (both sides read the same
    saturated samples), and a run with capacity 0 that only counts."""
    w = synth.fsk_small(seed=15, snr_range=(22.0, 24.0))
    assert np.abs(w.iq16.astype(np.int32)).max() == 32767 or w.iq16.min() == -32768
    s, dets, n = gpu_run(torch_cuda, w)
    ora = oracle(w)
    assert n == len(ora) >= 1
    compare(dets, ora)
    _, none, n0 = gpu_run(torch_cuda, w, capacity=0)
    assert n0 == n and len(none) == 0


@pytest.mark.parametrize("n_chips", [2048, 4096, 8192])
def test_exchange_forms_are_bit_identical(torch_cuda, n_chips):
    """Transforms of 2^15-2^17 points, forward and inverse: the cluster form
    (distributed shared memory) and the two-pass form (device scratch) take
    the same values through the same arithmetic."""
    w = synth.fsk_realistic(seed=50 + n_chips, seconds=(6.3 * 2 * n_chips * 8) / 8e6, n_codes=12,
                            n_chips=n_chips, n_tags=4, snr_range=(-12.0, -3.0))
    _, a, na = gpu_run(torch_cuda, w, exchange=1)
    _, b, nb = gpu_run(torch_cuda, w, exchange=2)
    assert na == nb >= 1 and a.tobytes() == b.tobytes()


def test_zz_report_toa_error():
    """Reports the largest ToA difference the comparisons above saw."""
    print(f"largest FSK ToA difference against the oracle: {MAX_TOA_ERR[0]:.3g} samples (bar {TOA_ATOL})")
    assert MAX_TOA_ERR[0] <= TOA_ATOL
