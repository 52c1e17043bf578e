"""Continuous ingest and the scheduler (Section 2.2) on the GPU: periodic tags
are first found by a searching task and then tracked at every transmission;
the events agree with the FP64 FSK oracle run on the same task blocks; the
task sequence is deterministic; buffer overruns are reported (GPU only)."""
import numpy as np
import pytest

from oracle import fsk
from paper_2005_10445_gb300 import synth

from test_gpu_fsk import SCORE_RTOL, SUM_RTOL, TOA_ATOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_rt(w, periods, fft_len=0, **opt):
    from paper_2005_10445_gb300.binding import FskSearch, Runtime, rt_default_opts
    s = FskSearch(w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp, fft_len=fft_len)
    o = rt_default_opts(w.fs_hz)
    for k, v in opt.items():
        setattr(o, k, v)
    return Runtime(s, periods, o), o


def feed(rt, w, chunk):
    evs = []
    for a in range(0, w.n_samples, chunk):
        rt.push(w.iq16[a:a + chunk])
        evs.append(rt.pump())
    return np.concatenate(evs)


def oracle_block(w, start, length, code, toa_abs):
    """The oracle's detection of `code` in the task block [start, start + length)
    closest to toa_abs (windows around it only), in absolute samples."""
    T = len(w.h_bp) + w.sps - 1
    N, W, hop, n_c = fsk.plan(length, len(w.chips[code]), w.sps, T)
    wi = min(int((toa_abs - start) // hop), W - 1)
    pairs = [(k, code) for k in (wi - 1, wi, wi + 1) if 0 <= k < W]
    dets, _ = fsk.search(w.iq16[start:start + length], w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz,
                         w.h_bp, pairs=pairs)
    assert dets, (start, length, code)
    return min(dets, key=lambda d: abs(start + d.toa - toa_abs))


def test_runtime_tracks_periodic_tags(torch_cuda):
    from paper_2005_10445_gb300 import binding as b
    w, periods = synth.fsk_periodic(seed=7)
    rt, o = make_rt(w, periods)
    ev = feed(rt, w, 160000)
    st = rt.stats()
    assert st["search_tasks"] >= 1 and st["track_tasks"] >= 10
    assert not np.any(np.isin(ev["kind"], [b.RT_TRACK_MISS, b.RT_TRACK_LOST, b.RT_SEARCH_SKIPPED]))
    L = len(w.chips[0]) * w.sps
    for c in range(len(w.chips)):
        mine = ev[ev["code"] == c]
        # one searching task finds every transmission of its block (a block
        # holds one to three periods), then tracking takes over
        n_s = int(np.sum(mine["kind"] == b.RT_SEARCH_DETECTION))
        assert n_s >= 1 and np.all(mine["kind"][:n_s] == b.RT_SEARCH_DETECTION)
        assert len(set(mine["task_start"][:n_s].tolist())) == 1
        assert len(mine) > n_s and np.all(mine["kind"][n_s:] == b.RT_TRACK_DETECTION)
        truth = np.array([t.delay for t in w.tags if t.code == c])
        for e in mine:  # each event is one of the code's transmissions, each reported once
            assert np.min(np.abs(truth - e["toa"])) <= 2.0
        hit = {int(np.argmin(np.abs(truth - e["toa"]))) for e in mine}
        assert len(hit) == len(mine)
        # every transmission after the first detection whose tracking block has arrived is reported
        first = int(np.argmin(np.abs(truth - mine["toa"][0])))
        margin = (o.track_block - (L + len(w.h_bp) + w.sps - 2)) // 2
        due = [i for i in range(first, len(truth)) if truth[i] - margin + o.track_block <= w.n_samples - 3]
        assert set(due) <= hit
    assert st["search_units"] > 0 and st["track_units"] > 0 and st["searching"] == 0
    # a searching detection and two tracking detections against the oracle on their blocks
    picks = [ev[ev["kind"] == b.RT_SEARCH_DETECTION][0]] + list(ev[ev["kind"] == b.RT_TRACK_DETECTION][[0, -1]])
    for e in picks:
        length = o.search_block if e["kind"] == b.RT_SEARCH_DETECTION else o.track_block
        d = oracle_block(w, int(e["task_start"]), length, int(e["code"]), float(e["toa"]))
        assert abs(e["toa"] - (e["task_start"] + d.toa)) <= TOA_ATOL
        assert e["score"] == pytest.approx(d.score, rel=SCORE_RTOL)
        assert e["w_c"] == pytest.approx(d.w_c, rel=SUM_RTOL)
        assert e["q"] == pytest.approx(d.q, rel=SUM_RTOL)


def test_runtime_task_sequence_is_deterministic(torch_cuda):
    """The same input gives the same events, bit for bit; other push sizes
    change when tasks become ready, and so their order, but not the events."""
    w, periods = synth.fsk_periodic(seed=8, seconds=0.5)
    a = feed(make_rt(w, periods)[0], w, 160000)
    a2 = feed(make_rt(w, periods)[0], w, 160000)
    b_ = feed(make_rt(w, periods)[0], w, 100000)
    assert len(a) > 5 and a.tobytes() == a2.tobytes()
    key = lambda e: np.sort(e, order=["code", "toa"]).tobytes()
    assert key(a) == key(b_)


def test_runtime_reports_overruns(torch_cuda):
    """A cyclic buffer of a little more than one searching block: pushing well
    past it without processing skips searching blocks and loses the tracked
    codes' predicted transmissions; processing resumes on the newest samples."""
    from paper_2005_10445_gb300 import binding as b
    w, periods = synth.fsk_periodic(seed=9, seconds=1.0)
    o0 = b.rt_default_opts(w.fs_hz)
    rt, o = make_rt(w, periods, ring_samples=o0.search_block + o0.track_block + 50000)
    first = feed(rt, w.__class__(**{**w.__dict__, "iq16": w.iq16[:1200000]}), 200000)
    assert np.any(first["kind"] == b.RT_SEARCH_DETECTION)
    rt.push(w.iq16[1200000:3600000])   # 2.4 M samples, five times the buffer, unprocessed
    ev = rt.pump()
    kinds = set(ev["kind"].tolist())
    assert b.RT_SEARCH_SKIPPED in kinds and b.RT_TRACK_LOST in kinds
    rt.push(w.iq16[3600000:])
    ev2 = rt.pump()
    assert np.any(np.isin(ev2["kind"], [b.RT_SEARCH_DETECTION, b.RT_TRACK_DETECTION]))


def test_tracker_single_launch_equals_block_search(torch_cuda):
    """The tracker's one graph launch, reading its block out of a cyclic buffer
    (blocks that wrap around the buffer's end included), reports exactly what
    a search of the same code on the same block copied out linearly reports."""
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import FSK_DETECTION_DTYPE, FskSearch, FskTracker
    w, periods = synth.fsk_periodic(seed=10, seconds=0.3)
    s = FskSearch(w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp)
    ring_n, base, tb = 200000, 700000, 48000
    ring = np.zeros((ring_n, 2), np.int16)
    ring[np.arange(base, base + ring_n) % ring_n] = w.iq16[base:base + ring_n]
    d_ring = torch.from_numpy(ring).cuda()
    n_c = s.windows(0, tb)[3]
    margin = (tb - n_c) // 2
    starts = [(t.code, int(t.delay) - margin) for t in w.tags
              if base <= int(t.delay) - margin and int(t.delay) - margin + tb <= base + ring_n]
    starts += [(0, 780000), (1, 851234)]   # blocks without a transmission of the code
    assert any((st0 % ring_n) + tb > ring_n for _, st0 in starts)   # some blocks wrap around
    trackers = {}
    st = torch.cuda.current_stream()
    out = torch.zeros(64 * 48, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    found = 0
    for code, start in starts:
        t = trackers.setdefault(0, FskTracker(s, code, tb, d_ring.data_ptr(), ring_n))
        got, n = t.run(code, start, stream=st.cuda_stream)
        blk = torch.from_numpy(np.ascontiguousarray(w.iq16[start:start + tb])).cuda()
        s.run_codes_ptr(st.cuda_stream, blk.data_ptr(), tb, start, [code], out.data_ptr(), 64, cnt.data_ptr())
        st.synchronize()
        n_ref = int(cnt.item())
        ref = out.cpu().numpy().view(FSK_DETECTION_DTYPE)[:n_ref]
        assert n == n_ref and got.tobytes() == ref.tobytes(), (code, start)
        found += n
    assert found >= 2
    # one window, one code: demodulation, the transforms, selection and the peak sums
    assert 6 <= trackers[0].kernels() <= 10


def test_code_subsets_across_length_groups(torch_cuda):
    """atlas_fsk_run_codes with a subset spanning two code-length groups (and a
    continuing LO phase) reports exactly the full search's records of those
    codes; an empty list reports nothing."""
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import FSK_DETECTION_DTYPE, FskSearch
    w = synth.fsk_realistic(seed=61, seconds=0.04, chip_lengths=[1024, 2048, 1024, 2048, 1024], sps=8,
                            n_tags=6, snr_range=(-8.0, -2.0))
    s = FskSearch(w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp)
    iq = torch.from_numpy(np.ascontiguousarray(w.iq16)).cuda()
    full, n_full = s.run(iq)
    assert n_full >= 3
    st = torch.cuda.current_stream()
    out = torch.zeros(256 * 48, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for subset in ([4, 1], [0, 3], [2], []):
        s.run_codes_ptr(st.cuda_stream, iq.data_ptr(), w.n_samples, 0, subset, out.data_ptr(), 256, cnt.data_ptr())
        st.synchronize()
        n = int(cnt.item())
        got = out.cpu().numpy().view(FSK_DETECTION_DTYPE)[:n]
        want = full[np.isin(full["code"], subset)]
        assert n == len(want) and got.tobytes() == want.tobytes(), subset


def test_runtime_codes_of_two_lengths(torch_cuda):
    """Tags of two code lengths: each length gets its own tracking graph; every
    code is found by a searching task and then tracked without a miss."""
    from paper_2005_10445_gb300 import binding as b
    # each stream carries its own noise, so the sum has 3 dB more: the tags are stronger
    w, periods = synth.fsk_periodic(seed=12, seconds=0.6, n_codes=4, n_chips=1024, snr_range=(-2.0, 1.0))
    w2, periods2 = synth.fsk_periodic(seed=13, seconds=0.6, n_codes=2, n_chips=512, snr_range=(0.0, 3.0))
    # one stream holding both sets of tags: the second set's samples added to the first's
    x = w.iq16.astype(np.int32) + w2.iq16.astype(np.int32)
    merged = w.__class__(**{**w.__dict__, "iq16": np.clip(x, -32768, 32767).astype(np.int16),
                            "chips": list(w.chips) + list(w2.chips),
                            "tags": list(w.tags) + [t.__class__(**{**t.__dict__, "code": t.code + 4})
                                                    for t in w2.tags]})
    rt, o = make_rt(merged, list(periods) + list(periods2))
    ev = feed(rt, merged, 160000)
    assert not np.any(np.isin(ev["kind"], [b.RT_TRACK_MISS, b.RT_TRACK_LOST]))
    for c in range(6):
        mine = ev[ev["code"] == c]
        assert np.sum(mine["kind"] == b.RT_SEARCH_DETECTION) >= 1
        assert np.sum(mine["kind"] == b.RT_TRACK_DETECTION) >= 2, c


def test_runtime_over_a_two_pass_plan(torch_cuda):
    """An FSK context with N = 2^18 (sixteen blocks of 2^14 points, two passes,
    forward and inverse): searching blocks of two windows, tracking blocks of
    one zero-padded window run as captured graphs.  Every tag is found and
    then tracked at each transmission, within two samples of its delay."""
    from paper_2005_10445_gb300 import binding as b
    # periods above N / fs, so a window holds at most one transmission of a code
    w, periods = synth.fsk_periodic(seed=14, seconds=1.2, n_codes=3, period_s=(0.07, 0.09))
    rt, o = make_rt(w, periods, fft_len=1 << 18)
    ev = feed(rt, w, 160000)
    assert not np.any(np.isin(ev["kind"], [b.RT_TRACK_MISS, b.RT_TRACK_LOST, b.RT_SEARCH_SKIPPED]))
    for c in range(3):
        mine = ev[ev["code"] == c]
        assert np.sum(mine["kind"] == b.RT_SEARCH_DETECTION) >= 1
        assert np.sum(mine["kind"] == b.RT_TRACK_DETECTION) >= 5, c
        truth = np.array([t.delay for t in w.tags if t.code == c])
        for e in mine:
            assert np.min(np.abs(truth - e["toa"])) <= 2.0
