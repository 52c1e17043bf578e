"""Batched search (many receiver streams in one CUDA graph) and the autotuner,
against the per-stream entry point and the FP64 oracle (GPU only)."""
import numpy as np
import pytest

from oracle import acq
from paper_2005_10445_gb300 import synth

from test_gpu_parity import compare_all_cells, compare_detections, near_tie_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def small_batch():
    # 3 streams at 2 or 4 MS/s, 5 codes of three lengths (M = 2^11 .. 2^13), 3-7 bins
    return synth.batch(seed=5, n_streams=3, duration_s=(0.008, 0.012), fs_choices=(2e6, 4e6), n_codes=5,
                       chip_choices=(600, 1100, 2100), bins=(3, 7), tags_per_group=2, snr_range=(-10.0, -2.0))


def test_batch_graph_matches_streams_and_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import DETECTION_DTYPE, Batch, Search
    wls = small_batch()
    cap = 256
    searches = [Search(w.chips, w.sps, w.fs_hz, w.freqs_hz) for w in wls]
    xs = [torch.from_numpy(w.iq().copy()).cuda() for w in wls]
    out = torch.zeros(len(wls) * cap * 32, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(len(wls), dtype=torch.int32, device="cuda")
    b = Batch(searches, [x.data_ptr() for x in xs], [w.n_samples for w in wls], out.data_ptr(), cap, cnt.data_ptr())
    assert b.kernels() > 0
    st = torch.cuda.current_stream()
    results = []
    for _ in range(2):  # the graph can be replayed
        out.zero_()
        b.run(st.cuda_stream)
        st.synchronize()
        results.append((out.cpu().numpy().copy(), cnt.cpu().numpy().copy()))
    assert results[0][0].tobytes() == results[1][0].tobytes() and (results[0][1] == results[1][1]).all()
    dets_all = results[0][0].view(DETECTION_DTYPE).reshape(len(wls), cap)
    for i, (w, s, x) in enumerate(zip(wls, searches, xs)):
        n = int(results[0][1][i])
        got = dets_all[i, :min(n, cap)]
        ref, n_ref, _ = s.run(x, capacity=cap)
        assert n == n_ref and got.tobytes() == ref.tobytes()
        ora, _ = acq.search(w.x, w.chips, w.sps, w.fs_hz, w.freqs_hz, 0)
        assert n == len(ora)
        compare_detections(got, ora)
        # every injected tag found
        found = {(int(d["code"]), int(d["window"]), int(d["lag"])) for d in got}
        for t in w.tags:
            W, hop, N = s.windows(t.code, w.n_samples)
            wi = min(int(t.delay) // hop, W - 1)
            assert (t.code, wi, int(t.delay) - wi * hop) in found
    b.close()


def test_batch_rejects_shared_context(torch_cuda):
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import AtlasError, Batch, Search
    w = small_batch()[0]
    s = Search(w.chips, w.sps, w.fs_hz, w.freqs_hz)
    x = torch.from_numpy(w.iq().copy()).cuda()
    out = torch.zeros(2 * 16 * 32, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(AtlasError):
        Batch([s, s], [x.data_ptr()] * 2, [w.n_samples] * 2, out.data_ptr(), 16, cnt.data_ptr())


def test_autotune_choice_cache_and_parity(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import Search
    w = synth.small(seed=12)
    x = torch.from_numpy(w.iq().copy()).cuda()
    st = torch.cuda.current_stream()
    cache = str(tmp_path / "tune.jsonl")
    s1 = Search(w.chips, w.sps, w.fs_hz, w.freqs_hz, fft_len=w.fft_len)
    s1.autotune(st.cuda_stream, x.data_ptr(), w.n_samples, cache)
    t1 = s1.tuning(0)
    assert t1[0] in (4, 5) and t1[1] >= 1 and t1[2] in (0, 1)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"tile_log2"' in lines[0]
    s2 = Search(w.chips, w.sps, w.fs_hz, w.freqs_hz, fft_len=w.fft_len)
    s2.autotune(st.cuda_stream, x.data_ptr(), w.n_samples, cache)   # from the cache
    assert s2.tuning(0) == t1
    assert len(open(cache).read().strip().splitlines()) == 1
    dets, n, _ = s2.run(x)
    ora, _ = acq.search(w.x, w.chips, w.sps, w.fs_hz, w.freqs_hz, w.fft_len)
    assert n == len(ora)
    compare_detections(dets, ora)


def test_batch_full_size_sampled(torch_cuda):
    """The batching workload at full size (8 streams, 69 M samples, 64 codes of
    2048-16384 chips including 2^15-point split transforms, 15-63 bins) in one
    graph launch with autotuned plans; the oracle recomputes, bin by bin, the
    (window, code) cells of two detections and one injected tag per stream."""
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import DETECTION_DTYPE, Batch, Search
    wls = synth.batch()
    cap = 4096
    searches = [Search(w.chips, w.sps, w.fs_hz, w.freqs_hz) for w in wls]
    xs = [torch.from_numpy(w.iq().copy()).cuda() for w in wls]
    st = torch.cuda.current_stream()
    for s, x, w in zip(searches, xs, wls):
        s.autotune(st.cuda_stream, x.data_ptr(), w.n_samples, None)
    out = torch.zeros(len(wls) * cap * 32, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(len(wls), dtype=torch.int32, device="cuda")
    b = Batch(searches, [x.data_ptr() for x in xs], [w.n_samples for w in wls], out.data_ptr(), cap, cnt.data_ptr())
    b.run(st.cuda_stream)
    st.synchronize()
    dets_all = out.cpu().numpy().view(DETECTION_DTYPE).reshape(len(wls), cap)
    counts = cnt.cpu().numpy()
    rng = np.random.default_rng(17)
    for i, (w, s) in enumerate(zip(wls, searches)):
        got = dets_all[i, :min(int(counts[i]), cap)]
        assert len(got) > 0
        pick = [got[j] for j in rng.choice(len(got), size=min(2, len(got)), replace=False)]
        pairs = {(int(d["window"]), int(d["code"])) for d in pick}
        t = w.tags[int(rng.integers(0, len(w.tags)))]
        W, hop, N = s.windows(t.code, w.n_samples)
        pairs.add((min(int(t.delay) // hop, W - 1), t.code))
        ora, _ = acq.search(w.x, w.chips, w.sps, w.fs_hz, w.freqs_hz, 0, pairs=sorted(pairs))
        sel = np.array([d for d in got if (int(d["window"]), int(d["code"])) in pairs], dtype=got.dtype)
        compare_detections(sel, ora)
    b.close()


def test_batch_stream_all_pairs(torch_cuda):
    """One stream of the full batching workload (stream 7: 5.3 M samples at
    4 MS/s, 64 codes of 2048-16384 chips in four length groups, 15 bins): the
    batch graph's records equal the stream's own run, and the oracle (on every
    host core) searches all of its (window, code) pairs; every detection and
    every cell is compared."""
    torch = torch_cuda
    from oracle import parallel
    from paper_2005_10445_gb300.binding import DETECTION_DTYPE, Batch, Search
    wls = synth.batch()
    i = 7
    w = wls[i]
    cap = 4096
    searches = [Search(v.chips, v.sps, v.fs_hz, v.freqs_hz) for v in wls]
    xs = [torch.from_numpy(v.iq().copy()).cuda() for v in wls]
    out = torch.zeros(len(wls) * cap * 32, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(len(wls), dtype=torch.int32, device="cuda")
    b = Batch(searches, [x.data_ptr() for x in xs], [v.n_samples for v in wls], out.data_ptr(), cap, cnt.data_ptr())
    st = torch.cuda.current_stream()
    b.run(st.cuda_stream)
    st.synchronize()
    got = out.cpu().numpy().view(DETECTION_DTYPE).reshape(len(wls), cap)[i, :min(int(cnt[i].item()), cap)].copy()
    b.close()
    ref, n_ref, cells = searches[i].run(xs[i], capacity=cap, cells=True)
    assert got.tobytes() == ref.tobytes() and len(got) == n_ref
    ora, ora_cells, procs = parallel.search(w.x, w.chips, w.sps, w.fs_hz, w.freqs_hz, 0)
    assert len(ora_cells) == len(parallel.all_pairs(w.n_samples, w.chips, w.sps))
    compare_detections(got, ora)
    near_tie_ok(w, compare_all_cells(w, cells, ora_cells))
    print(f"batch stream {i}: {len(ora)} detections over {len(ora_cells)} pairs, oracle on {procs} processes")
