"""The multi-rank path on CPU: world_size-2 gloo ranks split one stream by
windows (with halos), search their shards (the FP64 oracle stands in for the
GPU search on CPU-only hosts), gather the detection lists, and must reproduce
the single-process search exactly."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _as_records(dets):
    from paper_2005_10445_gb300.binding import DETECTION_DTYPE
    out = np.zeros(len(dets), DETECTION_DTYPE)
    for i, d in enumerate(dets):
        out[i] = (d.code, d.window, d.lag, d.freq_bin, d.score, d.peak_power, d.toa)
    return out


def _rank(rank, world, port, seed, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import acq
        from paper_2005_10445_gb300 import shard, synth
        wl = synth.small(seed=seed, n_codes=2)
        L = len(wl.chips[0]) * wl.sps
        N = wl.fft_len
        W, hop = shard.window_plan(wl.n_samples, N, L)
        b, e = shard.split_windows(W, world)[rank]
        lo, n_local, kb, ke = shard.local_plan(wl.n_samples, N, L, b, e)
        xl = shard.local_stream(wl.x, N, L, b, e)
        assert xl.shape[0] == n_local
        dets, _ = acq.search(xl, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, N) if e > b else ([], None)
        mine = shard.to_global(_as_records(dets), lo, hop, kb, ke)
        allr = shard.gather(mine)
        if rank == 0:
            full, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, N)
            q.put((allr.tobytes(), _as_records(full).tobytes(), len(full)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("seed", [11, 13])
def test_two_rank_window_split_matches_single_search(seed):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, seed, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, want, n = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert n >= 2
    from paper_2005_10445_gb300.binding import DETECTION_DTYPE
    g = np.frombuffer(got, DETECTION_DTYPE)
    w = np.frombuffer(want, DETECTION_DTYPE)
    assert [tuple(r)[:4] for r in g] == [tuple(r)[:4] for r in w]
    np.testing.assert_allclose(g["score"], w["score"], rtol=1e-12)
    np.testing.assert_allclose(g["toa"], w["toa"], atol=1e-9)


def _fsk_records(dets):
    from paper_2005_10445_gb300.binding import FSK_DETECTION_DTYPE
    out = np.zeros(len(dets), FSK_DETECTION_DTYPE)
    for i, d in enumerate(dets):
        out[i] = (d.code, d.window, d.lag, d.score, d.toa, d.w_c, d.q, d.p_c)
    return out


def _fsk_rank(rank, world, port, seed, q):
    """The FSK front end split the same way: the window plan uses the support
    n_c of d_c in place of L; a shard's stream starts one window early, which
    also supplies the filters' history, and the LO phase of a shard differs
    from the whole stream's by a constant, which the magnitudes of step 5 do
    not see."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import fsk
        from paper_2005_10445_gb300 import shard, synth
        w = synth.fsk_small(seed=seed, n_codes=2, S=60000)
        T = len(w.h_bp) + w.sps - 1
        N, W, hop, n_c = fsk.plan(w.n_samples, len(w.chips[0]), w.sps, T)
        b, e = shard.split_windows(W, world)[rank]
        lo, n_local, kb, ke = shard.local_plan(w.n_samples, N, n_c, b, e)
        xl = shard.local_stream(w.iq16, N, n_c, b, e)
        assert xl.shape == (n_local, 2) and xl.dtype == np.int16
        args = (w.chips, w.sps, w.fs_hz, w.f1_hz, w.f0_hz, w.f_lo_hz, w.h_bp)
        dets, _ = fsk.search(xl, *args) if e > b else ([], None)
        mine = shard.to_global(_fsk_records(dets), lo, hop, kb, ke)
        allr = shard.gather(mine)
        if rank == 0:
            full, _ = fsk.search(w.iq16, *args)
            q.put((allr.tobytes(), _fsk_records(full).tobytes(), len(full)))
    finally:
        dist.destroy_process_group()


def test_two_rank_fsk_split_matches_single_search():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fsk_rank, args=(r, 2, port, 11, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, want, n = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert n >= 2
    from paper_2005_10445_gb300.binding import FSK_DETECTION_DTYPE
    g = np.frombuffer(got, FSK_DETECTION_DTYPE)
    w = np.frombuffer(want, FSK_DETECTION_DTYPE)
    assert [tuple(r)[:3] for r in g] == [tuple(r)[:3] for r in w]
    for f in ("score", "w_c", "q", "p_c"):
        np.testing.assert_allclose(g[f], w[f], rtol=1e-9)
    np.testing.assert_allclose(g["toa"], w["toa"], atol=1e-9)


def test_split_covers_every_window_once():
    from paper_2005_10445_gb300 import shard
    for W in (1, 2, 7, 122):
        for world in (1, 2, 3, 8):
            r = shard.split_windows(W, world)
            owned = [w for b, e in r for w in range(b, e)]
            assert owned == list(range(W))
