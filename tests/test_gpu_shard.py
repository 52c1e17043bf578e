"""The multi-rank path with the library on the GPU: two gloo ranks (spawned
processes sharing one GPU; their kernels are independent and the only
exchange is the host-side gather) split one stream by windows with halos,
search their shards with atlas_acq_run, gather the detection lists, and must
reproduce the single-process library search."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2005_10445_gb300 import binding, shard, synth
        wl = synth.realistic(seconds=0.25)
        L = len(wl.chips[0]) * wl.sps
        N = wl.fft_len
        W, hop = shard.window_plan(wl.n_samples, N, L)
        b, e = shard.split_windows(W, world)[rank]
        lo, n_local, kb, ke = shard.local_plan(wl.n_samples, N, L, b, e)
        xl = shard.local_stream(wl.x, N, L, b, e)
        assert xl.shape[0] == n_local
        s = binding.Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=N)
        x = torch.from_numpy(np.stack([xl.real, xl.imag], axis=1).astype(np.float32)).cuda()
        dets, n, _ = s.run(x, capacity=4096)
        assert n == len(dets)
        mine = shard.to_global(dets, lo, hop, kb, ke)
        allr = shard.gather(mine)
        if rank == 0:
            full, nf, _ = s.run(torch.from_numpy(wl.iq().copy()).cuda(), capacity=4096)
            q.put((allr.tobytes(), full.tobytes(), nf, W))
        s.close()
    finally:
        dist.destroy_process_group()


def test_two_rank_window_split_with_the_library():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, want, n, W = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from paper_2005_10445_gb300.binding import DETECTION_DTYPE
    g = np.frombuffer(got, DETECTION_DTYPE)
    w = np.frombuffer(want, DETECTION_DTYPE)
    assert n >= 10 and len(w) == n
    # the same windows hold the same samples, and the mix phase is
    # window-relative: the shards' cells, and so the scores, equal the whole
    # stream's
    assert [tuple(r)[:4] for r in g] == [tuple(r)[:4] for r in w]
    np.testing.assert_array_equal(g["score"], w["score"])
    # the refinement's phase starts at the shard's first sample: the same
    # direct correlation and parabola up to rounding
    np.testing.assert_allclose(g["peak_power"], w["peak_power"], rtol=1e-5)
    np.testing.assert_allclose(g["toa"], w["toa"], atol=1e-6)
    print(f"{W} windows on 2 ranks: {n} detections")
