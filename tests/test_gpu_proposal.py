"""The learned proposal on the GPU against its FP64 oracle: features, logits,
gradients of every parameter, the Adam step, training progress, and the
proposal-driven search against the exhaustive one (GPU only)."""
import numpy as np
import pytest

from oracle import acq
from oracle import proposal as pr
from paper_2005_10445_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _net(torch, C, K, seed=0):
    from paper_2005_10445_gb300.binding import Proposal
    net = Proposal(C, K, seed)
    p = pr.init_params(C, K, seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)
    net.set_params(pr.flatten(p).astype(np.float32))
    return net, pr.unflatten(pr.flatten(p).astype(np.float32).astype(np.float64), C, K)


def _windows(wl, first, stride, wlen, n_win):
    xs = wl.x.astype(np.complex128)
    out = []
    for w in range(n_win):
        a = first + w * stride
        seg = np.zeros(wlen, np.complex128)
        hi = min(a + wlen, wl.n_samples)
        seg[: hi - a] = xs[a:hi]
        out.append(seg)
    return out


def test_features_match_oracle(torch_cuda):
    """Spectrum features, and zero carrier-line features while no grid is set."""
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import Proposal
    net = Proposal(4, 3, 0)
    assert net.feature_len == pr.SEG + 3
    wl = synth.small(seed=11)
    x = torch.from_numpy(wl.iq().copy()).cuda()
    n_win, stride, wlen = 5, 5000, 2 * pr.SEG
    feat = torch.empty(n_win * net.feature_len, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    net.features(st.cuda_stream, x.data_ptr(), wl.n_samples, 1234, stride, wlen, n_win, feat.data_ptr())
    st.synchronize()
    got = feat.cpu().numpy().reshape(n_win, net.feature_len)
    for w, seg in enumerate(_windows(wl, 1234, stride, wlen, n_win)):
        np.testing.assert_allclose(got[w, :pr.SEG], pr.features(seg), atol=1e-4)
    assert (got[:, pr.SEG:] == 0).all()


def test_line_features_match_oracle(torch_cuda):
    """Carrier-line features on the GPU (FP32, exact fixed-point phase, phasor
    steps within a chunk) against the FP64 definition, on windows with tags,
    noise only and the zero-padded stream end; bounded in log10 units."""
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import Proposal
    wl = synth.small(seed=12, snr_range=(0.0, 6.0))
    K = len(wl.freqs_hz)
    net = Proposal(len(wl.chips), K, 0)
    net.set_grid(wl.fs_hz, wl.freqs_hz)
    x = torch.from_numpy(wl.iq().copy()).cuda()
    n_win, stride, wlen = 9, 4500, 2 * pr.SEG
    feat = torch.empty(n_win * net.feature_len, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    net.features(st.cuda_stream, x.data_ptr(), wl.n_samples, 0, stride, wlen, n_win, feat.data_ptr())
    st.synchronize()
    got = feat.cpu().numpy().reshape(n_win, net.feature_len)[:, pr.SEG:]
    want = np.array([pr.line_features(seg, wl.fs_hz, wl.freqs_hz) for seg in _windows(wl, 0, stride, wlen, n_win)])
    np.testing.assert_allclose(got, want, atol=2e-3)
    assert want.max() > 1.5  # some window holds a strong line


def test_logits_and_gradients_match_oracle(torch_cuda):
    torch = torch_cuda
    C, K, B = 6, 5, 24
    net, p = _net(torch, C, K, seed=3)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((B, pr.SEG)).astype(np.float32)
    L = rng.uniform(0.0, 3.0, size=(B, K)).astype(np.float32)
    code = rng.integers(0, C, B).astype(np.int32)
    bin_ = rng.integers(0, K, B).astype(np.int32)
    code[rng.uniform(size=B) < 0.3] = -1
    bin_[code < 0] = -1
    present = (code >= 0).astype(float)
    d_f = torch.from_numpy(np.concatenate([f, L], axis=1)).cuda()
    d_c = torch.from_numpy(code).cuda()
    d_b = torch.from_numpy(bin_).cuda()
    zc = torch.empty(B * C, device="cuda")
    zb = torch.empty(B * K, device="cuda")
    zp = torch.empty(B, device="cuda")
    st = torch.cuda.current_stream()
    net.logits(st.cuda_stream, d_f.data_ptr(), B, False, zc.data_ptr(), zb.data_ptr(), zp.data_ptr())
    st.synchronize()
    _, rc, rb, rp = pr.forward(p, f.astype(np.float64), L.astype(np.float64))
    np.testing.assert_allclose(zc.cpu().numpy().reshape(B, C), rc, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(zb.cpu().numpy().reshape(B, K), rb, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(zp.cpu().numpy(), rp, rtol=1e-4, atol=1e-4)
    # FP16 weights (inference path): close, not exact
    net.logits(st.cuda_stream, d_f.data_ptr(), B, True, zc.data_ptr(), 0, 0)
    st.synchronize()
    err16 = np.abs(zc.cpu().numpy().reshape(B, C) - rc).max() / np.abs(rc).max()
    assert err16 < 2e-2
    # loss and every parameter's gradient
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(net.n_params, device="cuda")
    net.loss_grad(st.cuda_stream, d_f.data_ptr(), d_c.data_ptr(), d_b.data_ptr(), B, loss.data_ptr(), grad.data_ptr())
    st.synchronize()
    ref_loss = pr.loss(p, f.astype(np.float64), np.maximum(code, 0), np.maximum(bin_, 0), present,
                       L.astype(np.float64))
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)
    g = pr.unflatten(grad.cpu().numpy().astype(np.float64), C, K)
    ref = pr.grads(p, f.astype(np.float64), np.maximum(code, 0), np.maximum(bin_, 0), present,
                   L.astype(np.float64))
    for k in pr.PARAM_ORDER:
        rel = np.linalg.norm(g[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-12)
        assert rel < 1e-4, (k, rel)


def test_adam_step_matches_reference_update(torch_cuda):
    torch = torch_cuda
    C, K = 3, 4
    net, p = _net(torch, C, K, seed=5)
    w0 = net.get_params().astype(np.float64)
    g = np.random.default_rng(6).standard_normal(net.n_params).astype(np.float32)
    d_g = torch.from_numpy(g).cuda()
    st = torch.cuda.current_stream()
    lr = 1e-3
    for _ in range(2):
        net.adam(st.cuda_stream, lr, d_g.data_ptr())
    st.synchronize()
    m = np.zeros_like(w0)
    v = np.zeros_like(w0)
    w = w0.copy()
    for t in (1, 2):
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g.astype(np.float64) ** 2
        w -= lr * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
    np.testing.assert_allclose(net.get_params(), w, rtol=1e-5, atol=1e-6)


def test_training_lowers_the_loss(torch_cuda):
    """A separable toy problem: the presence and bin labels are written into
    the features; 60 Adam steps must cut the loss by more than half."""
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import Proposal
    C, K, B = 4, 5, 64
    net = Proposal(C, K, 7)
    rng = np.random.default_rng(8)
    f = rng.standard_normal((B, pr.SEG)).astype(np.float32) * 0.1
    code = rng.integers(0, C, B).astype(np.int32)
    bin_ = rng.integers(0, K, B).astype(np.int32)
    for i in range(B):
        f[i, 400 * bin_[i]: 400 * bin_[i] + 200] += 2.0
        f[i, 2048 + 300 * code[i]: 2048 + 300 * code[i] + 100] += 2.0
    f = np.concatenate([f, np.zeros((B, K), np.float32)], axis=1)  # no carrier-line evidence
    d_f, d_c, d_b = (torch.from_numpy(a).cuda() for a in (f, code, bin_))
    loss = torch.zeros(1, device="cuda")
    st = torch.cuda.current_stream()
    first = None
    for it in range(60):
        net.loss_grad(st.cuda_stream, d_f.data_ptr(), d_c.data_ptr(), d_b.data_ptr(), B, loss.data_ptr())
        if first is None:
            st.synchronize()
            first = float(loss.item())
        net.adam(st.cuda_stream, 3e-3)
    st.synchronize()
    assert float(loss.item()) < 0.5 * first


def _proposed(torch, wl, net, topk, tau, cap=256, wpl=0, bins=False):
    from paper_2005_10445_gb300.binding import DETECTION_DTYPE, Search, run_proposed, run_proposed_bins
    s = Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len, windows_per_launch=wpl)
    x = torch.from_numpy(wl.iq().copy()).cuda()
    out = torch.zeros(cap * 32, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    fn = run_proposed_bins if bins else run_proposed
    nfb = fn(s, net, st.cuda_stream, x.data_ptr(), wl.n_samples, topk, tau, out.data_ptr(), cap, cnt.data_ptr())
    n = int(cnt.item())
    got = out.cpu().numpy().view(DETECTION_DTYPE)[: min(n, cap)].copy()
    ref, n_ref, _ = s.run(x, capacity=cap)
    return got, n, ref, n_ref, nfb


def test_proposed_search_full_fallback_equals_exhaustive(torch_cuda):
    from paper_2005_10445_gb300.binding import Proposal
    wl = synth.small(seed=13, N=8192)
    net = Proposal(len(wl.chips), len(wl.freqs_hz), 1)
    got, n, ref, n_ref, nfb = _proposed(torch_cuda, wl, net, topk=4, tau=2.0)
    assert nfb > 0 and n == n_ref and got.tobytes() == ref.tobytes()


@pytest.mark.parametrize("wpl", [0, 1])
def test_proposed_search_covering_candidates_equals_exhaustive(torch_cuda, wpl):
    """With top-k covering every (code, bin) pair and no fallback, the listed-cell
    path reproduces the exhaustive detections bit for bit; with one window per
    launch group the cells are processed in many chunks of whole windows."""
    from paper_2005_10445_gb300.binding import Proposal
    wl = synth.small(seed=12, N=8192)  # 3 codes x 5 bins = 15 pairs
    net = Proposal(len(wl.chips), len(wl.freqs_hz), 2)
    got, n, ref, n_ref, nfb = _proposed(torch_cuda, wl, net, topk=15, tau=0.0, wpl=wpl)
    assert nfb == 0 and n == n_ref >= 3
    assert got.tobytes() == ref.tobytes()
    ora, _ = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len)
    assert [(int(d["code"]), int(d["window"]), int(d["lag"]), int(d["freq_bin"])) for d in got] == \
        sorted([o.key() for o in ora], key=lambda k: (k[1], k[0]))


def test_checkpoint_resume_is_exact_and_corruption_is_refused(torch_cuda, tmp_path):
    """Save after 4 Adam steps, continue 3 more; a fresh network loaded from
    the file and run the same 3 steps ends bit-identical.  The file's header
    and CRC-32 (checked here against zlib's) pin the format; a flipped
    payload byte, a truncated file and a shape mismatch are refused and leave
    the network unchanged."""
    import struct
    import zlib
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import AtlasError, Proposal
    C, K, B = 5, 4, 16
    rng = np.random.default_rng(21)
    f = torch.from_numpy(rng.standard_normal((B, pr.SEG + K)).astype(np.float32)).cuda()
    code = torch.from_numpy(rng.integers(0, C, B).astype(np.int32)).cuda()
    bin_ = torch.from_numpy(rng.integers(0, K, B).astype(np.int32)).cuda()
    loss = torch.zeros(1, device="cuda")
    st = torch.cuda.current_stream()

    def steps(net, n):
        for _ in range(n):
            net.loss_grad(st.cuda_stream, f.data_ptr(), code.data_ptr(), bin_.data_ptr(), B, loss.data_ptr())
            net.adam(st.cuda_stream, 2e-3)
        st.synchronize()

    a = Proposal(C, K, 3)
    steps(a, 4)
    path = str(tmp_path / "prop.ckpt")
    a.save(path)
    steps(a, 3)
    b = Proposal(C, K, 99)
    b.load(path)
    steps(b, 3)
    assert a.get_params().tobytes() == b.get_params().tobytes()

    raw = open(path, "rb").read()
    magic, ver, nc, nb, crc, n, step = struct.unpack("<8sIiiIqq", raw[:40])
    assert (magic, ver, nc, nb, n, step) == (b"ATLPROP1", 2, C, K, a.n_params, 4)
    assert len(raw) == 40 + 3 * 4 * n and crc == zlib.crc32(raw[40:])
    before = b.get_params().tobytes()
    bad = bytearray(raw)
    bad[100] ^= 0x40
    for blob, name in ((bytes(bad), "flip"), (raw[:-4], "short")):
        p2 = str(tmp_path / name)
        open(p2, "wb").write(blob)
        with pytest.raises(AtlasError):
            b.load(p2)
    with pytest.raises(AtlasError):
        Proposal(C + 1, K, 0).load(path)
    assert b.get_params().tobytes() == before


@pytest.mark.parametrize("wpl", [0, 1])
def test_bin_proposals_covering_every_bin_equal_exhaustive(torch_cuda, wpl):
    """Bin proposals naming every bin, no fallback: every code in every bin is
    listed, so the records equal the exhaustive search's bit for bit."""
    from paper_2005_10445_gb300.binding import Proposal
    wl = synth.small(seed=12, N=8192)
    net = Proposal(len(wl.chips), len(wl.freqs_hz), 2)
    got, n, ref, n_ref, nfb = _proposed(torch_cuda, wl, net, topk=len(wl.freqs_hz), tau=0.0, wpl=wpl, bins=True)
    assert nfb == 0 and n == n_ref >= 3 and got.tobytes() == ref.tobytes()


def test_bin_proposals_on_the_tags_bins_find_the_tags(torch_cuda):
    """A network whose bin head is driven by the carrier-line features alone
    (every weight zero but a = 1): each confident window searches every code in
    its top two bins; every injected tag is still found, with the exhaustive
    search's record, and fewer cells are searched than bins exist."""
    torch = torch_cuda
    from paper_2005_10445_gb300.binding import Proposal
    wl = synth.small(seed=12, N=8192, snr_range=(2.0, 8.0))
    C, K = len(wl.chips), len(wl.freqs_hz)
    net = Proposal(C, K, 2)
    p = {k: np.zeros(v) for k, v in pr.param_shapes(C, K).items()}
    p["wl"] = np.array([8.0, 0.0])
    net.set_params(pr.flatten(p).astype(np.float32))
    got, n, ref, n_ref, nfb = _proposed(torch, wl, net, topk=2, tau=0.0, bins=True)
    assert nfb == 0
    key = lambda d: (int(d["code"]), int(d["window"]), int(d["lag"]), int(d["freq_bin"]))
    by_ref = {key(d): d.tobytes() for d in ref}
    found = {key(d): d.tobytes() for d in got}
    for t in wl.tags:
        N = wl.fft_len
        hop = N - len(wl.chips[t.code]) * wl.sps
        w = min(int(t.delay) // hop, (wl.n_samples - N + hop - 1) // hop)  # the last window is W - 1
        k = (t.code, w, int(t.delay) - w * hop, t.bin)
        assert k in by_ref and k in found and found[k] == by_ref[k]
