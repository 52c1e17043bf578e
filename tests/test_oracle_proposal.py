"""Pins for the FP64 proposal oracle (features, network, loss, gradients). CPU only."""
import numpy as np
import pytest

from oracle import proposal as pr


def _random_case(B=5, C=7, K=5, seed=0, seg=pr.SEG):
    rng = np.random.default_rng(seed)
    p = pr.init_params(C, K, seed)
    for k in p:  # non-zero biases so every term is exercised
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)
    f = rng.standard_normal((B, seg))
    code = rng.integers(0, C, B)
    bin_ = rng.integers(0, K, B)
    present = (rng.uniform(size=B) > 0.3).astype(float)
    present[0] = 1.0
    present[1] = 0.0
    return p, f, code, bin_, present


def test_param_count_is_about_200k_for_64_codes_63_bins():
    assert 190_000 <= pr.n_params(64, 63) <= 210_000


def test_gradients_match_central_finite_differences():
    p, f, code, bin_, present = _random_case()
    g = pr.grads(p, f, code, bin_, present)
    rng = np.random.default_rng(1)
    for k in pr.PARAM_ORDER:
        flat = p[k].ravel()
        picks = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in picks:
            old = flat[i]
            h = 1e-6 * max(1.0, abs(old))
            flat[i] = old + h
            lp = pr.loss(p, f, code, bin_, present)
            flat[i] = old - h
            lm = pr.loss(p, f, code, bin_, present)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].ravel()[i]
            # points next to a ReLU kink can disagree; skip those few
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)) or abs(fd - an) < 1e-7, (k, i, fd, an)


def test_forward_matches_explicit_loops():
    """Brute force on a tiny input with plain loops (conv, dense, heads)."""
    seg = 64
    p, f, code, bin_, present = _random_case(B=2, C=3, K=4, seed=3, seg=seg)
    P = seg // pr.ST
    p["w1"] = p["w1"][: pr.CH * P]
    cache, zc, zb, zp = pr.forward(p, f)
    for b in range(2):
        x1 = []
        for o in range(pr.CH):
            for q in range(P):
                acc = p["conv_b"][o]
                for t in range(pr.KW):
                    j = pr.ST * q + t
                    acc += p["conv_w"][o, t] * (f[b, j] if j < seg else 0.0)
                x1.append(max(acc, 0.0))
        h = [max(sum(x1[i] * p["w1"][i, j] for i in range(len(x1))) + p["b1"][j], 0.0) for j in range(pr.HID)]
        for c in range(3):
            assert zc[b, c] == pytest.approx(sum(h[j] * p["wc"][j, c] for j in range(pr.HID)) + p["bc"][c], rel=1e-12)
        assert zp[b] == pytest.approx(sum(h[j] * p["wp"][j] for j in range(pr.HID)) + p["bp"][0], rel=1e-12)


def test_psd_of_an_integer_bin_tone_is_closed_form():
    """A tone at integer bin k0 through a periodic Hann window: |X[k0]| = A SEG/2,
    |X[k0 +/- 1]| = A SEG/4, every other bin 0 -- in every segment."""
    A, k0 = 3.0, 700
    n = np.arange(2 * pr.SEG)
    x = A * np.exp(2j * np.pi * k0 * n / pr.SEG)
    f = pr.features(x)
    P = np.zeros(pr.SEG)
    P[k0] = (A * pr.SEG / 2) ** 2
    P[k0 - 1] = P[k0 + 1] = (A * pr.SEG / 4) ** 2
    v = np.log10(P + 1.0)
    np.testing.assert_allclose(f, v - v.mean(), atol=1e-9)


def test_features_ignore_the_overall_level():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(3 * pr.SEG) + 1j * rng.standard_normal(3 * pr.SEG)
    x *= 1e4
    a = pr.features(x)
    b = pr.features(x * 10.0)
    # log10(P + 1) with P >> 1: scaling by 10 adds 2 to every bin, removed by the mean
    np.testing.assert_allclose(a, b, atol=1e-6)


# --- carrier-line features --------------------------------------------------

def _bpsk_window(N=4096, sps=4, fs=1e6, f=1000.0, A=2.5, phase=0.7, seed=4):
    rng = np.random.default_rng(seed)
    chips = rng.choice([-1.0, 1.0], size=N // sps)
    m = np.arange(N)
    return A * np.repeat(chips, sps) * np.exp(1j * (2 * np.pi * f * m / fs + phase))


def test_line_feature_of_a_bpsk_tag_is_closed_form():
    """A noise-free +/-1-chip tag filling the window at offset f: x^2 is the
    tone A^2 e^{i(2 pi 2f m/fs + 2 phi)}, so the squared window's DFT at 2 f_j
    is A^2 times a geometric sum: the ratio to sum |x|^4 = N A^4 is N on the
    tag's bin and sin^2(pi D N) / (N sin^2(pi D)) elsewhere, D = 2 (f - f_j)/fs."""
    N, fs, f = 4096, 1e6, 1000.0
    grid = np.array([-3000.0, -1000.0, 0.0, 1000.0, 1500.0, 3000.0])
    x = _bpsk_window(N=N, fs=fs, f=f)
    L = pr.line_features(x, fs, grid)
    want = []
    for fj in grid:
        D = 2.0 * (f - fj) / fs
        r = float(N) if D == 0 else np.sin(np.pi * D * N) ** 2 / (N * np.sin(np.pi * D) ** 2)
        want.append(np.log10(r + 1.0))
    np.testing.assert_allclose(L, want, rtol=1e-9, atol=1e-9)
    assert int(np.argmax(L)) == 3


def test_line_feature_of_noise_is_near_zero_ratio_one():
    """Complex white noise: E|sum x^2 e|^2 = sum E|x|^4, so the ratio is about 1
    (log10(2) = 0.3) on every bin, and the feature ignores the overall level."""
    rng = np.random.default_rng(9)
    x = rng.standard_normal(1 << 15) + 1j * rng.standard_normal(1 << 15)
    grid = np.linspace(-15500.0, 15500.0, 63)
    L = pr.line_features(x, 8e6, grid)
    assert 0.0 < np.mean(L) < 0.6 and np.max(L) < 1.6
    np.testing.assert_allclose(pr.line_features(1e3 * x, 8e6, grid), L, rtol=1e-9, atol=1e-12)


def test_gradients_with_line_features_match_finite_differences():
    p, f, code, bin_, present = _random_case()
    p["wl"] = np.array([0.7, -0.4])
    rng = np.random.default_rng(5)
    L = rng.uniform(0.0, 3.0, size=(f.shape[0], p["wb"].shape[1]))
    g = pr.grads(p, f, code, bin_, present, L)
    for k in ("wl", "wb", "bb", "wp", "bp"):
        flat = p[k].ravel()
        for i in range(min(4, flat.size)):
            old = flat[i]
            h = 1e-6 * max(1.0, abs(old))
            flat[i] = old + h
            lp = pr.loss(p, f, code, bin_, present, L)
            flat[i] = old - h
            lm = pr.loss(p, f, code, bin_, present, L)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].ravel()[i]) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, g[k].ravel()[i])


def test_planted_line_at_f_instead_of_2f_is_caught(monkeypatch):
    def at_f(xw, fs_hz, freqs_hz):
        xw = np.asarray(xw, np.complex128)
        m = np.arange(xw.shape[0], dtype=np.float64)
        e4 = float(np.sum(np.abs(xw) ** 4))
        return np.array([np.log10(abs(np.dot(xw * xw, np.exp(-2j * np.pi * (f / fs_hz) * m))) ** 2 / e4 + 1.0)
                         for f in freqs_hz])
    monkeypatch.setattr(pr, "line_features", at_f)
    with pytest.raises(AssertionError):
        test_line_feature_of_a_bpsk_tag_is_closed_form()
