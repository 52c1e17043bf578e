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
