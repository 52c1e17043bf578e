"""FP64 CPU oracle of the learned (code, bin) proposal: features, network,
loss and gradients.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU legs, never by the product path.

The paper has no learned component; this part follows the proposal design
that prunes the exhaustive search of Section 3 (every code correlated in
every block, Section 2.1): a small network looks at a block's power spectrum
and ranks (code, bin) candidates, the exhaustive search labels its training
data and stays as the fallback.

Definitions (everything float64):
* features: Welch power spectrum of one window of N samples: non-overlapping
  segments of SEG = 4096 samples, periodic Hann taper h[n] = 1/2 - 1/2 cos(2 pi n / SEG),
  P[f] = mean over segments of |FFT_SEG(seg * h)[f]|^2, v[f] = log10(P[f] + 1),
  feature = v - mean(v)  (so the absolute noise level drops out);
* carrier-line features: for +/-1 chips the square of a transmission,
  (A chip e^{i(2 pi f m/fs + phi)})^2 = A^2 e^{i(2 pi (2f) m/fs + 2 phi)}, is a
  pure tone at twice the carrier offset, so the squared window's DFT at 2 f_k
  shows which bin holds a tag: L[k] = log10(|sum_m x[m]^2 e^{-2 pi i 2 f_k m/fs}|^2
  / sum_m |x[m]|^4 + 1) (the ratio is about 1 for noise and N for a tag that
  fills the window);
* network: conv1d (1 -> CH channels, kernel KW, stride ST, zero padding at the
  end) + ReLU -> flatten (channel-major) -> dense (HID) + ReLU -> three heads:
  code logits (C), bin logits (K), presence logit (1); the carrier-line
  features enter the heads through two learned scalars wl = (a, c): bin logit k
  += a L[k], presence logit += c max_k L[k];
* loss per window: BCE(presence logit, present) + present * (CE(code logits, code)
  + CE(bin logits, bin)); the batch loss is the mean over windows;
* gradients: the chain rule written out layer by layer (backward pass).
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

SEG = 4096
CH, KW, ST, HID = 8, 16, 8, 48

PARAM_ORDER = ("conv_w", "conv_b", "w1", "b1", "wc", "bc", "wb", "bb", "wp", "bp", "wl")


def param_shapes(n_codes: int, n_bins: int, seg: int = SEG) -> Dict[str, Tuple[int, ...]]:
    P = seg // ST
    return {"conv_w": (CH, KW), "conv_b": (CH,), "w1": (CH * P, HID), "b1": (HID,),
            "wc": (HID, n_codes), "bc": (n_codes,), "wb": (HID, n_bins), "bb": (n_bins,),
            "wp": (HID,), "bp": (1,), "wl": (2,)}


def n_params(n_codes: int, n_bins: int) -> int:
    return int(sum(np.prod(s) for s in param_shapes(n_codes, n_bins).values()))


def unflatten(flat: np.ndarray, n_codes: int, n_bins: int) -> Dict[str, np.ndarray]:
    out, o = {}, 0
    for k in PARAM_ORDER:
        shp = param_shapes(n_codes, n_bins)[k]
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float64).ravel() for k in PARAM_ORDER])


def hann(n: int = SEG) -> np.ndarray:
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / n)


def features(xw: np.ndarray, seg: int = SEG) -> np.ndarray:
    """Welch log power spectrum of one window, mean removed."""
    xw = np.asarray(xw, np.complex128)
    n_seg = xw.shape[0] // seg
    h = hann(seg)
    P = np.zeros(seg)
    for s in range(n_seg):
        X = np.fft.fft(xw[s * seg:(s + 1) * seg] * h)
        P += X.real ** 2 + X.imag ** 2
    P /= n_seg
    v = np.log10(P + 1.0)
    return v - v.mean()


def line_features(xw: np.ndarray, fs_hz: float, freqs_hz) -> np.ndarray:
    """Carrier-line features of one window (window-relative sample index m)."""
    xw = np.asarray(xw, np.complex128)
    x2 = xw * xw
    m = np.arange(xw.shape[0], dtype=np.float64)
    e4 = float(np.sum(np.abs(xw) ** 4))
    out = np.zeros(len(freqs_hz))
    for k, f in enumerate(freqs_hz):
        S = np.dot(x2, np.exp(-2j * np.pi * (2.0 * f / fs_hz) * m))
        out[k] = np.log10(abs(S) ** 2 / e4 + 1.0) if e4 > 0 else 0.0
    return out


def forward(p: Dict[str, np.ndarray], f: np.ndarray, L: np.ndarray = None):
    """f: [B, SEG], L: [B, K] carrier-line features (None: zeros).
    Returns (cache, zc [B, C], zb [B, K], zp [B])."""
    B, S = f.shape
    P = S // ST
    fp = np.concatenate([f, np.zeros((B, KW))], axis=1)
    idx = ST * np.arange(P)[:, None] + np.arange(KW)[None, :]          # [P, KW]
    patches = fp[:, idx]                                                  # [B, P, KW]
    a1p = np.einsum("bpt,ot->bop", patches, p["conv_w"]) + p["conv_b"][None, :, None]
    a1 = np.maximum(a1p, 0.0)                                             # [B, CH, P]
    x1 = a1.reshape(B, CH * P)
    hp = x1 @ p["w1"] + p["b1"]
    h = np.maximum(hp, 0.0)
    zc = h @ p["wc"] + p["bc"]
    zb = h @ p["wb"] + p["bb"]
    zp = h @ p["wp"] + p["bp"][0]
    if L is None:
        L = np.zeros_like(zb)
    Lmax = L.max(axis=1)
    zb = zb + p["wl"][0] * L
    zp = zp + p["wl"][1] * Lmax
    cache = dict(patches=patches, a1p=a1p, x1=x1, hp=hp, h=h, L=L, Lmax=Lmax)
    return cache, zc, zb, zp


def _log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=1, keepdims=True))


def loss(p, f, code, bin_, present, L=None) -> float:
    _, zc, zb, zp = forward(p, f, L)
    present = np.asarray(present, np.float64)
    bce = np.maximum(zp, 0) - zp * present + np.log1p(np.exp(-np.abs(zp)))
    B = f.shape[0]
    lc = _log_softmax(zc)
    lb = _log_softmax(zb)
    ce = np.zeros(B)
    for i in range(B):
        if present[i] > 0:
            ce[i] = -lc[i, code[i]] - lb[i, bin_[i]]
    return float(np.mean(bce + ce))


def grads(p, f, code, bin_, present, L=None) -> Dict[str, np.ndarray]:
    """Backward pass of `loss` (chain rule, layer by layer)."""
    cache, zc, zb, zp = forward(p, f, L)
    B = f.shape[0]
    present = np.asarray(present, np.float64)
    sig = 1.0 / (1.0 + np.exp(-zp))
    dzp = (sig - present) / B
    pc = np.exp(_log_softmax(zc))
    pb = np.exp(_log_softmax(zb))
    dzc = np.zeros_like(zc)
    dzb = np.zeros_like(zb)
    for i in range(B):
        if present[i] > 0:
            dzc[i] = pc[i]
            dzc[i, code[i]] -= 1.0
            dzb[i] = pb[i]
            dzb[i, bin_[i]] -= 1.0
    dzc /= B
    dzb /= B
    h = cache["h"]
    g = {"wc": h.T @ dzc, "bc": dzc.sum(0), "wb": h.T @ dzb, "bb": dzb.sum(0),
         "wp": h.T @ dzp, "bp": np.array([dzp.sum()]),
         "wl": np.array([np.sum(dzb * cache["L"]), np.sum(dzp * cache["Lmax"])])}
    dh = dzc @ p["wc"].T + dzb @ p["wb"].T + np.outer(dzp, p["wp"])
    dhp = dh * (cache["hp"] > 0)
    g["w1"] = cache["x1"].T @ dhp
    g["b1"] = dhp.sum(0)
    dx1 = dhp @ p["w1"].T
    da1p = dx1.reshape(cache["a1p"].shape) * (cache["a1p"] > 0)          # [B, CH, P]
    g["conv_w"] = np.einsum("bop,bpt->ot", da1p, cache["patches"])
    g["conv_b"] = da1p.sum(axis=(0, 2))
    return g


def init_params(n_codes: int, n_bins: int, seed: int) -> Dict[str, np.ndarray]:
    """He-style uniform initialisation from a seeded numpy generator."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, shp in param_shapes(n_codes, n_bins).items():
        if k in ("conv_b", "b1", "bc", "bb", "bp", "wl"):
            out[k] = np.zeros(shp)
        else:
            fan_in = KW if k == "conv_w" else shp[0]
            lim = np.sqrt(6.0 / fan_in)
            out[k] = rng.uniform(-lim, lim, size=shp)
    return out
