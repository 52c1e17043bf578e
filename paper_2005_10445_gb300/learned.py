"""Training and evaluation loop of the learned (code, bin) proposal.

Host-side orchestration only: every step (exhaustive labelling search,
features, forward, backward, Adam, candidate selection, proposal search) runs
in the library's CUDA kernels through the C ABI.

Labels come from the exhaustive search itself: for each window, the
detection with the largest score gives the (code, bin) label; windows with no
detection are labelled empty.  Recall is the fraction of the exhaustive
search's detections that the proposal search reproduces exactly (same code,
window, lag and bin).
"""
from __future__ import annotations

import time
from typing import Dict, List, Tuple

import numpy as np

from . import binding, synth


def exhaustive(search: binding.Search, x, n_samples: int, capacity: int, torch):
    out = torch.zeros(capacity * 32, dtype=torch.uint8, device=x.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=x.device)
    st = torch.cuda.current_stream(x.device)
    torch.cuda.synchronize(x.device)
    t0 = time.perf_counter()
    search.run_ptr(st.cuda_stream, x.data_ptr(), n_samples, out.data_ptr(), capacity, cnt.data_ptr())
    st.synchronize()
    dt = time.perf_counter() - t0
    n = int(cnt.item())
    dets = out.cpu().numpy().view(binding.DETECTION_DTYPE)[: min(n, capacity)].copy()
    return dets, n, dt


def labels_from(dets, n_windows: int) -> Tuple[np.ndarray, np.ndarray]:
    code = np.full(n_windows, -1, np.int32)
    bin_ = np.full(n_windows, -1, np.int32)
    best = np.full(n_windows, -np.inf)
    for d in dets:
        w = int(d["window"])
        if d["score"] > best[w]:
            best[w] = d["score"]
            code[w] = int(d["code"])
            bin_[w] = int(d["freq_bin"])
    return code, bin_


def features(prop: binding.Proposal, x, n_samples: int, n_windows: int, hop: int, N: int, torch):
    """Feature rows [n_windows][prop.feature_len]: the spectrum, then the
    carrier-line values of the grid set on `prop` (zeros without one)."""
    feat = torch.empty(n_windows * prop.feature_len, dtype=torch.float32, device=x.device)
    st = torch.cuda.current_stream(x.device)
    prop.features(st.cuda_stream, x.data_ptr(), n_samples, 0, hop, N, n_windows, feat.data_ptr())
    return feat


def train(prop: binding.Proposal, feat, code: np.ndarray, bin_: np.ndarray, torch, epochs: int = 6,
          batch: int = 256, lr: float = 1e-3, seed: int = 0) -> List[float]:
    dev = feat.device
    n = code.shape[0]
    d_code = torch.from_numpy(code).to(dev)
    d_bin = torch.from_numpy(bin_).to(dev)
    f2 = feat.view(n, prop.feature_len)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).to(dev)
        tot, m = 0.0, 0
        for i0 in range(0, n - batch + 1, batch):
            idx = order[i0:i0 + batch]
            fb = f2.index_select(0, idx).contiguous()
            cb = d_code.index_select(0, idx).contiguous()
            bb = d_bin.index_select(0, idx).contiguous()
            prop.loss_grad(st.cuda_stream, fb.data_ptr(), cb.data_ptr(), bb.data_ptr(), batch, loss.data_ptr())
            prop.adam(st.cuda_stream, lr)
            tot += float(loss.item())
            m += 1
        hist.append(tot / max(m, 1))
    return hist


def evaluate(search: binding.Search, prop: binding.Proposal, x, n_samples: int, exh_dets, exh_time: float,
             topk: int, tau: float, capacity: int, torch, bins: bool = False) -> Dict[str, float]:
    """Recall, speedup and ToA difference of the proposal search against the
    exhaustive one.  bins=False: the top-k (code, bin) pairs of a confident
    window; bins=True: every code in its top-k bins."""
    dev = x.device
    out = torch.zeros(capacity * 32, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)
    run = binding.run_proposed_bins if bins else binding.run_proposed
    run(search, prop, st.cuda_stream, x.data_ptr(), n_samples, topk, tau, out.data_ptr(), capacity,
        cnt.data_ptr())  # warm the workspaces
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    nfb = run(search, prop, st.cuda_stream, x.data_ptr(), n_samples, topk, tau, out.data_ptr(), capacity,
              cnt.data_ptr())
    dt = time.perf_counter() - t0
    n = int(cnt.item())
    got = out.cpu().numpy().view(binding.DETECTION_DTYPE)[: min(n, capacity)]
    key = lambda d: (int(d["code"]), int(d["window"]), int(d["lag"]), int(d["freq_bin"]))
    exh = {key(d) for d in exh_dets}
    prp = {key(d) for d in got}
    hit = len(exh & prp)
    toa = {key(d): float(d["toa"]) for d in exh_dets}
    toa_err = max([abs(float(d["toa"]) - toa[key(d)]) for d in got if key(d) in toa] or [0.0])
    return {"mode": "bins" if bins else "pairs", "tau_fb": tau, "topk": topk, "recall": hit / max(len(exh), 1),
            "exhaustive_detections": len(exh),
            "proposal_detections": len(prp), "extra_detections": len(prp - exh), "fallback_windows": nfb,
            "time_s": dt, "speedup": exh_time / dt, "max_toa_diff_samples": toa_err}
