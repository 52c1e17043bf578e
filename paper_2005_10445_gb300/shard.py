"""Sharding one stream's search over ranks (one GPU per rank).

The search's units are independent: window w of a code group depends only on
samples [w*hop, w*hop + N) (Section 2.1: each block holds whole
transmissions).  A stream is split by windows: rank r owns the contiguous
window range [w_begin, w_end) of the full window plan and searches the sample
range those windows read, plus halos (one window in front, zero padding
behind; see local_plan), so no data-path exchange is needed.  The only
collective is one gather of the small detection lists; windows and ToAs are
shifted back to stream coordinates and the lists concatenated in rank order,
which keeps the (window, code) order of a single search.  The result equals
the single search's detection for detection.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def window_plan(n_samples: int, N: int, L: int) -> Tuple[int, int]:
    hop = N - L
    W = max(1, -(-(n_samples - N) // hop) + 1)
    return W, hop


def split_windows(W: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous, balanced window ranges [begin, end) per rank (empty ranges
    when there are more ranks than windows)."""
    out = []
    for r in range(world):
        b = (W * r) // world
        e = (W * (r + 1)) // world
        out.append((b, e))
    return out


def local_plan(n_samples: int, N: int, L: int, w_begin: int, w_end: int) -> Tuple[int, int, int, int]:
    """(first_window, n_samples_local, keep_begin, keep_end) for a rank that
    owns global windows [w_begin, w_end).

    The local stream starts at window first_window = max(w_begin - 1, 0): one
    extra window in front, so that the refinement of a peak at the shard's
    first lag can read the sample before it, as the single search does.  A
    shard that does not reach the stream's end is extended by zero padding to
    one window past its range, so that its last owned window keeps the whole
    hop of valid lags (an interior window, as in the single search).  Local
    windows [keep_begin, keep_end) are the owned ones."""
    W, hop = window_plan(n_samples, N, L)
    lo = max(w_begin - 1, 0)
    if w_end >= W:
        n_local = n_samples - lo * hop
    else:
        n_local = (w_end - lo - 1) * hop + N + hop
    return lo, n_local, w_begin - lo, w_end - lo


def local_stream(x: np.ndarray, N: int, L: int, w_begin: int, w_end: int) -> np.ndarray:
    """The rank's samples (zero beyond the stream, as the search reads them)."""
    S = x.shape[0]
    W, hop = window_plan(S, N, L)
    lo, n_local, _, _ = local_plan(S, N, L, w_begin, w_end)
    out = np.zeros((n_local,) + x.shape[1:], dtype=x.dtype)
    s0 = lo * hop
    s1 = min(S, s0 + n_local)
    out[: s1 - s0] = x[s0:s1]
    return out


def to_global(dets: np.ndarray, first_window: int, hop: int, keep_begin: int, keep_end: int) -> np.ndarray:
    """Keep a rank's owned windows and shift its detections (structured array
    with window and toa fields) to stream coordinates."""
    m = (dets["window"] >= keep_begin) & (dets["window"] < keep_end)
    d = dets[m].copy()
    d["window"] += first_window
    d["toa"] += first_window * hop
    return d


def gather(dets: np.ndarray, group=None) -> np.ndarray:
    """All ranks' detection lists, concatenated in rank order (one
    all_gather_object of the small lists; works with gloo or NCCL)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts: List = [None] * world
    dist.all_gather_object(parts, dets, group=group)
    return np.concatenate(parts) if parts else dets
