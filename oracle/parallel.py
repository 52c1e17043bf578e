"""Runs the FP64 oracle over many (window, code) pairs on all host cores.

TEST INFRASTRUCTURE ONLY.  Only the tests and the CPU legs of the benchmark
may import this module; the product path never calls it.

It adds no arithmetic of its own: the pairs are split into chunks and each
worker process runs ``acq.search`` on its chunk, exactly as a single process
would (the search of a pair depends only on that pair).  The detections come
back ordered by (window, code), the order ``acq.search`` uses.

Workers are started with the ``spawn`` method, never ``fork``: a process
forked after the parent has used a GPU can hang.  The stream is handed to the
workers once, through shared memory.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import acq

_W: dict = {}


def _init(shm_name: str, n: int, dtype: str, chips_list, sps, fs_hz, freqs_hz, fft_len, threshold):
    # one numpy thread per worker: the pool already uses every core
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    shm = shared_memory.SharedMemory(name=shm_name)
    _W.update(shm=shm, x=np.ndarray((n,), dtype=np.dtype(dtype), buffer=shm.buf), chips=chips_list, sps=sps,
              fs=fs_hz, freqs=freqs_hz, fft_len=fft_len, threshold=threshold)


def _run(pairs):
    return acq.search(_W["x"], _W["chips"], _W["sps"], _W["fs"], _W["freqs"], _W["fft_len"], _W["threshold"],
                      pairs=pairs, keep_cells=True)


def _noop(_):
    return None


def all_pairs(n_samples: int, chips_list: Sequence[np.ndarray], sps: int, fft_len: int = 0) -> List[Tuple[int, int]]:
    """Every (window, code) pair of a stream, in (window, code) order."""
    plans = []
    for ch in chips_list:
        L = len(ch) * sps
        N = fft_len if fft_len else acq.default_fft_len(L)
        plans.append(acq.window_plan(n_samples, N, L)[0])
    return [(w, c) for w in range(max(plans)) for c in range(len(chips_list)) if w < plans[c]]


class Pool:
    """Worker processes holding one stream and one search configuration;
    ``search(pairs)`` runs ``acq.search`` over the pairs on all of them."""

    def __init__(self, x: np.ndarray, chips_list: Sequence[np.ndarray], sps: int, fs_hz: float,
                 freqs_hz: Sequence[float], fft_len: int = 0, threshold: float = 25.0,
                 processes: Optional[int] = None):
        x = np.ascontiguousarray(x)
        self.x_len = x.shape[0]
        self.chips, self.sps, self.fft_len = list(chips_list), sps, fft_len
        self.processes = max(1, processes or os.cpu_count() or 1)
        self._shm = shared_memory.SharedMemory(create=True, size=max(1, x.nbytes))
        np.ndarray(x.shape, dtype=x.dtype, buffer=self._shm.buf)[:] = x
        args = (self._shm.name, x.shape[0], x.dtype.str, [np.asarray(c) for c in chips_list], sps, float(fs_hz),
                [float(f) for f in freqs_hz], fft_len, threshold)
        self._pool = mp.get_context("spawn").Pool(self.processes, initializer=_init, initargs=args)
        self._pool.map(_noop, range(self.processes))  # every worker started and initialised

    def search(self, pairs: Optional[Sequence[Tuple[int, int]]] = None, chunk: int = 0):
        """(detections ordered by (window, code), {(w, c): [Cell] * K})."""
        if pairs is None:
            pairs = all_pairs(self.x_len, self.chips, self.sps, self.fft_len)
        pairs = sorted(pairs)
        if chunk <= 0:
            chunk = max(1, -(-len(pairs) // (self.processes * 4)))
        results = self._pool.map(_run, [pairs[i:i + chunk] for i in range(0, len(pairs), chunk)])
        dets: list = []
        cells: Dict[Tuple[int, int], list] = {}
        for d, c in results:
            dets.extend(d)
            cells.update(c)
        dets.sort(key=lambda d: (d.window, d.code))
        return dets, cells

    def close(self) -> None:
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
            self._shm.close()
            self._shm.unlink()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def search(x: np.ndarray, chips_list: Sequence[np.ndarray], sps: int, fs_hz: float, freqs_hz: Sequence[float],
           fft_len: int = 0, threshold: float = 25.0, pairs: Optional[Sequence[Tuple[int, int]]] = None,
           processes: Optional[int] = None, chunk: int = 0):
    """``acq.search`` over ``pairs`` (every pair when None) on ``processes``
    worker processes (all cores when None).  Returns (detections ordered by
    (window, code), {(w, c): [Cell] * K}, processes used)."""
    n_pairs = len(pairs) if pairs is not None else len(all_pairs(len(x), chips_list, sps, fft_len))
    procs = max(1, min(processes or os.cpu_count() or 1, n_pairs))
    with Pool(x, chips_list, sps, fs_hz, freqs_hz, fft_len, threshold, procs) as p:
        dets, cells = p.search(pairs, chunk)
    return dets, cells, procs
