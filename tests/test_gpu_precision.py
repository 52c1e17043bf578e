"""Reduced-precision mode: the per-code inverse transforms as FP16 / BF16
tensor-core contractions (FP32 accumulation, power-of-two scaling per stage),
against the FP64 oracle.  The error is stated per result: detections of the
injected tags must be the oracle's (code, window, lag, bin); the score and the
noise floor may move by the operand precision; the ToA comes from the FP64
refinement and must stay within 1e-3 samples (GPU only)."""
import numpy as np
import pytest

from oracle import acq
from paper_2005_10445_gb300 import synth

from test_gpu_parity import gpu_search

pytestmark = pytest.mark.gpu

# bound on |score / oracle score - 1| per precision (operand rounding 2^-11 / 2^-8)
SCORE_TOL = {1: 2e-2, 2: 1e-1}


@pytest.fixture(scope="module")
def torch_cuda(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("n_chips,sps,N", [(5000, 2, 32768), (8192, 8, 131072)])
def test_tensor_core_transforms_against_oracle(torch_cuda, precision, n_chips, sps, N):
    L = n_chips * sps
    S = 2 * N + (N - L) // 2 + 5
    wl = synth.realistic(seed=n_chips + 10 * sps, seconds=S / 4e6, n_codes=2, n_chips=n_chips, sps=sps,
                         fs_hz=4e6, n_tags=3, snr_range=(-12.0, -4.0), freqs_hz=np.array([-2500.0, 0.0, 2500.0]),
                         min_same_code_gap=2 * N, fft_len=N)
    ora, cells_o = acq.search(wl.x, wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len, keep_cells=True)
    s, dets, n, cells = gpu_search(torch_cuda, wl, cells=True, precision=precision)
    by = {d.key(): d for d in ora}
    got = {(int(d["code"]), int(d["window"]), int(d["lag"]), int(d["freq_bin"])): d for d in dets}
    # every injected tag found exactly as the oracle finds it
    for t in wl.tags:
        W, hop, _ = s.windows(t.code, wl.n_samples)
        w = min(int(t.delay) // hop, W - 1)
        key = (t.code, w, int(t.delay) - w * hop, t.bin)
        assert key in by and key in got
        o, g = by[key], got[key]
        assert abs(g["score"] / o.score - 1) < SCORE_TOL[precision]
        assert abs(g["toa"] - o.toa) <= 1e-3
    # per-cell errors, stated
    errs = []
    for (w, c), cl in cells_o.items():
        for k, cell in enumerate(cl):
            gc = cells[w, c, k]
            errs.append(abs(gc["floor"] / cell.floor - 1))
    print(f"precision {precision}: max floor error {max(errs):.2e}, detections {n} vs oracle {len(ora)}")
    assert max(errs) < SCORE_TOL[precision]
