"""atlas_acq_run_static: the single-code search that allocates nothing.

It is for callers that cannot call cudaMalloc when they search (a caching
allocator that owns device memory, a plug-in that must not grow the
footprint, a real-time loop that cannot take an allocation's implicit
synchronisation).  Its records must equal atlas_acq_run's for the same code,
call after call, although every call reuses the same static device array.
Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2005_10445_gb300 import binding, synth

pytestmark = pytest.mark.gpu

SCORE_RTOL = 1e-4
TOA_ATOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class _StaticBuffers:
    """Every device buffer of a static call, allocated before the call."""

    def __init__(self, torch, wl, capacity=256):
        dev = torch.device("cuda")
        self.torch, self.wl, self.capacity = torch, wl, capacity
        self.x = torch.from_numpy(wl.iq().copy()).to(dev)
        self.chips = torch.from_numpy(wl.chips[0].astype(np.int8)).to(dev)
        self.out = torch.empty(capacity * 32, dtype=torch.uint8, device=dev)
        self.cnt = torch.full((1,), -7, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()

    def call(self):
        wl, st = self.wl, self.torch.cuda.current_stream()
        binding.run_static_ptr(st.cuda_stream, self.x.data_ptr(), wl.n_samples, self.chips.data_ptr(),
                               len(wl.chips[0]), wl.sps, wl.fs_hz, wl.freqs_hz, wl.fft_len, 25.0,
                               self.out.data_ptr(), self.capacity, self.cnt.data_ptr())
        st.synchronize()

    def result(self):
        n = int(self.cnt.item())
        dets = self.out.cpu().numpy().view(binding.DETECTION_DTYPE)[: min(n, self.capacity)].copy()
        return dets, n


def _context_call(torch, wl):
    s = binding.Search(wl.chips, wl.sps, wl.fs_hz, wl.freqs_hz, fft_len=wl.fft_len)
    dets, n, _ = s.run(torch.from_numpy(wl.iq().copy()).cuda(), capacity=256)
    s.close()
    return dets, n


def _same(a, b):
    assert len(a) == len(b)
    for p, q in zip(a, b):
        assert (p["code"], p["window"], p["lag"], p["freq_bin"]) == (q["code"], q["window"], q["lag"], q["freq_bin"])
        assert p["score"] == pytest.approx(q["score"], rel=SCORE_RTOL)
        assert p["peak_power"] == pytest.approx(q["peak_power"], rel=SCORE_RTOL)
        assert abs(p["toa"] - q["toa"]) <= TOA_ATOL
    # same tables, same kernels, one window per launch: the records are identical
    assert a.tobytes() == b.tobytes()


def _full_extent():
    """The largest region the static array holds: N = M = 2^14 (sps 1) and 32
    bins, over four windows with a ragged last one."""
    return synth.realistic(seed=41, seconds=40000 / 2e6, n_codes=1, n_chips=8000, sps=1, fs_hz=2e6, n_tags=3,
                           snr_range=(-16.0, -10.0), freqs_hz=synth.freq_grid(-7750.0, 7750.0, 500.0),
                           min_same_code_gap=2 * 16384, fft_len=16384)


@pytest.mark.parametrize("maker", [
    synth.tiny,                                                     # N 16384, sps 2, 5 bins, 1 window
    lambda: synth.small(seed=31, n_codes=1, n_tags=3),              # N 8192, sps 4, several windows
    _full_extent,                                                   # M 2^14, sps 1, 32 bins
])
def test_static_matches_context_entry_twice(torch_cuda, maker):
    wl = maker()
    assert len(wl.freqs_hz) <= 32
    ref, n_ref = _context_call(torch_cuda, wl)
    assert n_ref >= 1
    buf = _StaticBuffers(torch_cuda, wl)
    for _ in range(2):  # the second call runs on the first call's leftover scratch
        buf.call()
        got, n = buf.result()
        assert n == n_ref
        _same(got, ref)


def test_static_call_takes_no_device_memory(torch_cuda):
    """After a first call on the device, a call leaves the free device memory
    unchanged (every buffer is allocated before the measurement)."""
    wl = _full_extent()
    buf = _StaticBuffers(torch_cuda, wl)
    buf.call()
    free0, _ = torch_cuda.cuda.mem_get_info()
    buf.call()
    free1, _ = torch_cuda.cuda.mem_get_info()
    assert free1 == free0
    assert buf.result()[1] >= 1


def test_static_rejects_sizes_beyond_its_limits(torch_cuda):
    wl = synth.tiny()
    with pytest.raises(binding.AtlasError) as e:     # N = 32768 > 16384
        binding.run_static_ptr(0, 1, 40000, 1, len(wl.chips[0]), wl.sps, wl.fs_hz, wl.freqs_hz, 32768, 25.0, 1,
                               16, 1)
    assert e.value.status == binding.ATLAS_ERR_UNSUPPORTED
    with pytest.raises(binding.AtlasError) as e:     # 40 bins > 32
        binding.run_static_ptr(0, 1, 40000, 1, len(wl.chips[0]), wl.sps, wl.fs_hz, np.zeros(40), 16384, 25.0, 1,
                               16, 1)
    assert e.value.status == binding.ATLAS_ERR_UNSUPPORTED
    with pytest.raises(binding.AtlasError) as e:     # a stream longer than atlas_acq_run accepts
        binding.run_static_ptr(0, 1, 8 * (2 ** 31 - 1) + 1, 1, 16383, 1, wl.fs_hz, wl.freqs_hz, 16384, 25.0, 1,
                               16, 1)
    assert e.value.status == binding.ATLAS_ERR_INVALID_ARG
