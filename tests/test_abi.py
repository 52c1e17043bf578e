"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/atlas_acq.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2005_10445_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_10445_gb300 import build
    build.build()
    return binding.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "atlas_acq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(atlas_[a-z_]+)\s*\(", src)))


def test_header_lists_expected_functions():
    assert header_functions() == sorted(binding.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_struct_sizes_match_header():
    assert ctypes.sizeof(binding.Detection) == 32
    assert ctypes.sizeof(binding.Cell) == 16
    assert ctypes.sizeof(binding.Opts) == 32


def test_strerror_and_defaults(lib):
    assert binding.strerror(0) == "ok"
    assert "invalid" in binding.strerror(binding.ATLAS_ERR_INVALID_ARG)
    o = binding.default_opts()
    assert o.threshold == 25.0 and o.fft_len == 0


def _create(lib, chips, cpc, n_codes, sps, fs, freqs, nf, opts=None):
    ctx = ctypes.c_void_p()
    chips = np.ascontiguousarray(chips, np.int8)
    cpc = np.ascontiguousarray(cpc, np.int32)
    freqs = np.ascontiguousarray(freqs, np.float64)
    st = lib.atlas_acq_create(ctypes.byref(ctx), chips.ctypes.data, cpc.ctypes.data, n_codes, sps, fs,
                              freqs.ctypes.data, nf, ctypes.byref(opts) if opts is not None else None)
    assert not ctx.value  # nothing is created on failure
    return st


def test_create_rejects_bad_arguments(lib):
    ch = np.ones(1000, np.int8)
    E = binding.ATLAS_ERR_INVALID_ARG
    assert _create(lib, ch, [1000], 0, 2, 1e6, [0.0], 1) == E          # no codes
    assert _create(lib, ch, [1000], 1, 0, 1e6, [0.0], 1) == E          # sps 0
    assert _create(lib, ch, [1000], 1, 2, 0.0, [0.0], 1) == E          # fs 0
    assert _create(lib, ch, [1000], 1, 2, 1e6, [0.0], 0) == E          # no bins
    assert _create(lib, ch, [0], 1, 2, 1e6, [0.0], 1) == E             # empty code
    assert _create(lib, ch, [1000], 1, 2, 1e6, [float("nan")], 1) == E
    bad = ch.copy()
    bad[5] = 0
    assert _create(lib, bad, [1000], 1, 2, 1e6, [0.0], 1) == E         # chip not +/-1
    o = binding.default_opts()
    o.threshold = -1.0
    assert _create(lib, ch, [1000], 1, 2, 1e6, [0.0], 1, o) == E


def test_create_rejects_unsupported_sizes(lib):
    U = binding.ATLAS_ERR_UNSUPPORTED
    ch = np.ones(40000, np.int8)
    assert _create(lib, ch, [40000], 1, 1, 1e6, [0.0], 1) == U        # N/sps = 2^17 > 2^14
    assert _create(lib, ch[:100], [100], 1, 3, 1e6, [0.0], 1) == U    # sps not a power of two
    assert _create(lib, ch[:100], [100], 1, 32, 1e6, [0.0], 1) == U   # sps above 16
    o = binding.default_opts()
    o.fft_len = 3000                                                  # not a power of two
    assert _create(lib, ch[:100], [100], 1, 2, 1e6, [0.0], 1, o) == U
    o.fft_len = 512                                                   # N/sps = 256 < 2^10
    assert _create(lib, ch[:100], [100], 1, 2, 1e6, [0.0], 1, o) == U
    o.fft_len = 128                                                   # N < L
    assert _create(lib, ch[:100], [100], 1, 2, 1e6, [0.0], 1, o) == U


def test_null_context_calls(lib):
    assert lib.atlas_acq_run(None, None, None, 0, None, 0, None) == binding.ATLAS_ERR_INVALID_ARG
    assert lib.atlas_acq_windows(None, 0, 0, None, None, None) == binding.ATLAS_ERR_INVALID_ARG
    lib.atlas_acq_destroy(None)


# --- FSK front end (include/atlas_fsk.h) ------------------------------------

def fsk_header_functions():
    src = open(os.path.join(ROOT, "include", "atlas_fsk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(atlas_[a-z_]+)\s*\(", src)))


def test_fsk_header_lists_expected_functions():
    assert fsk_header_functions() == sorted(binding.EXPORTED_FSK)


def test_fsk_every_declared_symbol_is_exported(lib):
    for name in fsk_header_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_fsk_struct_sizes_and_defaults(lib):
    assert ctypes.sizeof(binding.FskDetection) == 48
    assert ctypes.sizeof(binding.FskOpts) == 32
    o = binding.FskOpts()
    lib.atlas_fsk_default_opts(ctypes.byref(o))
    assert o.threshold == 49.0 and o.fft_len == 0 and o.windows_per_launch == 0
    assert o.exchange == 0 and o.block_log2 == 0


def _fsk_create(lib, chips, cpc, n_codes, sps, fs, taps, n_bp, opts=None, f1=5e5, f0=-5e5, f_lo=0.0):
    ctx = ctypes.c_void_p()
    chips = np.ascontiguousarray(chips, np.int8)
    cpc = np.ascontiguousarray(cpc, np.int32)
    taps = np.ascontiguousarray(taps, np.float64)
    st = lib.atlas_fsk_create(ctypes.byref(ctx), chips.ctypes.data, cpc.ctypes.data, n_codes, sps, fs, f1, f0,
                              f_lo, taps.ctypes.data, n_bp, ctypes.byref(opts) if opts is not None else None)
    assert not ctx.value
    return st


def test_fsk_create_rejects_bad_arguments(lib):
    ch = np.ones(1000, np.int8)
    taps = np.zeros((200, 2))
    taps[:, 0] = 1.0 / 200
    E = binding.ATLAS_ERR_INVALID_ARG
    assert _fsk_create(lib, ch, [1000], 0, 2, 2e6, taps, 200) == E         # no codes
    assert _fsk_create(lib, ch, [1000], 1, 0, 2e6, taps, 200) == E         # sps 0
    assert _fsk_create(lib, ch, [1000], 1, 2, 0.0, taps, 200) == E         # fs 0
    assert _fsk_create(lib, ch, [1000], 1, 2, 2e6, taps, 0) == E           # no taps
    assert _fsk_create(lib, ch, [0], 1, 2, 2e6, taps, 200) == E            # empty code
    assert _fsk_create(lib, ch, [1000], 1, 2, 2e6, taps, 200, f1=float("nan")) == E
    bad_taps = taps.copy()
    bad_taps[3, 1] = float("inf")
    assert _fsk_create(lib, ch, [1000], 1, 2, 2e6, bad_taps, 200) == E
    bad = ch.copy()
    bad[7] = 0
    assert _fsk_create(lib, bad, [1000], 1, 2, 2e6, taps, 200) == E        # chip not +/-1
    o = binding.FskOpts()
    lib.atlas_fsk_default_opts(ctypes.byref(o))
    o.threshold = -2.0
    assert _fsk_create(lib, ch, [1000], 1, 2, 2e6, taps, 200, o) == E
    lib.atlas_fsk_default_opts(ctypes.byref(o))
    o.block_log2 = 12                                                      # 13, 14 or 0 only
    assert _fsk_create(lib, ch, [1000], 1, 2, 2e6, taps, 200, o) == E


def test_fsk_create_rejects_unsupported_sizes(lib):
    U = binding.ATLAS_ERR_UNSUPPORTED
    ch = np.ones(20000, np.int8)
    taps = np.zeros((1100, 2))
    taps[:, 0] = 1e-3
    assert _fsk_create(lib, ch[:1000], [1000], 1, 2, 2e6, taps, 1100) == U     # T = 1101 taps > 1024
    assert _fsk_create(lib, ch, [20000], 1, 8, 8e6, taps, 200) == U            # N = 2^19 > 2^18
    o = binding.FskOpts()
    lib.atlas_fsk_default_opts(ctypes.byref(o))
    o.fft_len = 5000                                                          # not a power of two
    assert _fsk_create(lib, ch[:1000], [1000], 1, 2, 2e6, taps, 200, o) == U
    o.fft_len = 512                                                           # below 2^10
    assert _fsk_create(lib, ch[:100], [100], 1, 2, 2e6, taps, 20, o) == U
    o.fft_len = 2048                                                          # N <= n_c = 2000 + 200
    assert _fsk_create(lib, ch[:1000], [1000], 1, 2, 2e6, taps, 200, o) == U
    o.fft_len = 1 << 19                                                       # above 2^18
    assert _fsk_create(lib, ch[:1000], [1000], 1, 2, 2e6, taps, 200, o) == U
    o.fft_len, o.block_log2 = 1 << 16, 14                                     # 4 blocks of 2^14: no kernels
    assert _fsk_create(lib, ch[:1000], [1000], 1, 2, 2e6, taps, 200, o) == U
    o.fft_len, o.block_log2, o.exchange = 1 << 18, 0, 1                       # 2^14-point blocks: two passes only
    assert _fsk_create(lib, ch[:1000], [1000], 1, 2, 2e6, taps, 200, o) == U


def test_fsk_null_context_calls(lib):
    E = binding.ATLAS_ERR_INVALID_ARG
    assert lib.atlas_fsk_run(None, None, None, 0, None, 0, None) == E
    assert lib.atlas_fsk_windows(None, 0, 1, None, None, None, None) == E
    assert lib.atlas_fsk_demod(None, None, None, 0, 0, 0, None, None) == E
    assert lib.atlas_fsk_code_demod(None, 0, None, 0, None) == E
    lib.atlas_fsk_destroy(None)


# --- runtime (include/atlas_rt.h) -------------------------------------------

def rt_header_functions():
    src = open(os.path.join(ROOT, "include", "atlas_rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(atlas_[a-z_]+)\s*\(", src)))


def test_rt_header_and_exports(lib):
    assert rt_header_functions() == sorted(binding.EXPORTED_RT)
    for name in rt_header_functions():
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_rt_structs_and_defaults(lib):
    assert ctypes.sizeof(binding.RtOpts) == 40
    assert ctypes.sizeof(binding.RtStats) == 96
    assert binding.RT_EVENT_DTYPE.itemsize == 48
    o = binding.rt_default_opts(8e6)
    assert (o.ring_samples, o.search_block, o.search_overlap, o.track_block, o.max_misses, o.capacity) == \
        (128000000, 800000, 80000, 96000, 3, 1024)


def test_rt_rejects_bad_arguments(lib):
    E = binding.ATLAS_ERR_INVALID_ARG
    o = binding.rt_default_opts(8e6)
    per = np.ones(2)
    ctx = ctypes.c_void_p()
    assert lib.atlas_rt_create(ctypes.byref(ctx), None, per.ctypes.data, 2, ctypes.byref(o)) == E
    assert not ctx.value
    assert lib.atlas_rt_push(None, None, None, 0) == E
    n = ctypes.c_int32()
    assert lib.atlas_rt_pump(None, None, 0, None, 0, ctypes.byref(n)) == E
    assert lib.atlas_rt_get_stats(None, None) == E
    lib.atlas_rt_destroy(None)


def test_unfused_header_and_exports(lib):
    src = open(os.path.join(ROOT, "include", "atlas_unfused.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(atlas_[a-z_]+)\s*\(", src)))
    assert names == sorted(binding.EXPORTED_UNFUSED)
    for name in names:
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value
    ctx = ctypes.c_void_p()
    ch = np.ones(200, np.int8)
    cpc = np.array([100, 50], np.int32)
    f = np.zeros(1)
    assert lib.atlas_unfused_create(ctypes.byref(ctx), ch.ctypes.data, cpc.ctypes.data, 2, 2, 1e6, f.ctypes.data, 1,
                                    0, 25.0, 0) == binding.ATLAS_ERR_UNSUPPORTED   # codes of two lengths
    assert lib.atlas_unfused_run(None, None, None, 0, None, 0, None) == binding.ATLAS_ERR_INVALID_ARG
    lib.atlas_unfused_destroy(None)


def test_prop_checkpoint_null_arguments(lib):
    E = binding.ATLAS_ERR_INVALID_ARG
    assert lib.atlas_prop_save(None, b"/nonexistent") == E
    assert lib.atlas_prop_load(None, b"/nonexistent") == E


def test_fsk_tracker_null_arguments(lib):
    E = binding.ATLAS_ERR_INVALID_ARG
    t = ctypes.c_void_p()
    assert lib.atlas_fsk_tracker_create(ctypes.byref(t), None, 0, 1000, None, 1000) == E and not t.value
    n = ctypes.c_int32()
    assert lib.atlas_fsk_tracker_run(None, None, 0, 0, None, 0, ctypes.byref(n)) == E
    assert lib.atlas_fsk_tracker_kernels(None) == -1
    lib.atlas_fsk_tracker_destroy(None)
