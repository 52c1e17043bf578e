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
