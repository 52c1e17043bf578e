"""Thin ctypes binding over ``libatlas_acq.so`` (include/atlas_acq.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  Device buffers are passed as raw pointers (``tensor.data_ptr()``
of torch CUDA tensors) and streams as ``torch.cuda.Stream.cuda_stream``.
Loading fails loudly when the library has not been built; there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libatlas_acq.so")

ATLAS_OK = 0
ATLAS_ERR_INVALID_ARG = -1
ATLAS_ERR_CUDA = -2
ATLAS_ERR_NO_MEMORY = -3
ATLAS_ERR_UNSUPPORTED = -4
ATLAS_ERR_TIMEOUT = -5
ATLAS_ERR_DEVICE = -6

# Every symbol include/atlas_acq.h declares.
EXPORTED = [
    "atlas_acq_default_opts", "atlas_acq_create", "atlas_acq_windows", "atlas_acq_run",
    "atlas_acq_run_cells", "atlas_acq_run_host", "atlas_acq_last_device_status",
    "atlas_acq_last_error", "atlas_acq_destroy", "atlas_acq_strerror", "atlas_acq_profile_begin",
    "atlas_acq_profile_end", "atlas_acq_run_static", "atlas_acq_autotune", "atlas_acq_tuning",
    "atlas_acq_batch_create", "atlas_acq_batch_run", "atlas_acq_batch_kernels", "atlas_acq_batch_destroy",
    "atlas_prop_create", "atlas_prop_num_params", "atlas_prop_get_params", "atlas_prop_set_params",
    "atlas_prop_save", "atlas_prop_load",
    "atlas_prop_features", "atlas_prop_loss_grad", "atlas_prop_adam", "atlas_prop_logits", "atlas_prop_candidates",
    "atlas_acq_run_proposed", "atlas_prop_last_error", "atlas_prop_destroy",
    "atlas_prop_set_grid", "atlas_prop_feature_len", "atlas_prop_bin_candidates", "atlas_acq_run_proposed_bins",
]
# Every symbol include/atlas_unfused.h declares (the comparison pipeline).
EXPORTED_UNFUSED = ["atlas_unfused_create", "atlas_unfused_run", "atlas_unfused_last_error", "atlas_unfused_destroy"]
# Every symbol include/atlas_rt.h declares.
EXPORTED_RT = [
    "atlas_rt_default_opts", "atlas_rt_create", "atlas_rt_push", "atlas_rt_pump", "atlas_rt_get_stats",
    "atlas_rt_last_error", "atlas_rt_destroy",
]
# Every symbol include/atlas_fsk.h declares.
EXPORTED_FSK = [
    "atlas_fsk_default_opts", "atlas_fsk_create", "atlas_fsk_windows", "atlas_fsk_run", "atlas_fsk_run_codes",
    "atlas_fsk_run_host",
    "atlas_fsk_demod", "atlas_fsk_code_demod", "atlas_fsk_profile_begin", "atlas_fsk_profile_end",
    "atlas_fsk_tracker_create", "atlas_fsk_tracker_run", "atlas_fsk_tracker_kernels", "atlas_fsk_tracker_destroy",
    "atlas_fsk_last_error", "atlas_fsk_destroy",
]


class Detection(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("window", ctypes.c_int32), ("lag", ctypes.c_int32),
                ("freq_bin", ctypes.c_int32), ("score", ctypes.c_float), ("peak_power", ctypes.c_float),
                ("toa", ctypes.c_double)]


class Cell(ctypes.Structure):
    _fields_ = [("p_max", ctypes.c_float), ("floor", ctypes.c_float), ("lag", ctypes.c_int32),
                ("valid", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_float), ("fft_len", ctypes.c_int32),
                ("windows_per_launch", ctypes.c_int32), ("tile_log2", ctypes.c_int32),
                ("split", ctypes.c_int32), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("corr_launches", ctypes.c_int64), ("corr_ms", ctypes.c_double),
                ("corr_units", ctypes.c_int64), ("timed_launches", ctypes.c_int64)]


class FskDetection(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("window", ctypes.c_int32), ("lag", ctypes.c_int32),
                ("score", ctypes.c_float), ("toa", ctypes.c_double), ("w_c", ctypes.c_double),
                ("q", ctypes.c_double), ("p_c", ctypes.c_double)]


class FskOpts(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_float), ("fft_len", ctypes.c_int32),
                ("windows_per_launch", ctypes.c_int32), ("exchange", ctypes.c_int32),
                ("block_log2", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class FskProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("corr_launches", ctypes.c_int64), ("corr_units", ctypes.c_int64),
                ("corr_timed", ctypes.c_int64), ("corr_ms", ctypes.c_double), ("demod_launches", ctypes.c_int64),
                ("demod_samples", ctypes.c_int64), ("demod_timed", ctypes.c_int64), ("demod_ms", ctypes.c_double)]


class RtOpts(ctypes.Structure):
    _fields_ = [("ring_samples", ctypes.c_int64), ("search_block", ctypes.c_int32),
                ("search_overlap", ctypes.c_int32), ("track_block", ctypes.c_int32), ("max_misses", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class RtStats(ctypes.Structure):
    _fields_ = [("pushed", ctypes.c_int64), ("search_tasks", ctypes.c_int64), ("track_tasks", ctypes.c_int64),
                ("searched_samples", ctypes.c_int64), ("search_units", ctypes.c_int64),
                ("track_units", ctypes.c_int64), ("events", ctypes.c_int64), ("track_kernels", ctypes.c_int64),
                ("search_ms", ctypes.c_double),
                ("track_ms", ctypes.c_double), ("searching", ctypes.c_int32), ("tracking", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


RT_SEARCH_DETECTION, RT_TRACK_DETECTION, RT_TRACK_MISS, RT_TRACK_LOST, RT_SEARCH_SKIPPED = range(5)
RT_EVENT_DTYPE = np.dtype([("kind", "<i4"), ("code", "<i4"), ("task_start", "<i8"), ("toa", "<f8"),
                           ("score", "<f4"), ("misses", "<i4"), ("w_c", "<f8"), ("q", "<f8")])
assert RT_EVENT_DTYPE.itemsize == 48

FSK_DETECTION_DTYPE = np.dtype([("code", "<i4"), ("window", "<i4"), ("lag", "<i4"), ("score", "<f4"),
                                ("toa", "<f8"), ("w_c", "<f8"), ("q", "<f8"), ("p_c", "<f8")])
assert FSK_DETECTION_DTYPE.itemsize == ctypes.sizeof(FskDetection) == 48

DETECTION_DTYPE = np.dtype([("code", "<i4"), ("window", "<i4"), ("lag", "<i4"), ("freq_bin", "<i4"),
                            ("score", "<f4"), ("peak_power", "<f4"), ("toa", "<f8")])
CELL_DTYPE = np.dtype([("p_max", "<f4"), ("floor", "<f4"), ("lag", "<i4"), ("valid", "<i4")])
assert DETECTION_DTYPE.itemsize == ctypes.sizeof(Detection) == 32
assert CELL_DTYPE.itemsize == ctypes.sizeof(Cell) == 16

_lib = None


class AtlasError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"atlas_acq error {status}: {msg}")
        self.status = status


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the shared library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.atlas_acq_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.atlas_acq_default_opts.restype = None
    lib.atlas_acq_create.argtypes = [ctypes.POINTER(vp), vp, vp, i32, i32, f64, vp, i32, ctypes.POINTER(Opts)]
    lib.atlas_acq_create.restype = ctypes.c_int
    lib.atlas_acq_windows.argtypes = [vp, i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.atlas_acq_windows.restype = ctypes.c_int
    lib.atlas_acq_run.argtypes = [vp, vp, vp, i64, vp, i32, vp]
    lib.atlas_acq_run.restype = ctypes.c_int
    lib.atlas_acq_run_cells.argtypes = [vp, vp, vp, i64, vp, vp, i32, vp]
    lib.atlas_acq_run_cells.restype = ctypes.c_int
    lib.atlas_acq_run_host.argtypes = [vp, vp, vp, i64, vp, i32, vp]
    lib.atlas_acq_run_host.restype = ctypes.c_int
    lib.atlas_acq_last_device_status.argtypes = [vp]
    lib.atlas_acq_last_device_status.restype = ctypes.c_int
    lib.atlas_acq_last_error.argtypes = [vp]
    lib.atlas_acq_last_error.restype = ctypes.c_char_p
    lib.atlas_acq_destroy.argtypes = [vp]
    lib.atlas_acq_destroy.restype = None
    lib.atlas_acq_profile_begin.argtypes = [vp, i32]
    lib.atlas_acq_profile_begin.restype = ctypes.c_int
    lib.atlas_acq_profile_end.argtypes = [vp, ctypes.POINTER(Profile)]
    lib.atlas_acq_profile_end.restype = ctypes.c_int
    lib.atlas_acq_run_static.argtypes = [vp, vp, i64, vp, i32, i32, f64, vp, i32, i32, ctypes.c_float, vp, i32, vp]
    lib.atlas_acq_run_static.restype = ctypes.c_int
    lib.atlas_acq_autotune.argtypes = [vp, vp, vp, i64, ctypes.c_char_p]
    lib.atlas_acq_autotune.restype = ctypes.c_int
    lib.atlas_acq_tuning.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.atlas_acq_tuning.restype = ctypes.c_int
    lib.atlas_acq_batch_create.argtypes = [ctypes.POINTER(vp), vp, i32, vp, vp, vp, i32, vp]
    lib.atlas_acq_batch_create.restype = ctypes.c_int
    lib.atlas_acq_batch_run.argtypes = [vp, vp]
    lib.atlas_acq_batch_run.restype = ctypes.c_int
    lib.atlas_acq_batch_kernels.argtypes = [vp]
    lib.atlas_acq_batch_kernels.restype = i64
    lib.atlas_acq_batch_destroy.argtypes = [vp]
    lib.atlas_acq_batch_destroy.restype = None
    u64, f32 = ctypes.c_uint64, ctypes.c_float
    lib.atlas_prop_create.argtypes = [ctypes.POINTER(vp), i32, i32, u64]
    lib.atlas_prop_create.restype = ctypes.c_int
    lib.atlas_prop_num_params.argtypes = [vp]
    lib.atlas_prop_num_params.restype = i64
    lib.atlas_prop_get_params.argtypes = [vp, vp]
    lib.atlas_prop_get_params.restype = ctypes.c_int
    lib.atlas_prop_set_params.argtypes = [vp, vp]
    lib.atlas_prop_set_params.restype = ctypes.c_int
    lib.atlas_prop_save.argtypes = [vp, ctypes.c_char_p]
    lib.atlas_prop_save.restype = ctypes.c_int
    lib.atlas_prop_load.argtypes = [vp, ctypes.c_char_p]
    lib.atlas_prop_load.restype = ctypes.c_int
    lib.atlas_prop_features.argtypes = [vp, vp, vp, i64, i64, i64, i32, i32, vp]
    lib.atlas_prop_features.restype = ctypes.c_int
    lib.atlas_prop_loss_grad.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp]
    lib.atlas_prop_loss_grad.restype = ctypes.c_int
    lib.atlas_prop_adam.argtypes = [vp, vp, vp, f32]
    lib.atlas_prop_adam.restype = ctypes.c_int
    lib.atlas_prop_logits.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp]
    lib.atlas_prop_logits.restype = ctypes.c_int
    lib.atlas_prop_candidates.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    lib.atlas_prop_candidates.restype = ctypes.c_int
    lib.atlas_acq_run_proposed.argtypes = [vp, vp, vp, vp, i64, i32, f32, vp, i32, vp, ctypes.POINTER(i32)]
    lib.atlas_acq_run_proposed.restype = ctypes.c_int
    lib.atlas_acq_run_proposed_bins.argtypes = [vp, vp, vp, vp, i64, i32, f32, vp, i32, vp, ctypes.POINTER(i32)]
    lib.atlas_acq_run_proposed_bins.restype = ctypes.c_int
    lib.atlas_prop_set_grid.argtypes = [vp, f64, vp, i32]
    lib.atlas_prop_set_grid.restype = ctypes.c_int
    lib.atlas_prop_feature_len.argtypes = [vp]
    lib.atlas_prop_feature_len.restype = i32
    lib.atlas_prop_bin_candidates.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    lib.atlas_prop_bin_candidates.restype = ctypes.c_int
    lib.atlas_prop_last_error.argtypes = [vp]
    lib.atlas_prop_last_error.restype = ctypes.c_char_p
    lib.atlas_prop_destroy.argtypes = [vp]
    lib.atlas_prop_destroy.restype = None
    lib.atlas_fsk_default_opts.argtypes = [ctypes.POINTER(FskOpts)]
    lib.atlas_fsk_default_opts.restype = None
    lib.atlas_fsk_create.argtypes = [ctypes.POINTER(vp), vp, vp, i32, i32, f64, f64, f64, f64, vp, i32,
                                     ctypes.POINTER(FskOpts)]
    lib.atlas_fsk_create.restype = ctypes.c_int
    lib.atlas_fsk_windows.argtypes = [vp, i32, i64] + [ctypes.POINTER(i32)] * 4
    lib.atlas_fsk_windows.restype = ctypes.c_int
    lib.atlas_fsk_run.argtypes = [vp, vp, vp, i64, vp, i32, vp]
    lib.atlas_fsk_run.restype = ctypes.c_int
    lib.atlas_fsk_run_codes.argtypes = [vp, vp, vp, i64, i64, vp, i32, vp, i32, vp]
    lib.atlas_fsk_run_codes.restype = ctypes.c_int
    lib.atlas_fsk_run_host.argtypes = [vp, vp, vp, i64, vp, i32, vp]
    lib.atlas_fsk_run_host.restype = ctypes.c_int
    lib.atlas_fsk_demod.argtypes = [vp, vp, vp, i64, i64, i64, vp, vp]
    lib.atlas_fsk_demod.restype = ctypes.c_int
    lib.atlas_fsk_code_demod.argtypes = [vp, i32, vp, i32, ctypes.POINTER(i32)]
    lib.atlas_fsk_code_demod.restype = ctypes.c_int
    lib.atlas_fsk_profile_begin.argtypes = [vp, i32]
    lib.atlas_fsk_profile_begin.restype = ctypes.c_int
    lib.atlas_fsk_profile_end.argtypes = [vp, ctypes.POINTER(FskProfile)]
    lib.atlas_fsk_profile_end.restype = ctypes.c_int
    lib.atlas_fsk_tracker_create.argtypes = [ctypes.POINTER(vp), vp, i32, i64, vp, i64]
    lib.atlas_fsk_tracker_create.restype = ctypes.c_int
    lib.atlas_fsk_tracker_run.argtypes = [vp, vp, i32, i64, vp, i32, ctypes.POINTER(i32)]
    lib.atlas_fsk_tracker_run.restype = ctypes.c_int
    lib.atlas_fsk_tracker_kernels.argtypes = [vp]
    lib.atlas_fsk_tracker_kernels.restype = i32
    lib.atlas_fsk_tracker_destroy.argtypes = [vp]
    lib.atlas_fsk_tracker_destroy.restype = None
    lib.atlas_fsk_last_error.argtypes = [vp]
    lib.atlas_fsk_last_error.restype = ctypes.c_char_p
    lib.atlas_fsk_destroy.argtypes = [vp]
    lib.atlas_fsk_destroy.restype = None
    lib.atlas_unfused_create.argtypes = [ctypes.POINTER(vp), vp, vp, i32, i32, f64, vp, i32, i32, ctypes.c_float, i32]
    lib.atlas_unfused_create.restype = ctypes.c_int
    lib.atlas_unfused_run.argtypes = [vp, vp, vp, i64, vp, i32, vp]
    lib.atlas_unfused_run.restype = ctypes.c_int
    lib.atlas_unfused_last_error.argtypes = [vp]
    lib.atlas_unfused_last_error.restype = ctypes.c_char_p
    lib.atlas_unfused_destroy.argtypes = [vp]
    lib.atlas_unfused_destroy.restype = None
    lib.atlas_rt_default_opts.argtypes = [ctypes.POINTER(RtOpts), f64]
    lib.atlas_rt_default_opts.restype = None
    lib.atlas_rt_create.argtypes = [ctypes.POINTER(vp), vp, vp, i32, ctypes.POINTER(RtOpts)]
    lib.atlas_rt_create.restype = ctypes.c_int
    lib.atlas_rt_push.argtypes = [vp, vp, vp, i64]
    lib.atlas_rt_push.restype = ctypes.c_int
    lib.atlas_rt_pump.argtypes = [vp, vp, i32, vp, i32, ctypes.POINTER(i32)]
    lib.atlas_rt_pump.restype = ctypes.c_int
    lib.atlas_rt_get_stats.argtypes = [vp, ctypes.POINTER(RtStats)]
    lib.atlas_rt_get_stats.restype = ctypes.c_int
    lib.atlas_rt_last_error.argtypes = [vp]
    lib.atlas_rt_last_error.restype = ctypes.c_char_p
    lib.atlas_rt_destroy.argtypes = [vp]
    lib.atlas_rt_destroy.restype = None
    lib.atlas_acq_strerror.argtypes = [ctypes.c_int]
    lib.atlas_acq_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load().atlas_acq_strerror(status).decode()


def _check(status: int, ctx=None) -> None:
    if status != ATLAS_OK:
        msg = strerror(status)
        if ctx is not None and status == ATLAS_ERR_CUDA:
            msg += ": " + load().atlas_acq_last_error(ctx).decode()
        raise AtlasError(status, msg)


def default_opts() -> Opts:
    o = Opts()
    load().atlas_acq_default_opts(ctypes.byref(o))
    return o


class Search:
    """A search context (atlas_acq_create / atlas_acq_destroy)."""

    def __init__(self, chips: Sequence[np.ndarray], samples_per_chip: int, fs_hz: float,
                 freq_offsets_hz: Sequence[float], threshold: float = 25.0, fft_len: int = 0,
                 windows_per_launch: int = 0, tile_log2: int = 0, split: int = 0, precision: int = 0):
        lib = load()
        self._lib = lib
        self.ctx = ctypes.c_void_p()
        cat = np.ascontiguousarray(np.concatenate([np.asarray(c, np.int8) for c in chips]))
        cpc = np.ascontiguousarray(np.array([len(c) for c in chips], np.int32))
        fr = np.ascontiguousarray(np.asarray(freq_offsets_hz, np.float64))
        o = default_opts()
        o.threshold = threshold
        o.fft_len = fft_len
        o.windows_per_launch = windows_per_launch
        o.tile_log2 = tile_log2
        o.split = split
        o.precision = precision
        self.n_codes = len(chips)
        self.n_freq = len(fr)
        st = lib.atlas_acq_create(ctypes.byref(self.ctx), cat.ctypes.data, cpc.ctypes.data, len(chips),
                                  samples_per_chip, float(fs_hz), fr.ctypes.data, len(fr), ctypes.byref(o))
        if st != ATLAS_OK:
            self.ctx = None
        _check(st)

    def close(self) -> None:
        if self.ctx:
            self._lib.atlas_acq_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def windows(self, code: int, n_samples: int):
        W, hop, N = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.atlas_acq_windows(self.ctx, code, n_samples, ctypes.byref(W), ctypes.byref(hop),
                                           ctypes.byref(N)))
        return W.value, hop.value, N.value

    def max_windows(self, n_samples: int) -> int:
        return max(self.windows(c, n_samples)[0] for c in range(self.n_codes))

    # raw pointer forms (device memory) ------------------------------------
    def run_ptr(self, stream: int, d_iq: int, n_samples: int, d_out: int, capacity: int, d_count: int) -> None:
        _check(self._lib.atlas_acq_run(self.ctx, stream, d_iq, n_samples, d_out, capacity, d_count), self.ctx)

    def run_cells_ptr(self, stream: int, d_iq: int, n_samples: int, d_cells: int, d_out: int, capacity: int,
                      d_count: int) -> None:
        _check(self._lib.atlas_acq_run_cells(self.ctx, stream, d_iq, n_samples, d_cells, d_out, capacity,
                                             d_count), self.ctx)

    def run_host_ptr(self, stream: int, h_iq: int, n_samples: int, h_out: int, capacity: int,
                     h_count: int) -> None:
        _check(self._lib.atlas_acq_run_host(self.ctx, stream, h_iq, n_samples, h_out, capacity, h_count),
               self.ctx)

    def profile_begin(self, max_timed: int = 65536) -> None:
        _check(self._lib.atlas_acq_profile_begin(self.ctx, max_timed), self.ctx)

    def profile_end(self) -> dict:
        p = Profile()
        _check(self._lib.atlas_acq_profile_end(self.ctx, ctypes.byref(p)), self.ctx)
        return {f: getattr(p, f) for f, _ in Profile._fields_}

    def autotune(self, stream: int, d_iq: int, n_samples: int, cache_path: Optional[str] = None) -> None:
        _check(self._lib.atlas_acq_autotune(self.ctx, stream, d_iq, n_samples,
                                            cache_path.encode() if cache_path else None), self.ctx)

    def tuning(self, code: int = 0):
        """(tile_log2, windows_per_launch, split) of the code's group."""
        t, w, sp = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.atlas_acq_tuning(self.ctx, code, ctypes.byref(t), ctypes.byref(w), ctypes.byref(sp)))
        return t.value, w.value, sp.value

    def device_status(self) -> int:
        return int(self._lib.atlas_acq_last_device_status(self.ctx))

    # torch conveniences ---------------------------------------------------
    def run(self, x_iq, capacity: int = 4096, stream=None, cells: bool = False):
        """x_iq: torch CUDA float32 tensor [S, 2] (or complex64 [S]).  Returns
        (detections as a numpy structured array, count, cells or None)."""
        import torch
        if x_iq.dtype == torch.complex64:
            x_iq = torch.view_as_real(x_iq)
        assert x_iq.is_cuda and x_iq.dtype == torch.float32 and x_iq.is_contiguous()
        S = x_iq.shape[0]
        dev = x_iq.device
        out = torch.empty(max(capacity, 1) * 32, dtype=torch.uint8, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        cell_buf = None
        if cells:
            nw = self.max_windows(S)
            cell_buf = torch.empty(nw * self.n_codes * self.n_freq * 16, dtype=torch.uint8, device=dev)
            self.run_cells_ptr(st.cuda_stream, x_iq.data_ptr(), S, cell_buf.data_ptr(), out.data_ptr(), capacity,
                               cnt.data_ptr())
        else:
            self.run_ptr(st.cuda_stream, x_iq.data_ptr(), S, out.data_ptr(), capacity, cnt.data_ptr())
        st.synchronize()
        n = int(cnt.item())
        dets = out.cpu().numpy().view(DETECTION_DTYPE)[: min(n, capacity)].copy()
        cell_np = None
        if cells:
            cell_np = cell_buf.cpu().numpy().view(CELL_DTYPE).reshape(nw, self.n_codes, self.n_freq).copy()
        return dets, n, cell_np

    def run_host(self, x_iq: np.ndarray, capacity: int = 4096, stream: int = 0):
        """Host numpy [S, 2] float32 (or complex64 [S]) in, host detections out."""
        if x_iq.dtype == np.complex64:
            x_iq = x_iq.view(np.float32).reshape(-1, 2)
        x_iq = np.ascontiguousarray(x_iq, dtype=np.float32)
        out = np.zeros(max(capacity, 1), DETECTION_DTYPE)
        cnt = np.zeros(1, np.int32)
        self.run_host_ptr(stream, x_iq.ctypes.data, x_iq.shape[0], out.ctypes.data, capacity, cnt.ctypes.data)
        n = int(cnt[0])
        return out[: min(n, capacity)].copy(), n


def run_static_ptr(stream: int, d_iq: int, n_samples: int, d_chips: int, n_chips: int, samples_per_chip: int,
                   fs_hz: float, freq_offsets_hz, fft_len: int, threshold: float, d_out: int, capacity: int,
                   d_count: int) -> None:
    """atlas_acq_run_static: one code, no context, no device allocation."""
    fr = np.ascontiguousarray(np.asarray(freq_offsets_hz, np.float64))
    _check(load().atlas_acq_run_static(stream, d_iq, n_samples, d_chips, n_chips, samples_per_chip, float(fs_hz),
                                       fr.ctypes.data, len(fr), fft_len, float(threshold), d_out, capacity,
                                       d_count))


class Batch:
    """atlas_acq_batch_*: one CUDA graph over many streams, each with its own Search."""

    def __init__(self, searches: Sequence["Search"], d_iq_ptrs: Sequence[int], n_samples: Sequence[int],
                 d_out: int, capacity: int, d_count: int):
        lib = load()
        self._lib = lib
        self.b = ctypes.c_void_p()
        n = len(searches)
        self._ctxs = (ctypes.c_void_p * n)(*[s.ctx.value if isinstance(s.ctx, ctypes.c_void_p) else s.ctx
                                            for s in searches])
        self._x = (ctypes.c_void_p * n)(*d_iq_ptrs)
        self._ns = (ctypes.c_int64 * n)(*n_samples)
        st = lib.atlas_acq_batch_create(ctypes.byref(self.b), ctypes.cast(self._ctxs, ctypes.c_void_p), n,
                                        ctypes.cast(self._x, ctypes.c_void_p), ctypes.cast(self._ns, ctypes.c_void_p),
                                        d_out, capacity, d_count)
        if st != ATLAS_OK:
            self.b = None
        _check(st, searches[0].ctx if st == ATLAS_ERR_CUDA else None)

    def run(self, stream: int) -> None:
        _check(self._lib.atlas_acq_batch_run(self.b, stream))

    def kernels(self) -> int:
        return int(self._lib.atlas_acq_batch_kernels(self.b))

    def close(self) -> None:
        if self.b:
            self._lib.atlas_acq_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Proposal:
    """atlas_prop_*: the learned (code, bin) proposal network."""

    def __init__(self, n_codes: int, n_bins: int, seed: int = 0):
        lib = load()
        self._lib = lib
        self.p = ctypes.c_void_p()
        _check(lib.atlas_prop_create(ctypes.byref(self.p), n_codes, n_bins, seed))
        self.n_codes, self.n_bins = n_codes, n_bins
        self.n_params = int(lib.atlas_prop_num_params(self.p))
        self.feature_len = int(lib.atlas_prop_feature_len(self.p))

    def _chk(self, st):
        if st != ATLAS_OK:
            msg = strerror(st)
            if st == ATLAS_ERR_CUDA:
                msg += ": " + self._lib.atlas_prop_last_error(self.p).decode()
            raise AtlasError(st, msg)

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        self._chk(self._lib.atlas_prop_get_params(self.p, out.ctypes.data))
        return out

    def set_params(self, v: np.ndarray) -> None:
        v = np.ascontiguousarray(v, np.float32)
        assert v.size == self.n_params
        self._chk(self._lib.atlas_prop_set_params(self.p, v.ctypes.data))

    def save(self, path: str) -> None:
        self._chk(self._lib.atlas_prop_save(self.p, path.encode()))

    def load(self, path: str) -> None:
        self._chk(self._lib.atlas_prop_load(self.p, path.encode()))

    def set_grid(self, fs_hz: float, freqs_hz) -> None:
        f = np.ascontiguousarray(freqs_hz, np.float64)
        self._chk(self._lib.atlas_prop_set_grid(self.p, float(fs_hz), f.ctypes.data, f.size))

    def features(self, stream: int, d_iq: int, n_samples: int, first: int, stride: int, window_len: int,
                 n_windows: int, d_feat: int) -> None:
        self._chk(self._lib.atlas_prop_features(self.p, stream, d_iq, n_samples, first, stride, window_len,
                                                n_windows, d_feat))

    def loss_grad(self, stream: int, d_feat: int, d_code: int, d_bin: int, batch: int, d_loss: int,
                  d_grad: int = 0) -> None:
        self._chk(self._lib.atlas_prop_loss_grad(self.p, stream, d_feat, d_code, d_bin, batch, d_loss,
                                                 d_grad or None))

    def adam(self, stream: int, lr: float, d_grad: int = 0) -> None:
        self._chk(self._lib.atlas_prop_adam(self.p, stream, d_grad or None, lr))

    def logits(self, stream: int, d_feat: int, batch: int, half: bool, d_zc: int, d_zb: int, d_zp: int) -> None:
        self._chk(self._lib.atlas_prop_logits(self.p, stream, d_feat, batch, 1 if half else 0, d_zc or None,
                                              d_zb or None, d_zp or None))

    def candidates(self, stream: int, d_feat: int, n_windows: int, topk: int, d_cand: int, d_conf: int) -> None:
        self._chk(self._lib.atlas_prop_candidates(self.p, stream, d_feat, n_windows, topk, d_cand, d_conf))

    def bin_candidates(self, stream: int, d_feat: int, n_windows: int, n_top: int, d_bins: int, d_conf: int) -> None:
        self._chk(self._lib.atlas_prop_bin_candidates(self.p, stream, d_feat, n_windows, n_top, d_bins, d_conf))

    def close(self) -> None:
        if self.p:
            self._lib.atlas_prop_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_proposed(search: "Search", prop: Proposal, stream: int, d_iq: int, n_samples: int, topk: int,
                 tau_fb: float, d_out: int, capacity: int, d_count: int) -> int:
    """atlas_acq_run_proposed; returns the number of windows that fell back to the exhaustive search."""
    nfb = ctypes.c_int32(0)
    _check(load().atlas_acq_run_proposed(search.ctx, prop.p, stream, d_iq, n_samples, topk, float(tau_fb), d_out,
                                         capacity, d_count, ctypes.byref(nfb)), search.ctx)
    return nfb.value


def run_proposed_bins(search: "Search", prop: Proposal, stream: int, d_iq: int, n_samples: int, n_top: int,
                      tau_fb: float, d_out: int, capacity: int, d_count: int) -> int:
    """atlas_acq_run_proposed_bins (every code in the top n_top bins of a confident
    window); returns the number of windows that fell back to the exhaustive search."""
    nfb = ctypes.c_int32(0)
    _check(load().atlas_acq_run_proposed_bins(search.ctx, prop.p, stream, d_iq, n_samples, n_top, float(tau_fb),
                                              d_out, capacity, d_count, ctypes.byref(nfb)), search.ctx)
    return nfb.value


# ---------------------------------------------------------------------------
# FSK front end (include/atlas_fsk.h)
# ---------------------------------------------------------------------------

def _check_fsk(status: int, ctx=None) -> None:
    if status != ATLAS_OK:
        msg = strerror(status)
        if ctx is not None and status == ATLAS_ERR_CUDA:
            msg += ": " + load().atlas_fsk_last_error(ctx).decode()
        raise AtlasError(status, msg)


class FskSearch:
    """An FSK search context (atlas_fsk_create / atlas_fsk_destroy)."""

    def __init__(self, chips: Sequence[np.ndarray], samples_per_chip: int, fs_hz: float, f1_hz: float,
                 f0_hz: float, f_lo_hz: float, h_bp: np.ndarray, threshold: float = 49.0, fft_len: int = 0,
                 windows_per_launch: int = 0, exchange: int = 0, block_log2: int = 0):
        lib = load()
        self._lib = lib
        self.ctx = ctypes.c_void_p()
        cat = np.ascontiguousarray(np.concatenate([np.asarray(c, np.int8) for c in chips]))
        cpc = np.ascontiguousarray(np.array([len(c) for c in chips], np.int32))
        h = np.asarray(h_bp)
        taps = np.ascontiguousarray(np.stack([h.real, h.imag], axis=-1).astype(np.float64)) \
            if np.iscomplexobj(h) else np.ascontiguousarray(
                np.stack([h.astype(np.float64), np.zeros(h.shape[0])], axis=-1))
        o = FskOpts()
        lib.atlas_fsk_default_opts(ctypes.byref(o))
        o.threshold = threshold
        o.fft_len = fft_len
        o.windows_per_launch = windows_per_launch
        o.exchange = exchange
        o.block_log2 = block_log2
        self.n_codes = len(chips)
        st = lib.atlas_fsk_create(ctypes.byref(self.ctx), cat.ctypes.data, cpc.ctypes.data, len(chips),
                                  samples_per_chip, float(fs_hz), float(f1_hz), float(f0_hz), float(f_lo_hz),
                                  taps.ctypes.data, taps.shape[0], ctypes.byref(o))
        if st != ATLAS_OK:
            self.ctx = None
        _check_fsk(st)

    def close(self) -> None:
        if self.ctx:
            self._lib.atlas_fsk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def windows(self, code: int, n_samples: int):
        """(W, hop, N, n_c) of a code."""
        v = [ctypes.c_int32() for _ in range(4)]
        _check_fsk(self._lib.atlas_fsk_windows(self.ctx, code, n_samples, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def run_ptr(self, stream: int, d_iq: int, n_samples: int, d_out: int, capacity: int, d_count: int) -> None:
        _check_fsk(self._lib.atlas_fsk_run(self.ctx, stream, d_iq, n_samples, d_out, capacity, d_count), self.ctx)

    def run_codes_ptr(self, stream: int, d_iq: int, n_samples: int, first_sample: int, codes, d_out: int,
                      capacity: int, d_count: int) -> None:
        """codes: None for every code, else a list of code indices (may be empty)."""
        if codes is None:
            ptr, n = None, 0
        else:
            lst = np.asarray(codes, np.int32).reshape(-1)
            sel = np.zeros(max(lst.size, 1), np.int32)
            sel[: lst.size] = lst
            ptr, n = sel.ctypes.data, lst.size
        _check_fsk(self._lib.atlas_fsk_run_codes(self.ctx, stream, d_iq, n_samples, first_sample, ptr, n, d_out,
                                                 capacity, d_count), self.ctx)

    def run_host_ptr(self, stream: int, h_iq: int, n_samples: int, h_out: int, capacity: int,
                     h_count: int) -> None:
        _check_fsk(self._lib.atlas_fsk_run_host(self.ctx, stream, h_iq, n_samples, h_out, capacity, h_count),
                   self.ctx)

    def demod_ptr(self, stream: int, d_iq: int, n_samples: int, start: int, count: int, d_d: int,
                  d_u: int = 0) -> None:
        _check_fsk(self._lib.atlas_fsk_demod(self.ctx, stream, d_iq, n_samples, start, count, d_d, d_u or None),
                   self.ctx)

    def code_demod(self, code: int) -> np.ndarray:
        n = ctypes.c_int32()
        _check_fsk(self._lib.atlas_fsk_code_demod(self.ctx, code, None, 0, ctypes.byref(n)), self.ctx)
        out = np.zeros(n.value, np.float32)
        _check_fsk(self._lib.atlas_fsk_code_demod(self.ctx, code, out.ctypes.data, n.value, ctypes.byref(n)),
                   self.ctx)
        return out

    def profile_begin(self, max_timed: int = 65536) -> None:
        _check_fsk(self._lib.atlas_fsk_profile_begin(self.ctx, max_timed), self.ctx)

    def profile_end(self) -> dict:
        p = FskProfile()
        _check_fsk(self._lib.atlas_fsk_profile_end(self.ctx, ctypes.byref(p)), self.ctx)
        return {f: getattr(p, f) for f, _ in FskProfile._fields_}

    # torch conveniences ---------------------------------------------------
    def run(self, iq, capacity: int = 4096, stream=None):
        """iq: torch CUDA int16 tensor [S, 2].  Returns (detections as a numpy
        structured array, count)."""
        import torch
        assert iq.is_cuda and iq.dtype == torch.int16 and iq.is_contiguous()
        S = iq.shape[0]
        out = torch.zeros(max(capacity, 1) * FSK_DETECTION_DTYPE.itemsize, dtype=torch.uint8, device=iq.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=iq.device)
        st = stream if stream is not None else torch.cuda.current_stream(iq.device).cuda_stream
        self.run_ptr(st, iq.data_ptr(), S, out.data_ptr(), capacity, cnt.data_ptr())
        torch.cuda.current_stream(iq.device).synchronize() if stream is None else None
        n = int(cnt.item())
        dets = out.cpu().numpy().view(FSK_DETECTION_DTYPE)[: min(n, capacity)].copy()
        return dets, n

    def run_host(self, iq16: np.ndarray, capacity: int = 4096, stream: int = 0):
        a = np.ascontiguousarray(iq16, dtype=np.int16)
        out = np.zeros(max(capacity, 1), FSK_DETECTION_DTYPE)
        cnt = ctypes.c_int32()
        self.run_host_ptr(stream, a.ctypes.data, a.shape[0], out.ctypes.data, capacity, ctypes.addressof(cnt))
        return out[: min(cnt.value, capacity)].copy(), cnt.value


# ---------------------------------------------------------------------------
# continuous ingest and scheduler (include/atlas_rt.h)
# ---------------------------------------------------------------------------

def rt_default_opts(fs_hz: float) -> RtOpts:
    o = RtOpts()
    load().atlas_rt_default_opts(ctypes.byref(o), float(fs_hz))
    return o


class Runtime:
    """Cyclic device buffer + searching/tracking scheduler over an FskSearch."""

    def __init__(self, fsk: FskSearch, period_samples: Sequence[float], opts: Optional[RtOpts] = None,
                 fs_hz: float = 8e6):
        lib = load()
        self._lib = lib
        self.fsk = fsk  # kept alive: the runtime borrows the context
        self.ctx = ctypes.c_void_p()
        per = np.ascontiguousarray(np.asarray(period_samples, np.float64))
        o = opts if opts is not None else rt_default_opts(fs_hz)
        st = lib.atlas_rt_create(ctypes.byref(self.ctx), fsk.ctx, per.ctypes.data, per.size, ctypes.byref(o))
        if st != ATLAS_OK:
            self.ctx = None
        _check(st)

    def _chk(self, st):
        if st != ATLAS_OK:
            msg = strerror(st)
            if st == ATLAS_ERR_CUDA:
                msg += ": " + self._lib.atlas_rt_last_error(self.ctx).decode()
            raise AtlasError(st, msg)

    def push(self, iq16: np.ndarray, stream: int = 0) -> None:
        a = np.ascontiguousarray(iq16, dtype=np.int16)
        self._chk(self._lib.atlas_rt_push(self.ctx, stream, a.ctypes.data, a.shape[0]))

    def pump(self, max_tasks: int = 0, cap: int = 4096, stream: int = 0) -> np.ndarray:
        ev = np.zeros(max(cap, 1), RT_EVENT_DTYPE)
        n = ctypes.c_int32()
        self._chk(self._lib.atlas_rt_pump(self.ctx, stream, max_tasks, ev.ctypes.data, cap, ctypes.byref(n)))
        return ev[: min(n.value, cap)].copy()

    def stats(self) -> dict:
        s = RtStats()
        self._chk(self._lib.atlas_rt_get_stats(self.ctx, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in RtStats._fields_ if f != "reserved"}

    def close(self) -> None:
        if self.ctx:
            self._lib.atlas_rt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# comparison pipeline (include/atlas_unfused.h): measurement baseline only
# ---------------------------------------------------------------------------

class UnfusedSearch:
    """The coherent search organised like the paper's GPU implementation (cuFFT +
    element-wise kernels, the correlation surface in device memory)."""

    def __init__(self, chips: Sequence[np.ndarray], samples_per_chip: int, fs_hz: float,
                 freq_offsets_hz: Sequence[float], threshold: float = 25.0, fft_len: int = 0,
                 windows_per_launch: int = 0):
        lib = load()
        self._lib = lib
        self.ctx = ctypes.c_void_p()
        cat = np.ascontiguousarray(np.concatenate([np.asarray(c, np.int8) for c in chips]))
        cpc = np.ascontiguousarray(np.array([len(c) for c in chips], np.int32))
        fr = np.ascontiguousarray(np.asarray(freq_offsets_hz, np.float64))
        st = lib.atlas_unfused_create(ctypes.byref(self.ctx), cat.ctypes.data, cpc.ctypes.data, len(chips),
                                      samples_per_chip, float(fs_hz), fr.ctypes.data, len(fr), fft_len,
                                      float(threshold), windows_per_launch)
        if st != ATLAS_OK:
            self.ctx = None
        _check(st)

    def run_ptr(self, stream: int, d_iq: int, n_samples: int, d_out: int, capacity: int, d_count: int) -> None:
        st = self._lib.atlas_unfused_run(self.ctx, stream, d_iq, n_samples, d_out, capacity, d_count)
        if st != ATLAS_OK:
            raise AtlasError(st, strerror(st) + ": " + self._lib.atlas_unfused_last_error(self.ctx).decode())

    def run(self, x_iq, capacity: int = 4096):
        import torch
        out = torch.zeros(max(capacity, 1) * 32, dtype=torch.uint8, device=x_iq.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=x_iq.device)
        st = torch.cuda.current_stream(x_iq.device)
        self.run_ptr(st.cuda_stream, x_iq.data_ptr(), x_iq.shape[0], out.data_ptr(), capacity, cnt.data_ptr())
        st.synchronize()
        n = int(cnt.item())
        return out.cpu().numpy().view(DETECTION_DTYPE)[: min(n, capacity)].copy(), n

    def close(self) -> None:
        if self.ctx:
            self._lib.atlas_unfused_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FskTracker:
    """atlas_fsk_tracker_*: one code on a block of a device cyclic buffer, one graph launch."""

    def __init__(self, fsk: FskSearch, code: int, n_samples: int, d_ring: int, ring_samples: int):
        lib = load()
        self._lib = lib
        self.fsk = fsk
        self.t = ctypes.c_void_p()
        _check_fsk(lib.atlas_fsk_tracker_create(ctypes.byref(self.t), fsk.ctx, code, n_samples, d_ring,
                                                ring_samples), fsk.ctx)

    def run(self, code: int, block_start: int, capacity: int = 64, stream: int = 0):
        out = np.zeros(max(capacity, 1), FSK_DETECTION_DTYPE)
        n = ctypes.c_int32()
        _check_fsk(self._lib.atlas_fsk_tracker_run(self.t, stream, code, block_start, out.ctypes.data, capacity,
                                                   ctypes.byref(n)), self.fsk.ctx)
        return out[: min(n.value, capacity)].copy(), n.value

    def kernels(self) -> int:
        """Kernel launches one run makes (the kernel nodes of the graph)."""
        return int(self._lib.atlas_fsk_tracker_kernels(self.t))

    def close(self) -> None:
        if self.t:
            self._lib.atlas_fsk_tracker_destroy(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
