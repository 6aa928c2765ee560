"""GB300 (sm_103a) FFA periodogram -- thin Python binding of libffa's C ABI.

Every step of the search (prefix sums, real-factor downsampling, FFA merges, boxcar
S/N) runs in the CUDA kernels of ``libffa.so``; this module only marshals arguments:
torch tensors supply device memory and the current CUDA stream.  There is no CPU
fallback: if the library is missing, every call raises.

Calls (names follow include/ffa.h and the paper, Morello et al. 2020):
  downsample(x, factor)                         Sec. 5.3, App. A.4
  ffa_transform(block)                          Sec. 2.2, Eq. ffa_merge_rule
  boxcar_snr(prof, widths, stdnoise)            Sec. 5.4
  periodogram_plan(n, tsamp, pmin, pmax, bmin, bmax, widths)
  periodogram(x, tsamp, pmin, pmax, bmin, bmax, widths)        Sec. 5.3, Fig. 4
  periodogram_host(x_host, ...)                 same, host buffers in and out
  BatchSearcher(series, widths)                 many series in one buffer, Sec. 5.7
  SegmentSearcher(n, tsamp, segments, widths)   dynamic duty-cycle resolution, Sec. 5.6
  running_median(x, width), deredden(x, width)  de-reddening before normalising, Sec. 5.2
  find_peaks(periods, snr, tobs)                peak finding per width, Sec. 5.5, Fig. 6
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, replace
from typing import Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "FFAError", "library", "build", "normalise", "downsample", "ffa_transform", "boxcar_snr",
    "PlanInfo", "periodogram_plan", "periodogram", "periodogram_host", "Searcher",
    "Series", "BatchInfo", "batch_plan", "BatchSearcher", "periodogram_batch", "shard_series",
    "Tiles", "tile_candidates", "tune", "tune_periodogram", "SegmentSearcher",
    "check", "plan_cache_clear", "launch_count", "kernel_names", "profile_enable", "profile_reset",
    "profile_query", "RunningMedian", "running_median", "deredden", "median_width",
    "PeakFinder", "find_peaks", "PEAK_DTYPE", "prepare_batch", "set_wait_limit_ms",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libffa.so")
# The bounds-checked debug build (same entry points); loaded instead of libffa.so when the
# environment has FFA_LIBRARY=checked at the first call (FFA_LIBRARY=<path to a .so>
# loads another build of the same sources).
LIB_CHECKED_PATH = os.path.join(_PKG, "libffa_checked.so")


def _lib_path() -> str:
    v = os.environ.get("FFA_LIBRARY", "")
    if v == "checked":
        return LIB_CHECKED_PATH
    return v if v.endswith(".so") else LIB_PATH

FFA_F32, FFA_F16, FFA_I8 = 0, 1, 2
_STATUS = {0: "FFA_OK", 1: "FFA_ERR_ARG", 2: "FFA_ERR_CAPACITY", 3: "FFA_ERR_CUDA",
           4: "FFA_ERR_TIMEOUT", 5: "FFA_ERR_UNSUPPORTED", 6: "FFA_ERR_DEVICE"}


class FFAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), message))
        self.status = status


MAX_TILE_CLASSES = 8  # FFA_MAX_TILE_CLASSES


class _TileClass(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int32), ("p_max", ctypes.c_int32),
                ("subtree_rows", ctypes.c_int32), ("top_levels", ctypes.c_int32),
                ("top_rows", ctypes.c_int32)]


class _PlanOpts(ctypes.Structure):
    _fields_ = [("subtree_rows", ctypes.c_int32), ("top_levels", ctypes.c_int32),
                ("top_rows", ctypes.c_int32), ("boxcar", ctypes.c_int32),
                ("nclasses", ctypes.c_int32), ("classes", _TileClass * MAX_TILE_CLASSES)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("ntrials", ctypes.c_int64), ("noctaves", ctypes.c_int32),
                ("ntransforms", ctypes.c_int32), ("nwidths", ctypes.c_int32),
                ("max_rows", ctypes.c_int32), ("downsampled_samples", ctypes.c_int64),
                ("folded_samples", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t),
                ("host_workspace_bytes", ctypes.c_size_t), ("opts", _PlanOpts),
                ("ffa_adds", ctypes.c_double), ("snr_ops", ctypes.c_double)]


class _Series(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("n", ctypes.c_int64), ("tsamp", ctypes.c_double),
                ("pmin", ctypes.c_double), ("pmax", ctypes.c_double), ("bmin", ctypes.c_int32),
                ("bmax", ctypes.c_int32)]


class _PeakOpts(ctypes.Structure):
    _fields_ = [("dzseg", ctypes.c_double), ("nsigma", ctypes.c_double),
                ("clrad", ctypes.c_double), ("degree", ctypes.c_int32),
                ("min_seg", ctypes.c_int32), ("max_segments", ctypes.c_int64)]


# one ffa_peak record
PEAK_DTYPE = np.dtype([("trial", "<i8"), ("period", "<f8"), ("snr", "<f4"), ("iw", "<i4")])


class _BatchInfo(ctypes.Structure):
    _fields_ = [("ntrials", ctypes.c_int64), ("nchunks", ctypes.c_int32),
                ("ntransforms", ctypes.c_int32), ("folded_samples", ctypes.c_int64),
                ("input_samples", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t)]


_lib = None


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def library() -> ctypes.CDLL:
    """The loaded libffa.so (libffa_checked.so with FFA_LIBRARY=checked).  Raises if it
    has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _lib_path()
    if not os.path.exists(path):
        raise RuntimeError("%s is not built (run __graft_entry__.build()); "
                           "there is no CPU fallback" % os.path.basename(path))
    L = ctypes.CDLL(path)
    i32, i64, dbl, vp, sz = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                             ctypes.c_size_t)
    L.ffa_last_error.restype = ctypes.c_char_p
    L.ffa_version.restype = ctypes.c_char_p
    L.ffa_downsample_workspace.argtypes = [i64, ctypes.POINTER(sz)]
    L.ffa_downsample.argtypes = [vp, i64, dbl, vp, i64, ctypes.POINTER(i64), vp, sz, vp]
    L.ffa_downsample_length.argtypes = [i64, dbl, ctypes.POINTER(i64)]
    L.ffa_transform_workspace.argtypes = [i32, i32, ctypes.POINTER(sz)]
    L.ffa_transform.argtypes = [vp, i32, i32, vp, vp, sz, vp]
    L.ffa_boxcar_snr.argtypes = [vp, i32, i32, vp, i32, dbl, vp, vp]
    L.ffa_periodogram_plan.argtypes = [i64, dbl, dbl, dbl, i32, i32, vp, i32,
                                       ctypes.POINTER(_PlanInfo)]
    L.ffa_periodogram_plan_opts.argtypes = [i64, dbl, dbl, dbl, i32, i32, vp, i32, vp,
                                            ctypes.POINTER(_PlanInfo)]
    L.ffa_periodogram_opts.argtypes = [vp, i32, i64, dbl, dbl, dbl, i32, i32, vp, i32, vp, vp,
                                       vp, vp, i64, vp, sz, vp]
    L.ffa_batch_plan_opts.argtypes = [vp, i32, vp, i32, sz, vp, vp, ctypes.POINTER(_BatchInfo)]
    L.ffa_periodogram_batch_opts.argtypes = [vp, i32, vp, i32, vp, i32, sz, vp, vp, vp, vp,
                                             i64, vp, sz, vp]
    L.ffa_boxcar_snr_template.argtypes = [vp, i32, i32, vp, i32, dbl, i32, vp, vp]
    L.ffa_periodogram.argtypes = [vp, i32, i64, dbl, dbl, dbl, i32, i32, vp, i32, vp, vp, vp,
                                  i64, vp, sz, vp]
    L.ffa_periodogram_host.argtypes = [vp, i64, dbl, dbl, dbl, i32, i32, vp, i32, vp, vp, vp,
                                       i64, vp, sz, vp]
    L.ffa_check.argtypes = [vp, vp]
    L.ffa_set_wait_limit_ms.argtypes = [dbl]
    L.ffa_checked_status.argtypes = [ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint32)]
    L.ffa_periodogram_queue.argtypes = [i64, dbl, dbl, dbl, i32, i32, vp, i32, vp, vp, sz, vp,
                                        i64, ctypes.POINTER(i64), vp]
    L.ffa_batch_plan.argtypes = [vp, i32, vp, i32, sz, vp, ctypes.POINTER(_BatchInfo)]
    L.ffa_periodogram_batch.argtypes = [vp, i32, vp, i32, vp, i32, sz, vp, vp, vp, i64, vp,
                                        sz, vp]
    L.ffa_normalise_workspace.argtypes = [i64, ctypes.POINTER(sz)]
    L.ffa_normalise.argtypes = [vp, i64, vp, i32, vp, vp, sz, vp]
    L.ffa_peak_opts_default.restype = None
    L.ffa_peak_opts_default.argtypes = [ctypes.POINTER(_PeakOpts)]
    L.ffa_find_peaks_workspace.argtypes = [i64, i32, ctypes.POINTER(_PeakOpts), ctypes.POINTER(sz)]
    L.ffa_find_peaks.argtypes = [vp, vp, i64, i32, dbl, ctypes.POINTER(_PeakOpts), vp, i64, vp,
                                 vp, sz, vp]
    L.ffa_find_peaks_fits.argtypes = [vp, i64, i32, ctypes.POINTER(_PeakOpts),
                                      ctypes.POINTER(i64), vp, i64, vp, vp]
    L.ffa_running_median_workspace.argtypes = [i64, ctypes.POINTER(sz)]
    L.ffa_running_median.argtypes = [vp, i64, i64, vp, vp, vp, sz, vp]
    L.ffa_launch_count.restype = i64
    L.ffa_kernel_kinds.restype = i32
    L.ffa_kernel_name.restype = ctypes.c_char_p
    L.ffa_kernel_name.argtypes = [i32]
    L.ffa_profile_enable.argtypes = [i32]
    L.ffa_profile_query.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                    ctypes.POINTER(dbl)]
    for f in ("ffa_downsample_workspace", "ffa_downsample", "ffa_downsample_length",
              "ffa_transform_workspace",
              "ffa_transform", "ffa_boxcar_snr", "ffa_periodogram_plan", "ffa_periodogram",
              "ffa_periodogram_host", "ffa_check", "ffa_profile_enable", "ffa_profile_reset",
              "ffa_normalise_workspace", "ffa_normalise", "ffa_batch_plan",
              "ffa_periodogram_batch", "ffa_plan_cache_clear", "ffa_periodogram_plan_opts",
              "ffa_periodogram_opts", "ffa_batch_plan_opts", "ffa_periodogram_batch_opts",
              "ffa_boxcar_snr_template", "ffa_running_median_workspace",
              "ffa_running_median", "ffa_find_peaks_workspace", "ffa_find_peaks",
              "ffa_profile_query", "ffa_set_wait_limit_ms", "ffa_find_peaks_fits",
              "ffa_checked_status", "ffa_periodogram_queue"):
        getattr(L, f).restype = i32
    _lib = L
    return L


def _check(status: int) -> None:
    if status != 0:
        raise FFAError(status, library().ffa_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> ctypes.c_void_p:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _on(stream):
    """Context of a one-shot call on `stream`: its workspace and outputs are allocated on
    the stream its kernels run on, so that torch's caching allocator never hands that
    memory to work on another stream while the kernels may still use it (and reads such
    as tolist() are ordered after them)."""
    import contextlib
    return _torch().cuda.stream(stream) if stream is not None else contextlib.nullcontext()


def _keep(stream, *tensors):
    """A long-lived object's buffers used on `stream`: the allocator waits for that
    stream's work before it reuses them once they are freed."""
    if stream is None:
        return
    for t in tensors:
        if t is not None:
            t.record_stream(stream)


def _dev_tensor(t, name: str):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _workspace(nbytes: int, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _widths_array(widths: Sequence[int]) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(widths, dtype=np.int32))


def _vp(a) -> ctypes.c_void_p:
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(a.data_ptr())


# ----------------------------------------------------------------------------------
def normalise(x, dtype=None, stream=None):
    """Whole-series normalisation (Sec. 3.1, 5.2) of a float32 CUDA series.

    Returns (x', mean, std): x' of `dtype` (torch.float32, torch.float16, or torch.int8
    holding q with value q/16), mean and std as Python floats (FP64 on the device)."""
    torch = _torch()
    _dev_tensor(x, "x")
    if x.dtype != torch.float32 or x.dim() != 1:
        raise TypeError("x must be a 1-D float32 tensor")
    dtype = torch.float32 if dtype is None else dtype
    code = {torch.float32: FFA_F32, torch.float16: FFA_F16, torch.int8: FFA_I8}[dtype]
    L = library()
    need = ctypes.c_size_t()
    _check(L.ffa_normalise_workspace(x.numel(), ctypes.byref(need)))
    with _on(stream):
        ws = _workspace(need.value, x.device)
        out = torch.empty(x.numel(), dtype=dtype, device=x.device)
        stats = torch.empty(2, dtype=torch.float64, device=x.device)
        _check(L.ffa_normalise(_vp(x), x.numel(), _vp(out), code, _vp(stats), _vp(ws),
                               ws.numel(), _stream_handle(stream)))
        m, s = stats.tolist()
    return out, m, s


def median_width(seconds: float, tsamp: float) -> int:
    """Samples of a running-median window of `seconds`, made odd (Sec. 5.2 leaves the
    width to the user)."""
    return max(1, int(round(seconds / tsamp))) | 1


class RunningMedian:
    """Running median over an odd window of `width` samples (Sec. 5.2 de-reddening),
    for float32 CUDA series of `n` samples, with a workspace kept across calls.

    ``S(x, med=None, y=None)`` writes med[i], the median of x[i-h .. i+h] with the
    series extended by its end samples (width = 2h + 1), and/or y = x - med; either
    output may be ``x`` itself (in place).  Asynchronous on the current stream."""

    def __init__(self, n: int, width: int, device="cuda"):
        torch = _torch()
        L = library()
        need = ctypes.c_size_t()
        _check(L.ffa_running_median_workspace(int(n), ctypes.byref(need)))
        self.n, self.width = int(n), int(width)
        self.device = torch.device(device)
        self.ws = _workspace(need.value, self.device)

    def __call__(self, x, med=None, y=None, stream=None):
        torch = _torch()
        _dev_tensor(x, "x")
        if x.dtype != torch.float32 or x.numel() != self.n:
            raise TypeError("x must be a float32 CUDA tensor of %d samples" % self.n)
        for t, name in ((med, "med"), (y, "y")):
            if t is not None:
                _dev_tensor(t, name)
                if t.dtype != torch.float32 or t.numel() != self.n:
                    raise TypeError("%s must be a float32 CUDA tensor of %d samples" % (name, self.n))
        _check(library().ffa_running_median(
            _vp(x), self.n, self.width, _vp(med) if med is not None else None,
            _vp(y) if y is not None else None, _vp(self.ws), self.ws.numel(),
            _stream_handle(stream)))
        _keep(stream, self.ws)
        return med, y


def prepare_batch(x, spans, width: Optional[int], dtype=None, stream=None):
    """The steps before the search of a batch of series (Sec. 5.2), each series on its
    own: de-redden x in place by a running median of `width` samples (None: skip), then
    normalise into a new buffer of `dtype` (float32, float16 or int8 holding q with value
    q/16).  `spans`: (offset, n) of every series in the float32 CUDA buffer x."""
    torch = _torch()
    _dev_tensor(x, "x")
    with _on(stream):
        out = torch.empty(x.numel(), dtype=torch.float32 if dtype is None else dtype,
                          device=x.device)
        med = {}
        for o, n in spans:
            v = x[o:o + n]
            if width is not None:
                if n not in med:
                    med[n] = RunningMedian(n, width, x.device)
                med[n](v, y=v)
            out[o:o + n] = normalise(v, dtype=out.dtype)[0]
    return out


def running_median(x, width: int, stream=None):
    """The running median of a float32 CUDA series (Sec. 5.2), a new tensor."""
    with _on(stream):
        med = _torch().empty_like(x)
        RunningMedian(x.numel(), width, x.device)(x, med=med)
    return med


def deredden(x, width: int, inplace: bool = False, stream=None):
    """x minus its running median over `width` samples (Sec. 5.2): the red-noise removal
    that precedes `normalise`.  In place if `inplace`."""
    with _on(stream):
        y = x if inplace else _torch().empty_like(x)
        RunningMedian(x.numel(), width, x.device)(x, y=y)
    return y


class PeakFinder:
    """Peak finding on periodograms of `ntrials` trials and `nw` widths (Sec. 5.5,
    Fig. 6), with its workspace and output buffers kept across calls.

    ``F(periods, snr)`` searches a periodogram on the device (float64 periods, positive
    and non-decreasing; float32 S/N of shape (ntrials, nw)), asynchronously on the
    current stream.  ``F.result()`` synchronises and returns the peaks (a numpy array of
    PEAK_DTYPE: width by width, by increasing period within a width) and the number of
    peaks per width.  Options as in ffa_peak_opts; `peak_cap` bounds the stored peaks."""

    def __init__(self, ntrials: int, nw: int, tobs: float, dzseg: float = 5.0,
                 nsigma: float = 6.0, degree: int = 2, clrad: float = 1.0, min_seg: int = 8,
                 max_segments: int = 1 << 16, peak_cap: Optional[int] = None, device="cuda"):
        torch = _torch()
        L = library()
        self.opts = _PeakOpts(float(dzseg), float(nsigma), float(clrad), int(degree),
                              int(min_seg), int(max_segments))
        need = ctypes.c_size_t()
        _check(L.ffa_find_peaks_workspace(int(ntrials), int(nw), ctypes.byref(self.opts),
                                          ctypes.byref(need)))
        self.ntrials, self.nw, self.tobs = int(ntrials), int(nw), float(tobs)
        self.device = torch.device(device)
        self.ws = _workspace(need.value, self.device)
        self.cap = int(peak_cap) if peak_cap is not None else max(1024, 4 * self.ntrials // 1000)
        self.peaks = torch.empty(max(self.cap, 1) * PEAK_DTYPE.itemsize, dtype=torch.uint8,
                                 device=self.device)
        self.npeaks = torch.zeros(self.nw + 1, dtype=torch.int64, device=self.device)

    def __call__(self, periods, snr, stream=None):
        torch = _torch()
        _dev_tensor(periods, "periods")
        _dev_tensor(snr, "snr")
        if periods.dtype != torch.float64 or periods.numel() != self.ntrials:
            raise TypeError("periods must be %d float64 values" % self.ntrials)
        if snr.dtype != torch.float32 or snr.numel() != self.ntrials * self.nw:
            raise TypeError("snr must be %d x %d float32 values" % (self.ntrials, self.nw))
        _check(library().ffa_find_peaks(
            _vp(periods), _vp(snr), self.ntrials, self.nw, self.tobs, ctypes.byref(self.opts),
            _vp(self.peaks), self.cap, _vp(self.npeaks), _vp(self.ws), self.ws.numel(),
            _stream_handle(stream)))
        _keep(stream, self.ws, self.peaks, self.npeaks)

    def check(self, stream=None) -> None:
        _check(library().ffa_check(_vp(self.ws), _stream_handle(stream)))

    def fits(self, stream=None):
        """The last search's control points and threshold fits (see ffa_find_peaks_fits):
        (ctrl [segments, nw, 2] {nu_j, s_j, NaN s_j without a point}, fits [nw, 10]
        {xbar, xscale, valid, c_0 .. c_6})."""
        nseg = ctypes.c_int64()
        cap = int(self.opts.max_segments)
        ctrl = np.empty((cap, self.nw, 2), np.float64)
        fits = np.empty((self.nw, 10), np.float64)
        _check(library().ffa_find_peaks_fits(_vp(self.ws), self.ntrials, self.nw,
                                             ctypes.byref(self.opts), ctypes.byref(nseg),
                                             _vp(ctrl), cap, _vp(fits), _stream_handle(stream)))
        return ctrl[:min(nseg.value, cap)].copy(), fits

    def result(self):
        counts = self.npeaks.cpu().numpy()
        k = int(min(counts[-1], self.cap))
        raw = self.peaks[:k * PEAK_DTYPE.itemsize].cpu().numpy()
        return raw.view(PEAK_DTYPE).copy(), counts[:-1].copy()


def find_peaks(periods, snr, tobs: float, **opts):
    """Peaks of a periodogram (Sec. 5.5): returns (peaks, counts per width); see
    PeakFinder for the options."""
    snr2 = snr if snr.dim() == 2 else snr.reshape(-1, 1)
    F = PeakFinder(periods.numel(), snr2.shape[1], tobs, device=periods.device, **opts)
    F(periods, snr2)
    return F.result()


def downsample(x, factor: float, stream=None):
    """Real-factor downsampling of a float32 CUDA series (Sec. 5.3, App. A.4)."""
    torch = _torch()
    _dev_tensor(x, "x")
    if x.dtype != torch.float32 or x.dim() != 1:
        raise TypeError("x must be a 1-D float32 tensor")
    L = library()
    n = x.numel()
    need = ctypes.c_size_t()
    _check(L.ffa_downsample_workspace(n, ctypes.byref(need)))
    nout = ctypes.c_int64()
    _check(L.ffa_downsample_length(n, float(factor), ctypes.byref(nout)))
    with _on(stream):
        ws = _workspace(need.value, x.device)
        out = torch.empty(max(nout.value, 1), dtype=torch.float32, device=x.device)
        got = ctypes.c_int64()
        _check(L.ffa_downsample(_vp(x), n, float(factor), _vp(out), out.numel(),
                                ctypes.byref(got), _vp(ws), ws.numel(), _stream_handle(stream)))
    return out[: got.value]


def ffa_transform(block, stream=None):
    """Folding transform of a (rows, cols) float32 CUDA block (Sec. 2.2)."""
    torch = _torch()
    _dev_tensor(block, "block")
    if block.dtype != torch.float32 or block.dim() != 2:
        raise TypeError("block must be a 2-D float32 tensor")
    L = library()
    m, p = block.shape
    need = ctypes.c_size_t()
    _check(L.ffa_transform_workspace(m, p, ctypes.byref(need)))
    with _on(stream):
        ws = _workspace(need.value, block.device)
        out = torch.empty_like(block)
        _check(L.ffa_transform(_vp(block), m, p, _vp(out), _vp(ws), ws.numel(),
                               _stream_handle(stream)))
    return out


def boxcar_snr(prof, widths: Sequence[int], stdnoise: float, stream=None,
               zero_mean: bool = False):
    """Boxcar S/N (rows, nw) of a (rows, cols) float32 CUDA profile array (Sec. 5.4);
    zero_mean: the zero-sum, unit-square-sum boxcar (widths below cols)."""
    torch = _torch()
    _dev_tensor(prof, "prof")
    if prof.dtype != torch.float32 or prof.dim() != 2:
        raise TypeError("prof must be a 2-D float32 tensor")
    w = _widths_array(widths)
    rows, cols = prof.shape
    with _on(stream):
        out = torch.empty((rows, len(w)), dtype=torch.float32, device=prof.device)
        _check(library().ffa_boxcar_snr_template(_vp(prof), rows, cols, _vp(w), len(w),
                                                 float(stdnoise),
                                                 BOXCAR_ZERO_MEAN if zero_mean else BOXCAR_PLAIN,
                                                 _vp(out), _stream_handle(stream)))
    return out


@dataclass
class PlanInfo:
    ntrials: int
    noctaves: int
    ntransforms: int
    nwidths: int
    max_rows: int
    downsampled_samples: int
    folded_samples: int
    workspace_bytes: int
    host_workspace_bytes: int
    tiles: "Tiles"
    ffa_adds: float
    snr_ops: float


@dataclass(frozen=True)
class TileClass:
    """Transforms with m <= m_max and p <= p_max (0: any) and their own tiles (0: the
    plan-wide value); see ffa_tile_class."""
    m_max: int = 0
    p_max: int = 0
    subtree_rows: int = 0
    top_levels: int = 0
    top_rows: int = 0


@dataclass(frozen=True)
class Tiles:
    """Tile shape of a plan (0 = the largest that fits shared memory), plus an optional
    table of per-class shapes (the first matching class of a transform wins); see
    ffa_plan_opts."""
    subtree_rows: int = 0
    top_levels: int = 0
    top_rows: int = 0
    classes: Tuple[TileClass, ...] = ()

    def with_class(self, i: int, **fields) -> "Tiles":
        cl = list(self.classes)
        cl[i] = replace(cl[i], **fields)
        return replace(self, classes=tuple(cl))


BOXCAR_PLAIN, BOXCAR_ZERO_MEAN = 0, 1


def _tiles_arg(tiles: Optional[Tiles], zero_mean: bool = False):
    """(struct kept alive, pointer) of plan options; NULL for all defaults."""
    if tiles is None and not zero_mean:
        return None, ctypes.c_void_p(None)
    t = tiles or Tiles()
    if len(t.classes) > MAX_TILE_CLASSES:
        raise ValueError("at most %d tile classes" % MAX_TILE_CLASSES)
    o = _PlanOpts(int(t.subtree_rows), int(t.top_levels), int(t.top_rows),
                  BOXCAR_ZERO_MEAN if zero_mean else BOXCAR_PLAIN, len(t.classes))
    for i, c in enumerate(t.classes):
        o.classes[i] = _TileClass(int(c.m_max), int(c.p_max), int(c.subtree_rows),
                                  int(c.top_levels), int(c.top_rows))
    return o, ctypes.cast(ctypes.byref(o), ctypes.c_void_p)


def _tiles_of(o: _PlanOpts) -> Tiles:
    return Tiles(o.subtree_rows, o.top_levels, o.top_rows,
                 tuple(TileClass(c.m_max, c.p_max, c.subtree_rows, c.top_levels, c.top_rows)
                       for c in o.classes[:o.nclasses]))


def periodogram_plan(n: int, tsamp: float, pmin: float, pmax: float, bmin: int, bmax: int,
                     widths: Sequence[int], tiles: Optional[Tiles] = None,
                     zero_mean: bool = False) -> PlanInfo:
    w = _widths_array(widths)
    info = _PlanInfo()
    keep, tp = _tiles_arg(tiles, zero_mean)
    _check(library().ffa_periodogram_plan_opts(n, tsamp, pmin, pmax, bmin, bmax, _vp(w), len(w),
                                               tp, ctypes.byref(info)))
    vals = [getattr(info, f) for f, _ in _PlanInfo._fields_[:-3]]
    return PlanInfo(*vals, _tiles_of(info.opts), info.ffa_adds, info.snr_ops)


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return FFA_F32
    if t.dtype == torch.float16:
        return FFA_F16
    if t.dtype == torch.int8:
        return FFA_I8
    raise TypeError("series dtype must be float32, float16 or int8 (value q/16)")


class Searcher:
    """Holds the workspace and outputs of one search configuration for repeated calls."""

    def __init__(self, n, tsamp, pmin, pmax, bmin, bmax, widths, device="cuda",
                 tiles: Optional[Tiles] = None, zero_mean: bool = False):
        torch = _torch()
        self.args = (int(n), float(tsamp), float(pmin), float(pmax), int(bmin), int(bmax))
        self.widths = _widths_array(widths)
        self.tiles = tiles
        self.zero_mean = bool(zero_mean)
        self._tiles_keep, self._tiles_ptr = _tiles_arg(tiles, zero_mean)
        self.info = periodogram_plan(*self.args, self.widths, tiles, zero_mean)
        T, nw = self.info.ntrials, len(self.widths)
        self.device = torch.device(device)
        self.ws = _workspace(self.info.workspace_bytes, self.device)
        # at least one element each, so that the device pointers are never null
        self._per = torch.empty(max(T, 1), dtype=torch.float64, device=self.device)
        self._fb = torch.empty(max(T, 1), dtype=torch.int32, device=self.device)
        self._snr = torch.empty((max(T, 1), nw), dtype=torch.float32, device=self.device)
        self.periods, self.foldbins, self.snr = self._per[:T], self._fb[:T], self._snr[:T]
        self._host_ws = None

    def __call__(self, x, stream=None):
        _dev_tensor(x, "x")
        if x.numel() != self.args[0]:
            raise ValueError("series length differs from the plan")
        n, tsamp, pmin, pmax, bmin, bmax = self.args
        _check(library().ffa_periodogram_opts(
            _vp(x), _dtype_code(x), n, tsamp, pmin, pmax, bmin, bmax, _vp(self.widths),
            len(self.widths), self._tiles_ptr, _vp(self._per), _vp(self._fb), _vp(self._snr),
            self.periods.numel(), _vp(self.ws), self.ws.numel(), _stream_handle(stream)))
        _keep(stream, self.ws, self._per, self._fb, self._snr)
        return self.periods, self.foldbins, self.snr

    def run_host(self, x_host, periods_h, foldbins_h, snr_h, stream=None):
        """End to end from host memory: copies in, searches, copies out, synchronises
        (with the default plan options)."""
        if self.zero_mean:
            raise ValueError("the host-buffer call uses the plain boxcar")
        if self._host_ws is None:
            info0 = self.info if self.tiles is None else periodogram_plan(*self.args, self.widths)
            self._host_ws = _workspace(info0.host_workspace_bytes, self.device)
        n, tsamp, pmin, pmax, bmin, bmax = self.args
        _check(library().ffa_periodogram_host(
            _vp(x_host), n, tsamp, pmin, pmax, bmin, bmax, _vp(self.widths), len(self.widths),
            _vp(periods_h), _vp(foldbins_h), _vp(snr_h), max(len(periods_h), self.info.ntrials),
            _vp(self._host_ws),
            self._host_ws.numel(), _stream_handle(stream)))

    def check(self, stream=None):
        check(self.ws, stream)

    def queue_records(self, stream=None) -> np.ndarray:
        """The work-item records of the last search's persistent launch (see
        ffa_periodogram_queue): an int32 array [items, 8] of {transform, index, pass,
        batch, wait counter, count needed, released counter, depth}, in queue order."""
        L = library()
        n = ctypes.c_int64()
        args = (*self.args, _vp(self.widths), len(self.widths), self._tiles_ptr, _vp(self.ws),
                self.ws.numel())
        _check(L.ffa_periodogram_queue(*args, None, 0, ctypes.byref(n), _stream_handle(stream)))
        out = np.zeros((max(n.value, 1), 8), np.int32)
        _check(L.ffa_periodogram_queue(*args, _vp(out), n.value, ctypes.byref(n),
                                       _stream_handle(stream)))
        return out[:n.value]


def periodogram(x, tsamp: float, pmin: float, pmax: float, bmin: int, bmax: int,
                widths: Sequence[int], stream=None, zero_mean: bool = False):
    """FFA periodogram of a normalised CUDA series (float32, float16 or int8 as q/16).

    Returns (periods float64 [T], foldbins int32 [T], snr float32 [T, nw]) on the device.
    """
    with _on(stream):
        s = Searcher(x.numel(), tsamp, pmin, pmax, bmin, bmax, widths, device=x.device,
                     zero_mean=zero_mean)
        return s(x)


def periodogram_host(x: np.ndarray, tsamp, pmin, pmax, bmin, bmax, widths, device="cuda"):
    """Same search from and to host numpy arrays (copies inside the call)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    s = Searcher(len(x), tsamp, pmin, pmax, bmin, bmax, widths, device=device)
    T, nw = s.info.ntrials, len(s.widths)
    per = np.empty(max(T, 1), np.float64)
    fb = np.empty(max(T, 1), np.int32)
    snr = np.empty((max(T, 1), nw), np.float32)
    s.run_host(x, per, fb, snr)
    return per[:T], fb[:T], snr[:T]


@dataclass(frozen=True)
class Series:
    """One series of a batch: samples [offset, offset + n) of the batch buffer."""
    offset: int
    n: int
    tsamp: float
    pmin: float
    pmax: float
    bmin: int
    bmax: int


@dataclass
class BatchInfo:
    ntrials: int
    nchunks: int
    ntransforms: int
    folded_samples: int
    input_samples: int
    workspace_bytes: int


def _series_array(series: Sequence[Series]):
    arr = (_Series * max(len(series), 1))()
    for i, s in enumerate(series):
        arr[i] = _Series(int(s.offset), int(s.n), float(s.tsamp), float(s.pmin), float(s.pmax),
                         int(s.bmin), int(s.bmax))
    return arr


# default workspace budget of one launch sequence of a batch (bytes)
DEFAULT_BATCH_BUDGET = 1 << 30


def batch_plan(series: Sequence[Series], widths: Sequence[int],
               ws_budget: int = DEFAULT_BATCH_BUDGET, tiles: Optional[Tiles] = None,
               zero_mean: bool = False):
    """(BatchInfo, trial offsets int64 [len(series) + 1]) of a batch search."""
    w = _widths_array(widths)
    arr = _series_array(series)
    offs = np.zeros(len(series) + 1, np.int64)
    info = _BatchInfo()
    keep, tp = _tiles_arg(tiles, zero_mean)
    _check(library().ffa_batch_plan_opts(ctypes.cast(arr, ctypes.c_void_p), len(series), _vp(w),
                                          len(w), int(ws_budget), tp, _vp(offs),
                                          ctypes.byref(info)))
    return BatchInfo(*(getattr(info, f) for f, _ in _BatchInfo._fields_)), offs


class BatchSearcher:
    """Periodograms of many series stored one after another in one device buffer.

    Outputs of series i are rows trial_offsets[i]:trial_offsets[i+1] of periods,
    foldbins and snr.  The call is a fixed sequence of launches on one stream, so it can
    be captured into a CUDA graph once the searcher exists.
    """

    def __init__(self, series: Sequence[Series], widths: Sequence[int],
                 ws_budget: int = DEFAULT_BATCH_BUDGET, device="cuda",
                 tiles: Optional[Tiles] = None, zero_mean: bool = False):
        torch = _torch()
        self.series = list(series)
        self.widths = _widths_array(widths)
        self.ws_budget = int(ws_budget)
        self.tiles = tiles
        self._tiles_keep, self._tiles_ptr = _tiles_arg(tiles, zero_mean)
        self._arr = _series_array(self.series)
        self.info, self.trial_offsets = batch_plan(self.series, self.widths, self.ws_budget,
                                                   tiles, zero_mean)
        self.span = max(s.offset + s.n for s in self.series)
        T, nw = self.info.ntrials, len(self.widths)
        self.device = torch.device(device)
        self.ws = _workspace(self.info.workspace_bytes, self.device)
        self._per = torch.empty(max(T, 1), dtype=torch.float64, device=self.device)
        self._fb = torch.empty(max(T, 1), dtype=torch.int32, device=self.device)
        self._snr = torch.empty((max(T, 1), nw), dtype=torch.float32, device=self.device)
        self.periods, self.foldbins, self.snr = self._per[:T], self._fb[:T], self._snr[:T]

    def __call__(self, x, stream=None):
        _dev_tensor(x, "x")
        if x.numel() < self.span:
            raise ValueError("batch buffer is shorter than the series span")
        _check(library().ffa_periodogram_batch_opts(
            _vp(x), _dtype_code(x), ctypes.cast(self._arr, ctypes.c_void_p), len(self.series),
            _vp(self.widths), len(self.widths), self.ws_budget, self._tiles_ptr, _vp(self._per),
            _vp(self._fb), _vp(self._snr), self.periods.numel(), _vp(self.ws), self.ws.numel(),
            _stream_handle(stream)))
        _keep(stream, self.ws, self._per, self._fb, self._snr)
        return self.periods, self.foldbins, self.snr

    def series_result(self, i: int):
        a, b = int(self.trial_offsets[i]), int(self.trial_offsets[i + 1])
        return self.periods[a:b], self.foldbins[a:b], self.snr[a:b]

    def check(self, stream=None):
        check(self.ws, stream)


def periodogram_batch(x, series: Sequence[Series], widths: Sequence[int],
                      ws_budget: int = DEFAULT_BATCH_BUDGET, stream=None):
    """Batched periodograms; returns (periods, foldbins, snr, trial_offsets)."""
    with _on(stream):
        s = BatchSearcher(series, widths, ws_budget, device=x.device)
        per, fb, snr = s(x)
    return per, fb, snr, s.trial_offsets


class SegmentSearcher:
    """Dynamic duty-cycle resolution (Sec. 5.6): one series searched over consecutive
    period segments, each with its own bins range (more bins at longer periods), as one
    batch whose series all point at the same samples.  Widths are shared: each must lie below
    every segment's bmin.  Results of segment k: `segment_result(k)`."""

    def __init__(self, n: int, tsamp: float, segments, widths: Sequence[int],
                 ws_budget: int = DEFAULT_BATCH_BUDGET, device="cuda",
                 tiles: Optional[Tiles] = None, zero_mean: bool = False):
        self.segments = [tuple(s) for s in segments]
        series = [Series(0, int(n), float(tsamp), float(pmin), float(pmax), int(bmin), int(bmax))
                  for pmin, pmax, bmin, bmax in self.segments]
        self.batch = BatchSearcher(series, widths, ws_budget, device, tiles, zero_mean)
        self.n = int(n)

    def __call__(self, x, stream=None):
        if x.numel() != self.n:
            raise ValueError("series length differs from the plan")
        return self.batch(x, stream)

    def segment_result(self, k: int):
        return self.batch.series_result(k)

    @property
    def info(self):
        return self.batch.info


def tile_candidates(auto: Tiles):
    """A small grid around the automatic tile shape `auto` (the effective tiles that a
    plan reports): each size as is or halved, one merge level fewer per top pass."""
    rows = sorted({auto.subtree_rows, max(2, auto.subtree_rows // 2)}, reverse=True)
    levels = sorted({auto.top_levels, max(1, auto.top_levels - 1)}, reverse=True)
    krows = sorted({auto.top_rows, max(1, auto.top_rows // 2)}, reverse=True)
    return [Tiles(r, l, k) for r in rows for l in levels for k in krows]


def tune(make, run, candidates: Sequence[Tiles], repeats: int = 3, stream=None):
    """Times `run(make(tiles))` on the device for every candidate tile shape and returns
    (fastest tiles, [(tiles, ms per call)]).  `make(tiles)` builds a searcher (plans and
    workspace), `run(searcher)` launches one search on the current stream.  Every shape
    gives bit-identical results, so only time decides."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    timings = []
    for t in candidates:
        searcher = make(t)
        run(searcher)  # warm-up: plan tables pinned, caches filled
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(repeats):
            run(searcher)
        e1.record(s)
        e1.synchronize()
        timings.append((t, e0.elapsed_time(e1) / repeats))
        del searcher
    best = min(timings, key=lambda tm: tm[1])[0]
    return best, timings


def tune_periodogram(x, tsamp, pmin, pmax, bmin, bmax, widths, candidates=None, repeats=3):
    """Fastest tile shape for periodograms of series like `x` (see `tune`)."""
    args = (x.numel(), tsamp, pmin, pmax, bmin, bmax, widths)
    if candidates is None:
        candidates = tile_candidates(periodogram_plan(*args).tiles)
    return tune(lambda t: Searcher(*args, device=x.device, tiles=t), lambda s: s(x),
                candidates, repeats)


# Tile classes by transform rows m: the FFA's cost per element grows with log2 m and the
# split between sub-tree and top-pass levels changes with m (Sec. 5.6 cost model), so
# each octave of m may prefer its own tiles.  0: every larger m.
CLASS_M_BOUNDS = (64, 128, 256, 512, 1024, 2048, 4096, 0)


def tile_classes(bounds: Sequence[int] = CLASS_M_BOUNDS, p_max: int = 0) -> Tiles:
    """A class table by m (all classes automatic), the starting point of `tune_classes`."""
    return Tiles(classes=tuple(TileClass(int(b), int(p_max)) for b in bounds))


def class_candidates(eff: TileClass):
    """Tile choices to try for one class whose transforms got the effective tiles `eff`
    (as a plan reports them): sub-tree rows as is, halved or quartered, one merge level
    fewer per top pass, top-pass rows halved or cut to a multiple of 32; 0 keeps the
    automatic value."""
    rows = [0] + [r for r in (eff.subtree_rows // 2, eff.subtree_rows // 4) if r >= 8]
    levels = [0] + ([eff.top_levels - 1] if eff.top_levels > 1 else [])
    # top-pass rows halved, or cut to a multiple of 32 (the S/N scores 32 rows per round)
    krows = [0] + sorted({k for k in (eff.top_rows // 2, 32 * (eff.top_rows // 32))
                          if k >= 8 and k != eff.top_rows}, reverse=True)
    return [dict(subtree_rows=r, top_levels=l, top_rows=k) for r in rows for l in levels
            for k in krows if (r, l, k) != (0, 0, 0)]


def _min_ms(run, searcher, repeats, stream):
    torch = _torch()
    run(searcher)  # warm-up: plan tables pinned, caches filled
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(searcher)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_classes(make, run, plan_tiles, start: Optional[Tiles] = None, repeats: int = 5,
                 min_gain: float = 0.005, stream=None):
    """Per-class tile tuning: for each class of `start` (default `tile_classes()`) in
    turn, times `run(make(tiles))` with each of `class_candidates` for that class (the
    other classes at their best so far) and keeps a choice only if it is faster than the
    current one by more than `min_gain`.  `plan_tiles(tiles)` returns the effective tiles
    that a plan with `tiles` reports (empty classes: all zero; they are skipped).
    Returns (tiles, log) with log = [(class index, fields, min ms of `repeats` calls)];
    every shape gives bit-identical results, so only time decides."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    cur = start if start is not None else tile_classes()
    cur_ms = _min_ms(run, make(cur), repeats, s)
    log = [(-1, {}, cur_ms)]
    for i in range(len(cur.classes)):
        eff = plan_tiles(cur).classes[i]
        if eff.subtree_rows == 0:
            continue  # no transform in this class
        best, best_ms = None, cur_ms
        for f in class_candidates(eff):
            t = cur.with_class(i, **f)
            ms = _min_ms(run, make(t), repeats, s)
            log.append((i, f, ms))
            if ms < best_ms * (1.0 - min_gain):
                best, best_ms = t, ms
        if best is not None:
            cur, cur_ms = best, best_ms
    return cur, log


def tune_periodogram_classes(x, tsamp, pmin, pmax, bmin, bmax, widths, repeats=5):
    """Per-class tiles for periodograms of series like `x` (see `tune_classes`)."""
    args = (x.numel(), tsamp, pmin, pmax, bmin, bmax, widths)
    return tune_classes(lambda t: Searcher(*args, device=x.device, tiles=t), lambda s: s(x),
                        lambda t: periodogram_plan(*args, tiles=t).tiles, repeats=repeats)


def shard_series(costs: Sequence[float], rank: int, world: int):
    """Indices of the series that rank `rank` of `world` searches.

    Series are independent, so ranks split the list with no exchange of data: longest
    first, each to the rank with the least total cost so far (ties to the lower rank).
    Every rank computes the same assignment from the same cost list; the indices come
    back in ascending order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += float(costs[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def plan_cache_clear() -> None:
    """Release every cached plan (only when no call or captured graph still uses one)."""
    _check(library().ffa_plan_cache_clear())


def set_wait_limit_ms(ms: float) -> None:
    """Limit of every device-side wait of a periodogram launch (default 1000 ms); a wait
    that runs out makes the search report FFA_ERR_TIMEOUT (see ffa_set_wait_limit_ms)."""
    _check(library().ffa_set_wait_limit_ms(float(ms)))


def check(ws, stream=None) -> None:
    """Raises FFAError if a device-side check of the last calls on `ws` failed."""
    _check(library().ffa_check(_vp(ws), _stream_handle(stream)))


def checked_status() -> Tuple[bool, int]:
    """(whether the loaded library is the bounds-checked build, the violation bits its
    kernels recorded since the last call; synchronises the device in that build)."""
    c, bits = ctypes.c_int32(), ctypes.c_uint32()
    _check(library().ffa_checked_status(ctypes.byref(c), ctypes.byref(bits)))
    return bool(c.value), int(bits.value)


def launch_count() -> int:
    return int(library().ffa_launch_count())


def kernel_names() -> Tuple[str, ...]:
    L = library()
    return tuple(L.ffa_kernel_name(k).decode() for k in range(L.ffa_kernel_kinds()))


def profile_enable(on: bool = True) -> None:
    _check(library().ffa_profile_enable(1 if on else 0))


def profile_reset() -> None:
    _check(library().ffa_profile_reset())


def profile_query(kind) -> dict:
    L = library()
    if isinstance(kind, str):
        kind = kernel_names().index(kind)
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    b = ctypes.c_double()
    _check(L.ffa_profile_query(kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)))
    return {"launches": n.value, "ms": ms.value, "alg_bytes": b.value}
