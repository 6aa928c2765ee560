"""CPU oracle of the FFA periodogram (Morello et al. 2020) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports, links or
calls it, and it shares no code with the CUDA library.

The arithmetic lives in ``ffa_oracle.c`` (plain C, FP64 except for the FP32
instantiation of the FFA, which fixes the exact sequence of float additions of the
paper's recursion).  This module only compiles it with gcc and marshals numpy
arrays through ctypes.

Paper passages followed (sections and equations of the paper):
  * plan ............ Sec. 5.3 (pseudo-octaves), Sec. 5.6 (initial tau = Pmin/bmin)
  * downsample ...... Sec. 5.3, App. A.4 (overlap-weighted real-factor windows)
  * ffa ............. Sec. 2.2, Eq. ffa_merge_rule (depth-first, m_h = floor(m/2))
  * trial periods ... Sec. 2.3 (P_s = p^2 tau / (p - s/(m-1)); redundant rows)
  * boxcar S/N ...... Sec. 5.4, Sec. 3.3 (Z = x.s, unit square sum), App. A.3; the
                      zero-mean boxcar: Sec. 3.3 and 3.5 (another unit-square-sum template)
  * normalise ....... Sec. 3.1, Sec. 5.2 (zero mean, unit std from the whole series)
  * running median .. Sec. 5.2 (de-reddening: subtract a running median, odd window,
                      the series extended by its end samples)
  * peak finding .... Sec. 5.5, Fig. 6 (per width: robust median/IQR threshold per
                      frequency segment, polynomial fit in log frequency, clustering)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffa_oracle.c")
_LIB = os.path.join(_HERE, "libffa_oracle.so")
_lib = None

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction into FMA, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ffa_oracle_api.h"))
    ):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"],
            cwd=_HERE,
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.oracle_plan.restype = _int
    lib.oracle_plan.argtypes = [_i64, _dbl, _dbl, _dbl, _int, _int, _int, _p, _p, _int,
                                _p, _p, _p, _p, _p, _p, _p, _p]
    lib.oracle_downsampled_length.restype = _i64
    lib.oracle_downsampled_length.argtypes = [_i64, _dbl]
    lib.oracle_downsample.restype = _int
    lib.oracle_downsample.argtypes = [_p, _i64, _dbl, _p, _i64]
    lib.oracle_downsampled_variance.restype = _dbl
    lib.oracle_downsampled_variance.argtypes = [_dbl]
    lib.oracle_ffa_split.restype = None
    lib.oracle_ffa_split.argtypes = [_i64, _i64, _p, _p, _p]
    lib.oracle_ffa_f64.restype = _int
    lib.oracle_ffa_f64.argtypes = [_p, _i64, _i64, _p]
    lib.oracle_ffa_f32.restype = _int
    lib.oracle_ffa_f32.argtypes = [_p, _i64, _i64, _p]
    lib.oracle_trial_period.restype = _dbl
    lib.oracle_trial_period.argtypes = [_dbl, _i64, _i64, _i64]
    lib.oracle_boxcar_snr.restype = _int
    lib.oracle_boxcar_snr.argtypes = [_p, _i64, _i64, _p, _int, _dbl, _p]
    lib.oracle_boxcar_snr_kind.restype = _int
    lib.oracle_boxcar_snr_kind.argtypes = [_p, _i64, _i64, _p, _int, _dbl, _int, _p]
    lib.oracle_periodogram_kind.restype = _i64
    lib.oracle_periodogram_kind.argtypes = [_p, _i64, _dbl, _dbl, _dbl, _int, _int, _p, _int,
                                            _int, _p, _p, _p, _p, _i64]
    lib.oracle_running_median.restype = _int
    lib.oracle_running_median.argtypes = [_p, _i64, _i64, _p]
    lib.oracle_running_median_at.restype = _int
    lib.oracle_running_median_at.argtypes = [_p, _i64, _i64, _p, _i64, _p]
    lib.oracle_normalise.restype = _int
    lib.oracle_normalise.argtypes = [_p, _i64, _p, _p, _p]
    lib.oracle_periodogram.restype = _i64
    lib.oracle_periodogram.argtypes = [_p, _i64, _dbl, _dbl, _dbl, _int, _int, _p, _int,
                                       _p, _p, _p, _p, _i64]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Plan:
    """Search plan: octaves (factor, length) and transforms in (octave, p) order."""
    oct_factor: np.ndarray     # float64 [n_octaves]
    oct_len: np.ndarray        # int64   [n_octaves]
    tr_octave: np.ndarray      # int32   [n_transforms]
    tr_p: np.ndarray           # int32
    tr_m: np.ndarray           # int64
    tr_kept: np.ndarray        # int64
    tr_first_trial: np.ndarray # int64
    n_trials: int

    @property
    def n_octaves(self) -> int:
        return len(self.oct_factor)

    @property
    def n_transforms(self) -> int:
        return len(self.tr_p)


def plan(n, tsamp, pmin, pmax, bmin, bmax) -> Plan:
    """Sec. 5.3 search plan.  Raises ValueError on invalid parameters."""
    lib = _load()
    no = ctypes.c_int(0)
    nt = ctypes.c_int(0)
    ntr = ctypes.c_int64(0)
    z = np.zeros(1)
    rc = lib.oracle_plan(n, tsamp, pmin, pmax, bmin, bmax, 0, _ptr(z), _ptr(z), 0,
                         _ptr(z), _ptr(z), _ptr(z), _ptr(z), _ptr(z),
                         ctypes.byref(no), ctypes.byref(nt), ctypes.byref(ntr))
    if rc != 0:
        raise ValueError("invalid search parameters")
    O, T = no.value, nt.value
    of = np.zeros(O, np.float64)
    ol = np.zeros(O, np.int64)
    to = np.zeros(T, np.int32)
    tp = np.zeros(T, np.int32)
    tm = np.zeros(T, np.int64)
    tk = np.zeros(T, np.int64)
    tf = np.zeros(T, np.int64)
    lib.oracle_plan(n, tsamp, pmin, pmax, bmin, bmax, O, _ptr(of), _ptr(ol), T,
                    _ptr(to), _ptr(tp), _ptr(tm), _ptr(tk), _ptr(tf),
                    ctypes.byref(no), ctypes.byref(nt), ctypes.byref(ntr))
    return Plan(of, ol, to, tp, tm, tk, tf, int(ntr.value))


def downsampled_length(n: int, f: float) -> int:
    return int(_load().oracle_downsampled_length(n, f))


def downsample(x: np.ndarray, f: float) -> np.ndarray:
    """App. A.4 downsampling of a float32 series by real factor f >= 1 (FP64 out)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    nout = lib.oracle_downsampled_length(len(x), f)
    if nout < 0:
        raise ValueError("invalid downsampling factor")
    out = np.zeros(nout, np.float64)
    if lib.oracle_downsample(_ptr(x), len(x), f, _ptr(out), nout) != 0:
        raise ValueError("downsample failed")
    return out


def downsampled_variance(f: float) -> float:
    return float(_load().oracle_downsampled_variance(f))


def ffa_split(m: int, s: int):
    """(i, j, b) of the merge rule for output row s of an m-row transform."""
    i, j, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _load().oracle_ffa_split(m, s, ctypes.byref(i), ctypes.byref(j), ctypes.byref(b))
    return i.value, j.value, b.value


def ffa(block: np.ndarray) -> np.ndarray:
    """Folding transform of an m x p block by the depth-first FFA (Sec. 2.2).

    float32 input -> float32 output with the paper's exact sequence of float adds;
    float64 input -> float64 output.
    """
    lib = _load()
    if block.ndim != 2:
        raise ValueError("block must be 2-D")
    m, p = block.shape
    if block.dtype == np.float32:
        a = np.ascontiguousarray(block)
        out = np.empty_like(a)
        rc = lib.oracle_ffa_f32(_ptr(a), m, p, _ptr(out))
    else:
        a = np.ascontiguousarray(block, dtype=np.float64)
        out = np.empty_like(a)
        rc = lib.oracle_ffa_f64(_ptr(a), m, p, _ptr(out))
    if rc != 0:
        raise ValueError("invalid FFA shape")
    return out


def trial_period(tau: float, p: int, m: int, s: int) -> float:
    return float(_load().oracle_trial_period(tau, p, m, s))


def boxcar_snr(prof: np.ndarray, widths, stdnoise: float, zero_mean: bool = False) -> np.ndarray:
    """Boxcar S/N of every row of a profile array (Sec. 5.4), FP64, direct sums.
    zero_mean: the zero-sum, unit-square-sum boxcar instead of the plain one."""
    lib = _load()
    P = np.ascontiguousarray(prof, dtype=np.float64)
    if P.ndim == 1:
        P = P[None, :]
    rows, p = P.shape
    w = np.ascontiguousarray(widths, dtype=np.int32)
    out = np.zeros((rows, len(w)), np.float64)
    if lib.oracle_boxcar_snr_kind(_ptr(P), rows, p, _ptr(w), len(w), stdnoise,
                                  1 if zero_mean else 0, _ptr(out)) != 0:
        raise ValueError("invalid boxcar arguments")
    return out


def normalise(x: np.ndarray):
    """Sec. 3.1 / 5.2: (mean, std, (x - mean) / std) of a float32 series, FP64."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    mean, std = ctypes.c_double(), ctypes.c_double()
    out = np.zeros(len(x), np.float64)
    if lib.oracle_normalise(_ptr(x), len(x), ctypes.byref(mean), ctypes.byref(std), _ptr(out)) != 0:
        raise ValueError("empty series")
    return mean.value, std.value, out


def running_median(x: np.ndarray, width: int, at=None) -> np.ndarray:
    """Sec. 5.2 running median of a float32 series over an odd window of ``width``
    samples centred on each sample, the series extended by its end samples.
    ``at``: optional sample indices; only the medians there are computed."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    if at is None:
        out = np.zeros(len(x), np.float32)
        rc = lib.oracle_running_median(_ptr(x), len(x), int(width), _ptr(out))
    else:
        idx = np.ascontiguousarray(at, dtype=np.int64)
        out = np.zeros(len(idx), np.float32)
        rc = lib.oracle_running_median_at(_ptr(x), len(x), int(width), _ptr(idx), len(idx),
                                          _ptr(out))
    if rc != 0:
        raise ValueError("invalid running-median arguments (empty series, even width, "
                         "or index out of range)")
    return out


def deredden(x: np.ndarray, width: int) -> np.ndarray:
    """Sec. 5.2 de-reddening: the series minus its running median, in float32 (one
    rounding of the exact difference, as IEEE single subtraction gives)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    return x - running_median(x, width)


@dataclass
class Periodogram:
    periods: np.ndarray   # float64 [ntrials]
    foldbins: np.ndarray  # int32   [ntrials]
    snr: np.ndarray       # float64 [ntrials, nw]


def periodogram(x, tsamp, pmin, pmax, bmin, bmax, widths, select=None,
                zero_mean: bool = False) -> Periodogram:
    """Sec. 5.3 periodogram of a float32 series, FP64 throughout.

    ``select``: optional boolean mask over the plan's transforms; only those are
    computed and their trials are returned compactly in plan order.
    ``zero_mean``: score with the zero-mean boxcar (see boxcar_snr).
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    pl = plan(len(x), tsamp, pmin, pmax, bmin, bmax)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    if select is None:
        cap = pl.n_trials
        sel_ptr = None
    else:
        sel = np.ascontiguousarray(select, dtype=np.uint8)
        if len(sel) != pl.n_transforms:
            raise ValueError("select mask has the wrong length")
        cap = int(pl.tr_kept[sel.astype(bool)].sum())
        sel_ptr = _ptr(sel)
    periods = np.zeros(cap, np.float64)
    fb = np.zeros(cap, np.int32)
    snr = np.zeros((cap, len(w)), np.float64)
    got = lib.oracle_periodogram_kind(_ptr(x), len(x), tsamp, pmin, pmax, bmin, bmax, _ptr(w),
                                      len(w), 1 if zero_mean else 0, sel_ptr, _ptr(periods),
                                      _ptr(fb), _ptr(snr), cap)
    if got != cap:
        raise ValueError("oracle periodogram failed (%d)" % got)
    return Periodogram(periods, fb, snr)


# ----------------------------------------------------------------------------------
# Peak finding (Sec. 5.5, Fig. 6).  Written with numpy steps (a percentile, a
# least-squares polynomial fit, a sort) in the paper's order.  Readings where the paper
# leaves a choice:
#   - trial frequencies nu = 1 / P; segments of width dzseg / T start at the lowest
#     trial frequency; segment j holds floor((nu - nu_lo) / width) == j (the highest
#     frequency falls in the last segment); its control frequency is its centre;
#   - median and quartiles are the linear-interpolation percentiles 50, 25 and 75
#     (virtual index q (c - 1)); sigma = IQR / 1.349; s = median + nsigma * sigma;
#   - segments with fewer than min_seg trials give no control point; a width with fewer
#     than degree + 1 control points has no threshold and no peaks;
#   - the threshold is the least-squares polynomial of the given degree in the natural
#     log of frequency; a trial is selected when its S/N is strictly above it;
#   - selected trials are taken in order of decreasing frequency; a new peak starts
#     where the frequency gap to the previous selected trial exceeds clrad / T; a peak
#     is its brightest member (the lowest trial index among equal S/N).
# ----------------------------------------------------------------------------------
PEAK_DEFAULTS = dict(dzseg=5.0, nsigma=6.0, degree=2, clrad=1.0, min_seg=8)


@dataclass
class PeakWidth:
    ctrl_nu: np.ndarray      # control-point frequencies (Hz)
    ctrl_s: np.ndarray       # control-point thresholds m + k sigma
    coef: Optional[np.ndarray]  # polynomial in ln(nu), highest power first (np.polyval)
    threshold: Optional[np.ndarray]  # per trial, or None
    peaks: np.ndarray        # trial indices of the peaks, in order of increasing period


def segment_controls(nu: np.ndarray, snr_w: np.ndarray, tobs: float, dzseg: float,
                     nsigma: float, min_seg: int):
    """Control points (nu_j, s_j) of one width's periodogram (Sec. 5.5): frequency
    segments of dzseg / T, robust median and IQR-based sigma in each."""
    width = dzseg / tobs
    lo, hi = nu.min(), nu.max()
    nseg = max(1, int(math.ceil((hi - lo) / width)))
    j = np.minimum(np.floor((nu - lo) / width).astype(np.int64), nseg - 1)
    cn, cs = [], []
    for k in range(nseg):
        v = snr_w[j == k].astype(np.float64)
        if len(v) < min_seg:
            continue
        q25, q50, q75 = np.percentile(v, [25.0, 50.0, 75.0], method="linear")
        cn.append(lo + (k + 0.5) * width)
        cs.append(q50 + nsigma * ((q75 - q25) / 1.349))
    return np.array(cn), np.array(cs)


def find_peaks(periods: np.ndarray, snr: np.ndarray, tobs: float, **opts):
    """Sec. 5.5 peak detection on a two-dimensional periodogram (trials x widths), each
    width separately.  Returns one PeakWidth per width."""
    o = dict(PEAK_DEFAULTS)
    o.update(opts)
    P = np.asarray(periods, dtype=np.float64)
    S = np.asarray(snr)
    if S.ndim == 1:
        S = S[:, None]
    nu = 1.0 / P
    out = []
    for iw in range(S.shape[1]):
        sw = S[:, iw].astype(np.float64)
        cn, cs = segment_controls(nu, sw, tobs, o["dzseg"], o["nsigma"], o["min_seg"])
        if len(cn) < o["degree"] + 1:
            out.append(PeakWidth(cn, cs, None, None, np.zeros(0, np.int64)))
            continue
        coef = np.polyfit(np.log(cn), cs, o["degree"])
        thr = np.polyval(coef, np.log(nu))
        sel = np.flatnonzero(sw > thr)
        order = sel[np.argsort(-nu[sel], kind="stable")]   # decreasing frequency
        peaks = []
        gap = o["clrad"] / tobs
        start = 0
        for e in range(1, len(order) + 1):
            if e == len(order) or nu[order[e - 1]] - nu[order[e]] > gap:
                members = order[start:e]
                best = members[np.lexsort((members, -sw[members]))[0]]
                peaks.append(best)
                start = e
        out.append(PeakWidth(cn, cs, coef, thr, np.array(peaks, np.int64)))
    return out
