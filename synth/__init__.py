"""Seeded synthetic inputs shaped like the paper's search workloads.

Shared by the tests, the smoke check and the benchmark.  This module holds none of
the search method's arithmetic (no downsampling, folding or matched filtering): it
only draws noise and adds Gaussian pulse trains, so both the CUDA library and the
CPU oracle can be fed the very same arrays.

Noise: numpy's PCG64 generator, standard normal, float64, cast to float32 at the end.
Pulse trains (Sec. 3.1 of the paper): x = a * s + w, with s a periodic train of
Gaussian pulses normalised to unit square sum over the whole series, so that the
amplitude a is the Z-statistic (S/N) of a perfectly matched template.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 2004037010

# Boxcar width trials used by the workloads (bins).  The first set is the paper's
# default width recurrence (Sec. 5.4, f_sp = 1.5) up to 63 bins; the second is the
# same recurrence with f_sp = 1.37, reaching about a quarter of 480 bins.
WIDTHS_11 = (1, 2, 3, 4, 6, 9, 13, 19, 28, 42, 63)
WIDTHS_16 = (1, 2, 3, 4, 5, 6, 8, 10, 13, 17, 23, 31, 42, 57, 78, 106)


@dataclass
class Pulse:
    period: float      # seconds
    duty: float        # FWHM / period
    amplitude: float   # Z-statistic of the full train (unit-square-sum template)
    phase: float = 0.0 # pulse centre at t=0, in units of the period


@dataclass
class Workload:
    name: str
    x: np.ndarray      # float32 time series
    tsamp: float
    pmin: float
    pmax: float
    bmin: int
    bmax: int
    widths: Tuple[int, ...]
    pulses: List[Pulse] = field(default_factory=list)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def white_noise(n: int, seed: int) -> np.ndarray:
    """n samples of N(0, 1) noise in float64."""
    return rng(seed).standard_normal(n)


def red_noise(n: int, tsamp: float, seed: int, f1: float = 1.0) -> np.ndarray:
    """N(0, 1) white noise plus 1/f ("red") noise of the same power at frequency f1 (Hz):
    a Gaussian spectrum shaped by sqrt(f1 / f), no DC term, drawn with numpy's FFT.
    The input that running-median de-reddening (Sec. 5.2) is for."""
    r = rng(seed)
    white = r.standard_normal(n)
    spec = np.fft.rfft(r.standard_normal(n))
    f = np.fft.rfftfreq(n, tsamp)
    shape = np.zeros_like(f)
    shape[1:] = np.sqrt(f1 / f[1:])
    red = np.fft.irfft(spec * shape, n)
    return (white + red).astype(np.float32)


def pulse_train(n: int, tsamp: float, pulse: Pulse) -> np.ndarray:
    """Gaussian pulse train sampled at t_i = i * tsamp, scaled to unit square sum
    times the amplitude.  Pulse FWHM = duty * period."""
    t = np.arange(n, dtype=np.float64) * tsamp
    ph = np.mod(t / pulse.period - pulse.phase + 0.5, 1.0) - 0.5   # in [-0.5, 0.5)
    sigma = pulse.duty / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    s = np.exp(-0.5 * (ph / sigma) ** 2)
    norm = np.sqrt(np.sum(s * s))
    if not norm > 0.0:  # no sample near any pulse (a very narrow, sparse train): no signal
        return np.zeros(n, np.float64)
    return pulse.amplitude * (s / norm)


def make_series(n: int, tsamp: float, seed: int, pulses=(), red: bool = False) -> np.ndarray:
    """N(0, 1) noise (plus 1/f red noise if `red`) and the pulse trains, float32."""
    x = red_noise(n, tsamp, seed).astype(np.float64) if red else white_noise(n, seed)
    for p in pulses:
        x = x + pulse_train(n, tsamp, p)
    return x.astype(np.float32)


def plain_small(seed: Optional[int] = None) -> Workload:
    """2^18 samples at 1 ms, one pulse train (P=2.345 s, FWHM 2%, S/N 15);
    periods 1-10 s, bins 240-260, 11 widths."""
    seed = SEED_BASE + 1 if seed is None else seed
    ph = rng(seed ^ 0x5A5A).uniform(0.0, 1.0)
    pulses = [Pulse(2.345, 0.02, 15.0, ph)]
    n, tsamp = 262144, 1e-3
    return Workload("plain_fp32_2^18_1ms", make_series(n, tsamp, seed, pulses), tsamp,
                    1.0, 10.0, 240, 260, WIDTHS_11, pulses)


def survey(seed: Optional[int] = None) -> Workload:
    """2^23 samples at 64 us (the paper's benchmark shape), three pulse trains;
    periods 0.2-20 s, bins 240-260, 11 widths."""
    seed = SEED_BASE + 2 if seed is None else seed
    r = rng(seed ^ 0x5A5A)
    pulses = [Pulse(0.31, 0.01, 8.0, r.uniform()),
              Pulse(1.7, 0.03, 14.0, r.uniform()),
              Pulse(7.9, 0.05, 20.0, r.uniform())]
    n, tsamp = 2 ** 23, 64e-6
    return Workload("survey_fp32_2^23_64us", make_series(n, tsamp, seed, pulses), tsamp,
                    0.2, 20.0, 240, 260, WIDTHS_11, pulses)


# Period segments of the survey series for dynamic duty-cycle resolution (Sec. 5.6):
# about 100 bins down to 0.1 s, more bins at longer periods, 1000-1100 from 2 s to 20 s.
SURVEY_SEGMENTS = ((0.1, 0.5, 100, 110), (0.5, 2.0, 400, 440), (2.0, 20.0, 1000, 1100))


def survey_segments(seed: Optional[int] = None) -> BatchWorkload:
    """The survey series searched over SURVEY_SEGMENTS: one batch whose three series
    are the same samples, each with its own period and bins range; 11 widths (all
    below the smallest bmin)."""
    w = survey(seed)
    series = [SeriesParams(0, w.n, w.tsamp, pmin, pmax, bmin, bmax, list(w.pulses))
              for pmin, pmax, bmin, bmax in SURVEY_SEGMENTS]
    return BatchWorkload("survey_segments_2^23_64us", w.x, series, WIDTHS_11, shared=True)


def custom(n: int, tsamp: float, pmin: float, pmax: float, bmin: int, bmax: int,
           widths, seed: int, pulses=()) -> Workload:
    return Workload("custom", make_series(n, tsamp, seed, pulses), tsamp, pmin, pmax,
                    bmin, bmax, tuple(widths), list(pulses))


def small_integer_block(m: int, p: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """m x p float32 block of small integers: every float sum of it is exact."""
    return rng(seed).integers(lo, hi + 1, size=(m, p)).astype(np.float32)


def normal_block(m: int, p: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal((m, p)).astype(np.float32)


# ---------------------------------------------------------------------------------
# Batches of series (many dedispersed time series searched together)

@dataclass
class SeriesParams:
    offset: int        # first sample in the batch buffer
    n: int
    tsamp: float
    pmin: float
    pmax: float
    bmin: int
    bmax: int
    pulses: List[Pulse] = field(default_factory=list)
    red: bool = False  # N(0,1) plus 1/f red noise (to be de-reddened before the search)


@dataclass
class BatchWorkload:
    name: str
    x: np.ndarray                   # float32, all series one after another
    series: List[SeriesParams]
    widths: Tuple[int, ...]
    shared: bool = False            # all "series" are period segments of one series

    @property
    def n(self) -> int:
        """Input samples searched: the series' total, or the one series' length."""
        if self.shared:
            return int(max(s.offset + s.n for s in self.series))
        return int(sum(s.n for s in self.series))

    def series_x(self, i: int) -> np.ndarray:
        s = self.series[i]
        return self.x[s.offset:s.offset + s.n]


def _fill_batch(series: Sequence[SeriesParams], seeds: Sequence[int], threads: int) -> np.ndarray:
    """Concatenated float32 buffer of the series' noise + pulses, drawn in parallel
    (each series from its own seeded generator, so the result does not depend on
    the number of threads)."""
    total = max((s.offset + s.n for s in series), default=0)
    x = np.zeros(total, np.float32)

    def one(k):
        s = series[k]
        x[s.offset:s.offset + s.n] = make_series(s.n, s.tsamp, seeds[k], s.pulses, s.red)

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        list(ex.map(one, range(len(series))))
    return x


def batch_uneven(nseries: int = 256, nmin: int = 2 ** 20, nmax: int = 2 ** 23,
                 seed: Optional[int] = None, threads: int = 16) -> BatchWorkload:
    """Series of uneven length n ~ U[nmin, nmax] at 64 us, each N(0,1) noise plus one
    Gaussian pulse train, each with its own period range inside 0.1-30 s: two
    log-uniform draws in [0.1, 30] s, sorted, with Pmax raised to at least 2 Pmin
    (capped at 30 s); bins 240-260, 11 widths.  Series are stored back to back in one
    buffer."""
    seed = SEED_BASE + 3 if seed is None else seed
    r = rng(seed)
    tsamp = 64e-6
    series, seeds, off = [], [], 0
    for i in range(nseries):
        n = int(r.integers(nmin, nmax + 1))
        lo, hi = sorted(float(v) for v in np.exp(r.uniform(np.log(0.1), np.log(30.0), 2)))
        pmin = lo
        pmax = min(30.0, max(hi, 2.0 * lo))
        per = float(np.exp(r.uniform(np.log(pmin), np.log(pmax))))
        pulse = Pulse(per, float(r.uniform(0.01, 0.05)), float(r.uniform(8.0, 20.0)),
                      float(r.uniform()))
        series.append(SeriesParams(off, n, tsamp, pmin, pmax, 240, 260, [pulse]))
        seeds.append(seed * 7919 + i)
        off += n
    return BatchWorkload("batch_uneven_%dx2^20-2^23_64us" % nseries if (nmin, nmax) ==
                         (2 ** 20, 2 ** 23) else "batch_uneven_%d" % nseries,
                         _fill_batch(series, seeds, threads), series, WIDTHS_11)


def batch_int8_stress(nseries: int = 1024, n: int = 2 ** 21, seed: Optional[int] = None,
                      threads: int = 16) -> BatchWorkload:
    """nseries series of n samples at 64 us, N(0,1) noise plus 1/f red noise
    (`red_noise`), one Gaussian pulse train in every tenth series; periods 0.1-10 s,
    bins 480-520, the 16-width set.  Meant to be de-reddened by a running median of
    about 1 s (Sec. 5.2), normalised and stored as int8 before the search, all on the
    device by the library (`deredden_normalise_batch` in the benchmark and tests)."""
    seed = SEED_BASE + 5 if seed is None else seed
    r = rng(seed)
    tsamp = 64e-6
    series, seeds = [], []
    for i in range(nseries):
        pulses = []
        if i % 10 == 0:
            pulses = [Pulse(float(np.exp(r.uniform(np.log(0.1), np.log(10.0)))),
                            float(r.uniform(0.01, 0.05)), float(r.uniform(8.0, 20.0)),
                            float(r.uniform()))]
        series.append(SeriesParams(i * n, n, tsamp, 0.1, 10.0, 480, 520, pulses, red=True))
        seeds.append(seed * 7919 + i)
    return BatchWorkload("batch_int8_%dx2^21_64us" % nseries, _fill_batch(series, seeds, threads),
                         series, WIDTHS_16)


# Running-median window of the batch_int8 stress series (Sec. 5.2: about 1 s): odd samples
DEREDDEN_SECONDS = 1.0
