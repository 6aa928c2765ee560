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

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

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


def pulse_train(n: int, tsamp: float, pulse: Pulse) -> np.ndarray:
    """Gaussian pulse train sampled at t_i = i * tsamp, scaled to unit square sum
    times the amplitude.  Pulse FWHM = duty * period."""
    t = np.arange(n, dtype=np.float64) * tsamp
    ph = np.mod(t / pulse.period - pulse.phase + 0.5, 1.0) - 0.5   # in [-0.5, 0.5)
    sigma = pulse.duty / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    s = np.exp(-0.5 * (ph / sigma) ** 2)
    s /= np.sqrt(np.sum(s * s))
    return pulse.amplitude * s


def make_series(n: int, tsamp: float, seed: int, pulses=()) -> np.ndarray:
    x = white_noise(n, seed)
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


def custom(n: int, tsamp: float, pmin: float, pmax: float, bmin: int, bmax: int,
           widths, seed: int, pulses=()) -> Workload:
    return Workload("custom", make_series(n, tsamp, seed, pulses), tsamp, pmin, pmax,
                    bmin, bmax, tuple(widths), list(pulses))


def small_integer_block(m: int, p: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """m x p float32 block of small integers: every float sum of it is exact."""
    return rng(seed).integers(lo, hi + 1, size=(m, p)).astype(np.float32)


def normal_block(m: int, p: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal((m, p)).astype(np.float32)
