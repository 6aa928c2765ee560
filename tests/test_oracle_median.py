"""Pins of the oracle's running median (Sec. 5.2: the low-frequency noise is removed by
subtracting a running median before normalisation).  Reading: an odd window of
w = 2h + 1 samples centred on each sample, the series extended at both ends by its end
samples.  Under that reading the running median is scipy.ndimage.median_filter with
mode="nearest"; it also equals a brute-force median of the explicitly padded window,
reproduces any non-decreasing series, commutes with negation and exact shifts, and
leaves intact a constant impulse narrower than half the window (the filter property
that Sec. 5.2 relies on), while an impulse of h + 1 samples is not left intact."""
import statistics

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth


@pytest.mark.parametrize("n,w", [(1, 1), (1, 5), (7, 1), (7, 3), (7, 15), (100, 9),
                                 (1000, 101), (4097, 255), (3000, 2999), (50, 999)])
def test_equals_library_median_filter(n, w):
    x = synth.rng(n + w).standard_normal(n).astype(np.float32)
    got = oracle.running_median(x, w)
    ref = ndimage.median_filter(x, size=w, mode="nearest")
    np.testing.assert_array_equal(got, ref)


def test_ties_and_repeated_values():
    """Integer-valued samples with many ties: still the library's median filter."""
    x = synth.rng(3).integers(-3, 4, 2000).astype(np.float32)
    for w in (5, 31, 333):
        np.testing.assert_array_equal(oracle.running_median(x, w),
                                      ndimage.median_filter(x, size=w, mode="nearest"))


@pytest.mark.parametrize("n,w", [(1, 3), (5, 3), (6, 7), (9, 5), (12, 11)])
def test_brute_force_tiny(n, w):
    x = synth.rng(10 * n + w).standard_normal(n).astype(np.float32)
    h = w // 2
    ref = [statistics.median([x[min(max(i + j, 0), n - 1)] for j in range(-h, h + 1)])
           for i in range(n)]
    np.testing.assert_array_equal(oracle.running_median(x, w), np.array(ref, np.float32))


def test_monotone_series_is_its_own_median():
    """Every window of a non-decreasing series (end-extended) is sorted, so its middle
    element is the centre sample: the de-reddened series is exactly zero."""
    x = np.sort(synth.rng(1).standard_normal(5000)).astype(np.float32)
    x[1000:1200] = x[1000]      # flat stretches too
    for w in (1, 3, 101, 9999):
        np.testing.assert_array_equal(oracle.running_median(x, w), x)
        assert not oracle.deredden(x, w).any()


def test_negation_and_shift():
    x = synth.rng(2).integers(-1000, 1000, 3000).astype(np.float32)
    w = 77
    m = oracle.running_median(x, w)
    np.testing.assert_array_equal(oracle.running_median(-x, w), -m)
    np.testing.assert_array_equal(oracle.running_median(x + 4096, w), m + 4096)


@pytest.mark.parametrize("h", [1, 5, 50])
def test_narrow_impulse_left_intact(h):
    """A constant impulse of at most h samples (less than half of w = 2h + 1) on a
    constant baseline never holds the middle of a window, so subtracting the running
    median returns the impulse exactly; an impulse of h + 1 samples does reach it."""
    w = 2 * h + 1
    n = 20 * w
    base = np.full(n, 3.25, np.float32)
    for L, start in ((h, 7 * w), (1, 1), (h, n - h - 1), (h, 2)):
        x = base.copy()
        x[start:start + L] += 2.5
        y = oracle.deredden(x, w)
        np.testing.assert_array_equal(y, x - base)
    x = base.copy()
    x[7 * w:7 * w + h + 1] += 2.5
    y = oracle.deredden(x, w)
    assert y[7 * w + h // 2] == 0.0


def test_end_samples_extend_the_series():
    """The reading at the ends: the window of sample 0 holds h copies of x[0], so a
    one-sample impulse on x[0] fills h + 1 of its w places and is taken as the median
    (a mirrored extension would not repeat x[0], and a truncated window would have an
    even length)."""
    for h in (1, 4):
        w = 2 * h + 1
        x = np.zeros(10 * w, np.float32)
        x[0] = 1.0
        x[-1] = -1.0
        m = oracle.running_median(x, w)
        assert m[0] == 1.0 and m[-1] == -1.0
        assert not m[1:-1].any()


def test_sampled_equals_full():
    x = synth.rng(4).standard_normal(3001).astype(np.float32)
    at = np.array([0, 1, 17, 1500, 2999, 3000])
    np.testing.assert_array_equal(oracle.running_median(x, 41, at=at),
                                  oracle.running_median(x, 41)[at])


def test_rejects():
    x = np.zeros(10, np.float32)
    for bad in (0, 2, 10, -3):
        with pytest.raises(ValueError):
            oracle.running_median(x, bad)
    with pytest.raises(ValueError):
        oracle.running_median(np.zeros(0, np.float32), 3)
    with pytest.raises(ValueError):
        oracle.running_median(x, 3, at=[10])
