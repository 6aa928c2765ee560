"""Checks of the seeded input generators (no method arithmetic lives there): the red
noise has the 1/f spectrum it is meant to have on top of unit white noise, the period
segments of the survey series share one series' samples, and draws are reproducible."""
import numpy as np

import synth


def test_red_noise_spectrum():
    """Power of N(0,1) + 1/f noise: band means follow 1 + (1 Hz)/f, flat at the white
    level far above 1 Hz, twice it at 1 Hz, ten times the white level near 0.1 Hz
    (a missing square root in the spectral shape would give 1/f^2)."""
    n, tsamp = 2 ** 20, 1e-3
    x = synth.red_noise(n, tsamp, seed=3).astype(np.float64)
    f = np.fft.rfftfreq(n, tsamp)
    P = np.abs(np.fft.rfft(x)) ** 2 / n          # white N(0,1): mean 1 per bin
    for lo, hi, tol in ((0.01, 0.1, 0.25), (0.1, 1.0, 0.1), (0.9, 1.1, 0.15),
                        (10.0, 20.0, 0.05), (200.0, 400.0, 0.02)):
        sel = (f >= lo) & (f < hi)
        assert abs(P[sel].mean() / (1.0 + 1.0 / f[sel]).mean() - 1.0) < tol, (lo, hi)


def test_red_noise_is_reproducible():
    a = synth.red_noise(4096, 1e-3, seed=7)
    b = synth.red_noise(4096, 1e-3, seed=7)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, synth.red_noise(4096, 1e-3, seed=8))


def test_survey_segments_share_the_series():
    b = synth.survey_segments()
    w = synth.survey()
    assert b.shared and b.n == w.n == len(b.x)
    np.testing.assert_array_equal(b.x, w.x)
    for s, (pmin, pmax, bmin, bmax) in zip(b.series, synth.SURVEY_SEGMENTS):
        assert (s.offset, s.n, s.pmin, s.pmax, s.bmin, s.bmax) == (0, w.n, pmin, pmax, bmin, bmax)
        assert max(b.widths) < bmin
    # consecutive, non-overlapping period ranges covering 0.1-20 s
    assert [s.pmax for s in b.series[:-1]] == [s.pmin for s in b.series[1:]]
