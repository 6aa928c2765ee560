"""Pins of the oracle's peak finding (Sec. 5.5, Fig. 6): per width, frequency segments
of dzseg / T, a control point m + k sigma per segment from the median and the IQR
(sigma = IQR / 1.349), a least-squares polynomial in ln(nu), and clustering of the
trials above it.  Checked against hand-computed order statistics, a trend the fit must
reproduce exactly, the N(0, 1) noise level (sigma from the IQR of a normal sample is 1),
the frequency gap that separates clusters, and a pulse injected into a periodogram that
the oracle itself searches."""
import math

import numpy as np
import pytest

import oracle
import synth


def _grid(nseg, per_seg, tobs=100.0, dz=5.0, nu0=0.5):
    """Trial frequencies: per_seg evenly inside each of nseg segments, returned as
    increasing periods (the periodogram's order).  Segments after the first are shifted
    by a fifth of a spacing, so that no trial sits on a segment edge (which starts from
    the lowest frequency)."""
    w = dz / tobs
    nu = np.concatenate([nu0 + (j + (np.arange(per_seg) + 0.5 + (0.2 if j else 0.0)) / per_seg) * w
                         for j in range(nseg)])
    nu = np.sort(nu)[::-1]
    return 1.0 / nu, nu


def test_control_point_order_statistics():
    """Segment values 1..9 (shuffled): median 5, quartiles 3 and 7, so s = 5 + 6 * 4/1.349;
    values 1..4: linear-interpolation quartiles 1.75 and 3.25, median 2.5."""
    tobs, dz = 100.0, 5.0
    P, nu = _grid(2, 9, tobs, dz)
    r = synth.rng(1)
    snr = np.concatenate([r.permutation(np.arange(1.0, 10.0)) for _ in range(2)])
    cn, cs = oracle.segment_controls(nu, snr, tobs, dz, 6.0, 4)
    assert len(cs) == 2
    np.testing.assert_allclose(cs, 5.0 + 6.0 * 4.0 / 1.349, rtol=1e-15)
    # segments start at the lowest trial frequency
    np.testing.assert_allclose(cn, nu.min() + (np.arange(2) + 0.5) * dz / tobs, rtol=1e-15)
    P4, nu4 = _grid(1, 4, tobs, dz)
    cn4, cs4 = oracle.segment_controls(nu4, np.array([4.0, 1.0, 3.0, 2.0]), tobs, dz, 2.0, 4)
    assert cs4[0] == pytest.approx(2.5 + 2.0 * (3.25 - 1.75) / 1.349, rel=1e-15)


def test_small_segments_give_no_control_point():
    tobs, dz = 100.0, 5.0
    P, nu = _grid(3, 9, tobs, dz)
    keep = np.ones(len(nu), bool)
    keep[np.flatnonzero((nu >= 0.55) & (nu < 0.6))[3:]] = False   # segment 1: 3 trials
    cn, _ = oracle.segment_controls(nu[keep], np.zeros(keep.sum()), tobs, dz, 6.0, 4)
    np.testing.assert_allclose(cn, nu.min() + np.array([0.5, 2.5]) * dz / tobs, rtol=1e-14)
    res = oracle.find_peaks(P[keep], np.zeros(keep.sum()), tobs, min_seg=4, degree=2)
    assert res[0].coef is None and len(res[0].peaks) == 0


def test_fit_reproduces_a_quadratic_trend():
    """Control points on an exact quadratic in ln(nu) (constant spread per segment) give
    that quadratic back as the threshold."""
    tobs, dz = 200.0, 5.0
    P, nu = _grid(40, 21, tobs, dz, nu0=0.2)
    width = dz / tobs
    j = np.floor((nu - nu.min()) / width).astype(int)
    cj = nu.min() + (j + 0.5) * width
    a, b, c = 3.0, -1.5, 0.4
    base = a + b * np.log(cj) + c * np.log(cj) ** 2
    spread = np.tile(np.linspace(-1.0, 1.0, 21), 40)   # same values in every segment
    snr = base + spread
    res = oracle.find_peaks(P, snr, tobs, dzseg=dz, nsigma=6.0, min_seg=8)[0]
    q = np.percentile(np.linspace(-1.0, 1.0, 21), [25, 50, 75])
    off = q[1] + 6.0 * (q[2] - q[0]) / 1.349
    np.testing.assert_allclose(res.coef, [c, b, a + off], rtol=1e-9, atol=1e-9)
    assert len(res.peaks) == 0


def test_gaussian_noise_level_and_no_false_peaks():
    """N(0, 1) S/N: control points scatter about 0 + 6 * 1 (the IQR of N(0, 1) is 1.349;
    with 250 trials a segment's m + 6 sigma has a standard error of about 0.45), the fit
    is flat at 6, and there is no peak (P(> 6 sigma) ~ 1e-9 per trial)."""
    tobs = 500.0
    P, nu = _grid(300, 250, tobs, 5.0, nu0=0.1)
    snr = synth.rng(3).standard_normal(len(P))
    res = oracle.find_peaks(P, snr, tobs)[0]
    assert abs(res.ctrl_s.mean() - 6.0) < 0.1
    assert 0.3 < res.ctrl_s.std() < 0.6
    assert np.all(np.abs(res.ctrl_s - 6.0) < 2.0)
    assert np.all(np.abs(res.threshold - 6.0) < 0.4)     # a quadratic fit wanders at the ends
    assert abs(res.threshold.mean() - 6.0) < 0.1
    assert len(res.peaks) == 0


def test_clusters_split_at_the_frequency_gap():
    """Two bumps: trials above threshold closer than clrad / T in frequency form one peak,
    farther apart two; each peak is its brightest member."""
    tobs = 500.0
    P, nu = _grid(100, 250, tobs, 5.0, nu0=0.1)
    snr = synth.rng(4).standard_normal(len(P)) * 0.01
    i0 = 10000
    step = nu[i0] - nu[i0 + 1]                       # trial spacing in frequency
    snr[i0:i0 + 3] = [12.0, 15.0, 11.0]
    far = i0 + int(math.ceil(2.0 / tobs / step)) + 3  # gap of ~2 / T: a second peak
    snr[far] = 9.0
    near = i0 + 2 + int(0.5 / tobs / step)            # gap of ~0.5 / T: same peak
    snr[near] = 20.0
    res = oracle.find_peaks(P, snr, tobs, clrad=1.0)[0]
    np.testing.assert_array_equal(res.peaks, [near, far])
    res = oracle.find_peaks(P, snr, tobs, clrad=0.1)[0]
    np.testing.assert_array_equal(res.peaks, [i0 + 1, near, far])


def test_peak_above_a_rising_trend_is_found():
    """A red-noise-like trend rising towards low frequency: a pulse that sits below the
    trend's largest values but well above its local level is still found (the point of
    Sec. 5.5), and only it."""
    tobs = 500.0
    P, nu = _grid(300, 250, tobs, 5.0, nu0=0.1)
    trend = 2.0 - 3.0 * np.log(nu) + 1.0 * np.log(nu) ** 2
    snr = trend + synth.rng(5).standard_normal(len(P))
    k = len(P) // 3
    assert trend[k] + 9.0 < trend.max()
    snr[k] = trend[k] + 9.0
    res = oracle.find_peaks(P, snr, tobs)[0]
    np.testing.assert_array_equal(res.peaks, [k])


def test_injected_pulse_found_in_an_oracle_periodogram():
    """End to end on the oracle's own periodogram: a 0.77 s pulse train of S/N 14 in
    white noise is the brightest peak at its best width, within 0.2 % of its period."""
    w = synth.custom(2 ** 15, 1e-3, 0.5, 3.0, 40, 44, (1, 2, 4, 8), seed=5,
                     pulses=[synth.Pulse(0.77, 0.05, 14.0, 0.2)])
    pg = oracle.periodogram(w.x, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    tobs = len(w.x) * w.tsamp
    res = oracle.find_peaks(pg.periods, pg.snr, tobs)
    iw = int(np.argmax(pg.snr.max(axis=0)))
    pk = res[iw].peaks
    assert len(pk) >= 1
    best = pk[np.argmax(pg.snr[pk, iw])]
    assert abs(pg.periods[best] / 0.77 - 1.0) < 2e-3
