"""Pins of the oracle's boxcar S/N (Sec. 3.3, Sec. 5.4, App. A.3): it equals the
Z-statistic x.s of an explicit unit-square-sum template, the prefix-sum identity of
Sec. 5.4, the closed-form boxcar efficiency on a Gaussian pulse (0.943 / 0.930 /
0.901), N(0, 1) under pure noise, and the Cauchy-Schwarz bound.  The zero-mean boxcar
(Sec. 3.3 and 3.5: another unit-square-sum template) equals an FFT circular correlation
with the explicit template vector, ignores a constant offset, and is N(0, 1) at a fixed
phase under pure noise."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
import synth


def test_prefix_sum_identity():
    """C_k = S_{k+w} - S_k with S the exclusive prefix sum of two concatenated
    repeats of the profile (Sec. 5.4)."""
    rng = synth.rng(5)
    p = 37
    prof = rng.standard_normal((6, p))
    widths = [1, 2, 5, 13, 36]
    got = oracle.boxcar_snr(prof, widths, 1.0)
    for r in range(prof.shape[0]):
        S = np.concatenate([[0.0], np.cumsum(np.concatenate([prof[r], prof[r]]))])
        for iw, w in enumerate(widths):
            C = S[np.arange(p) + w] - S[np.arange(p)]
            assert got[r, iw] == pytest.approx(C.max() / math.sqrt(w), abs=1e-12)


@pytest.mark.parametrize("w", [1, 3, 8])
def test_equals_z_statistic_of_explicit_template(w):
    """With no downsampling, S/N at width w is max over phase of x.s, where s is a
    boxcar of w samples per period, repeated m times, unit square sum (Sec. 3.3-3.4)."""
    m, p = 16, 23
    x = synth.white_noise(m * p, seed=w).astype(np.float32)
    F = oracle.ffa(x.reshape(m, p).astype(np.float64))
    snr0 = oracle.boxcar_snr(F[0], [w], math.sqrt(m * 1.0))[0, 0]
    best = -np.inf
    for k in range(p):
        s = np.zeros(m * p)
        for i in range(m):
            for q in range(w):
                s[i * p + (k + q) % p] = 1.0
        s /= np.linalg.norm(s)
        best = max(best, float(x.astype(np.float64) @ s))
    assert snr0 == pytest.approx(best, abs=1e-10)


def gaussian_profile(p, sigma_bins):
    x = np.arange(p) - p / 2
    g = np.exp(-0.5 * (x / sigma_bins) ** 2)
    return g / np.linalg.norm(g)


def efficiency(u):
    return (math.pi / u ** 2) ** 0.25 * erf(u / math.sqrt(2))


def test_boxcar_efficiency_closed_form(paper_values):
    """App. A.3: a well-resolved unit-square-sum Gaussian scored by a boxcar of
    half-width u sigma gives E(u) = (pi/u^2)^(1/4) erf(u/sqrt2)."""
    g = paper_values["boxcar_efficiency"]
    sigma = 100.0
    prof = gaussian_profile(4000, sigma)
    u_star = g["u_star"]
    us = [u_star / math.sqrt(2), 0.8, u_star, 2.0, u_star * math.sqrt(2)]
    widths = [int(round(2 * u * sigma)) for u in us]
    got = oracle.boxcar_snr(prof, widths, 1.0)[0]
    for w, e in zip(widths, got):
        assert e == pytest.approx(efficiency(w / (2 * sigma)), abs=2e-3)
    # printed values: peak 0.943 at u* = 1.40, worst 0.901 at u* sqrt(2)
    assert got[2] == pytest.approx(g["e_max"], abs=1.5e-3)
    assert got[4] == pytest.approx(g["e_worst"], abs=1.5e-3)
    # w* = 2.80 sigma = 1.19 FWHM
    fwhm = 2 * math.sqrt(2 * math.log(2))
    assert g["w_star_over_sigma"] / fwhm == pytest.approx(g["w_star_over_fwhm"], abs=6e-3)


def test_average_efficiency_over_doubling_grid(paper_values):
    """App. A.3: the mean of E over [u*/sqrt2, u* sqrt2] is 0.930; evaluated here
    with the oracle on Gaussians of many widths against one boxcar."""
    g = paper_values["boxcar_efficiency"]
    w = 140
    vals = []
    for u in np.linspace(g["u_star"] / math.sqrt(2), g["u_star"] * math.sqrt(2), 41):
        sigma = w / (2 * u)
        vals.append(oracle.boxcar_snr(gaussian_profile(3000, sigma), [w], 1.0)[0, 0])
    # trapezoid mean in u equals the paper's integral average
    mean = np.trapezoid(vals, dx=1.0) / (len(vals) - 1)
    assert mean == pytest.approx(g["e_avg"], abs=1.5e-3)


def test_null_distribution_fixed_phase_standard_normal():
    """Under H0 the Z-statistic of a fixed template is N(0,1) (Sec. 3.3): p = 1 bin
    leaves a single phase and width, so S/N = (sum of the folded samples)/sqrt(m V)."""
    vals = []
    f = 3.0
    for seed in range(1500):
        x = synth.white_noise(300, seed=seed).astype(np.float32)
        d = oracle.downsample(x, f)
        m = len(d)
        F = oracle.ffa(d.reshape(m, 1))
        vals.append(oracle.boxcar_snr(F[0], [1], math.sqrt(m * oracle.downsampled_variance(f)))[0, 0])
    vals = np.array(vals)
    assert abs(vals.mean()) < 3 / math.sqrt(len(vals))
    assert abs(vals.std() - 1) < 3 / math.sqrt(2 * len(vals))


def test_null_distribution_noninteger_factor():
    """With a non-integer factor, bins folded at a stride of p >= 2 downsampled
    samples are uncorrelated with variance averaging f - 1/3 (Sec. 5.3), so the S/N
    of a fixed bin stays close to unit variance."""
    vals = []
    f, p = math.pi, 7
    for seed in range(800):
        x = synth.white_noise(4000, seed=10_000 + seed).astype(np.float32)
        d = oracle.downsample(x, f)
        m = len(d) // p
        col = d[: m * p].reshape(m, p)[:, 3]
        vals.append(col.sum() / math.sqrt(m * oracle.downsampled_variance(f)))
    vals = np.array(vals)
    assert abs(vals.std() - 1) < 4 / math.sqrt(2 * len(vals))


def test_cauchy_schwarz_bound():
    """A noiseless unit-square-sum train of amplitude a never scores above a."""
    n, tsamp = 20000, 1e-3
    pulse = synth.Pulse(0.25, 0.05, 12.0, 0.3)
    x = synth.pulse_train(n, tsamp, pulse).astype(np.float32)
    p = 250
    m = n // p
    F = oracle.ffa(x[: m * p].reshape(m, p).astype(np.float64))
    snr = oracle.boxcar_snr(F, [1, 2, 4, 8, 16, 32], math.sqrt(m))
    assert snr.max() <= 12.0 + 1e-9
    assert snr.max() > 0.85 * 12.0   # the matched row recovers most of it


def test_invalid_arguments():
    with pytest.raises(ValueError):
        oracle.boxcar_snr(np.zeros((2, 5)), [0], 1.0)
    with pytest.raises(ValueError):
        oracle.boxcar_snr(np.zeros((2, 5)), [6], 1.0)
    with pytest.raises(ValueError):
        oracle.boxcar_snr(np.zeros((2, 5)), [1], 0.0)


# ------------------------------------------------------------ zero-mean boxcar template
def _zm_template(p, w):
    """The zero-mean boxcar as an explicit vector: equal values on w bins, equal values
    on the rest, zero sum and unit square sum (built by projection, not by formula)."""
    t = np.zeros(p)
    t[:w] = 1.0
    t -= t.mean()
    return t / np.sqrt(np.sum(t * t))


@pytest.mark.parametrize("p,widths", [(7, (1, 2, 3, 6)), (40, (1, 3, 9, 20)), (251, (1, 13, 63))])
def test_zero_mean_boxcar_is_a_circular_correlation(p, widths):
    """Z at every phase is the circular correlation of the profile with the explicit
    template (computed here by FFT), maximised over phase."""
    rng = synth.rng(p)
    prof = rng.standard_normal((5, p)) + 3.0
    got = oracle.boxcar_snr(prof, widths, 1.7, zero_mean=True)
    for iw, w in enumerate(widths):
        t = _zm_template(p, w)
        corr = np.real(np.fft.ifft(np.conj(np.fft.fft(t))[None, :] * np.fft.fft(prof, axis=1),
                                   axis=1))
        np.testing.assert_allclose(got[:, iw], corr.max(axis=1) / 1.7, rtol=1e-12, atol=1e-12)


def test_zero_mean_boxcar_ignores_a_constant_and_is_unit_normal():
    rng = synth.rng(5)
    prof = rng.standard_normal((2000, 64))
    a = oracle.boxcar_snr(prof, (1, 4, 16), 1.0, zero_mean=True)
    b = oracle.boxcar_snr(prof + 123.0, (1, 4, 16), 1.0, zero_mean=True)
    np.testing.assert_allclose(a, b, atol=1e-9)
    # the statistic at one fixed phase is N(0, 1) under pure noise (unit square sum)
    t = _zm_template(64, 4)
    z = prof @ t
    assert abs(z.mean()) < 3 / np.sqrt(len(z)) and abs(z.std() - 1.0) < 0.05


def test_zero_mean_boxcar_rejects_full_width():
    with pytest.raises(ValueError):
        oracle.boxcar_snr(np.zeros((1, 8)), (8,), 1.0, zero_mean=True)


def test_zero_mean_periodogram_recovers_the_pulse():
    w = synth.plain_small()
    ref = oracle.periodogram(w.x, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths,
                             zero_mean=True)
    best = ref.snr.max(axis=1)
    assert abs(ref.periods[best.argmax()] - 2.345) / 2.345 < 2e-3
