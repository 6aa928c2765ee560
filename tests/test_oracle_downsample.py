"""Pins of the oracle's real-factor downsampling (Sec. 5.3, App. A.4): integer
factors give block sums, the window weights partition unity, the per-window
variance follows the closed form of App. A.4 and averages f - 1/3."""
import math

import numpy as np
import pytest

import oracle
import synth


def weights_matrix(n, f):
    """Rows of the linear map x -> downsample(x), read off unit impulses."""
    nout = oracle.downsampled_length(n, f)
    W = np.zeros((nout, n))
    for j in range(n):
        e = np.zeros(n, np.float32)
        e[j] = 1.0
        W[:, j] = oracle.downsample(e, f)
    return W


@pytest.mark.parametrize("f", [1, 2, 3, 7, 16])
def test_integer_factor_is_block_sum(f):
    x = synth.normal_block(1, 1000, seed=f)[0]
    out = oracle.downsample(x, float(f))
    nout = len(x) // f
    ref = x[: nout * f].astype(np.float64).reshape(nout, f).sum(axis=1)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("f", [1.0, 1.5, math.pi, 4.1666666666666667, 13.020833333333334])
def test_constant_input_gives_window_length(f):
    x = np.ones(5000, np.float32)
    out = oracle.downsample(x, f)
    assert len(out) == int(math.floor(5000 / f))
    np.testing.assert_allclose(out, f, rtol=1e-12)


@pytest.mark.parametrize("f", [math.sqrt(2.0), 1.0875 * 3, math.e, 9.3])
def test_total_is_preserved(f):
    x = synth.normal_block(1, 3001, seed=4)[0].astype(np.float64)
    out = oracle.downsample(x.astype(np.float32), f)
    L = len(out) * f
    ref = x[: int(math.floor(L))].sum() + (L - math.floor(L)) * x[int(math.floor(L))]
    assert abs(out.sum() - ref) < 1e-9


def window_variance(phi, f):
    """App. A.4: variance of one output sample for window start phase phi."""
    n = math.floor(f)
    r = f - n
    if phi < 1 - r:
        return (1 - phi) ** 2 + (n - 1) + (r + phi) ** 2
    return (1 - phi) ** 2 + n + (r + phi - 1) ** 2


@pytest.mark.parametrize("f", [math.sqrt(2.0) + 1, math.pi, 2.71828, 13.0208])
def test_window_variance_closed_form(f):
    W = weights_matrix(200, f)
    for i in range(W.shape[0]):
        phi = i * f - math.floor(i * f)
        assert abs((W[i] ** 2).sum() - window_variance(phi, f)) < 1e-9


@pytest.mark.parametrize("f", [math.pi, math.sqrt(7.0), 4.53125 * 1.0001])
def test_mean_window_variance_is_f_minus_third(f, paper_values):
    """Irrational factor: window phases equidistribute, mean variance f - 1/3."""
    off = paper_values["noninteger_downsampling_variance"]["mean_offset"]
    n = 200000
    nout = oracle.downsampled_length(n, f)
    phis = np.array([i * f - math.floor(i * f) for i in range(nout)])
    v = np.array([window_variance(ph, f) for ph in phis]).mean()
    assert abs(v - (f + off)) < 2e-3
    assert oracle.downsampled_variance(f) == pytest.approx(f + off, abs=1e-15)
    assert oracle.downsampled_variance(float(math.floor(f))) == math.floor(f)


def test_noise_variance_numerically(paper_values):
    """App. A.4 'verified numerically by downsampling artificial Gaussian noise'."""
    f = math.pi
    x = synth.white_noise(2_000_000, seed=123).astype(np.float32)
    out = oracle.downsample(x, f)
    off = paper_values["noninteger_downsampling_variance"]["mean_offset"]
    assert abs(out.var() - (f + off)) < 0.02


def test_invalid_factor():
    with pytest.raises(ValueError):
        oracle.downsample(np.ones(10, np.float32), 0.5)
