"""Parity of the running-median de-reddening (Sec. 5.2) with the oracle, through the C
ABI: the medians are samples of the window, so the comparison is bit-exact, and so is
y = x - med (one float subtraction on both sides).  Sizes span several build tiles of
4096 samples and ragged tails, windows longer than the series, ties, in-place output,
series of more than 4096 tiles (the build's scan launch),
and the full size of a 2^23-sample series at 64 us with a 1 s window (15625 samples)
on sampled outputs, including every output whose window reaches past an end."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_03701_gb300 as ffa
    ffa.build()
    ffa.library()
    return ffa


def _run(F, x, w):
    xd = torch.from_numpy(x).cuda()
    med = torch.empty_like(xd)
    y = torch.empty_like(xd)
    F.RunningMedian(len(x), w)(xd, med=med, y=y)
    torch.cuda.synchronize()
    return med.cpu().numpy(), y.cpu().numpy()


@pytest.mark.parametrize("n,w", [(1, 1), (1, 5), (2, 3), (31, 3), (32, 5), (33, 65),
                                 (4096, 101), (4097, 33), (8192, 1), (5000, 4999),
                                 (3000, 6001), (12289, 255), (60000, 1001)])
def test_running_median_equals_oracle(F, n, w):
    x = synth.rng(n * 7 + w).standard_normal(n).astype(np.float32)
    med, y = _run(F, x, w)
    ref = oracle.running_median(x, w)
    np.testing.assert_array_equal(med, ref)
    np.testing.assert_array_equal(y, x - ref)


def test_ties(F):
    """Integer-valued samples: long runs of equal keys in every window."""
    x = synth.rng(9).integers(-4, 5, 50000).astype(np.float32)
    for w in (3, 777):
        med, _ = _run(F, x, w)
        np.testing.assert_array_equal(med, oracle.running_median(x, w))


def test_red_noise_in_place(F):
    """A red-noise series de-reddened in place equals the oracle's x - med."""
    n, w = 40000, 1563
    x = synth.red_noise(n, 64e-5, seed=12)
    xd = torch.from_numpy(x).cuda()
    F.deredden(xd, w, inplace=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(xd.cpu().numpy(), oracle.deredden(x, w))


def test_monotone_series_gives_zero(F):
    x = np.sort(synth.rng(2).standard_normal(20000)).astype(np.float32)
    med, y = _run(F, x, 501)
    np.testing.assert_array_equal(med, x)
    assert not y.any()


def test_full_size_survey_window(F):
    """2^23 samples at 64 us, 1 s window: sampled outputs against the oracle, with both
    ends' windows (which hold copies of the end samples) checked in full."""
    n, tsamp = 2 ** 23, 64e-6
    w = F.median_width(1.0, tsamp)
    h = w // 2
    x = synth.red_noise(n, tsamp, seed=5)
    med, y = _run(F, x, w)
    r = synth.rng(77)
    at = np.unique(np.concatenate([np.arange(0, 300), np.arange(h - 150, h + 150),
                                   np.arange(n - h - 150, n - h + 150), np.arange(n - 300, n),
                                   r.integers(0, n, 600)]))
    ref = oracle.running_median(x, w, at=at)
    np.testing.assert_array_equal(med[at], ref)
    np.testing.assert_array_equal(y[at], x[at] - ref)
    assert np.isfinite(med).all()


def test_series_longer_than_4096_tiles(F):
    """More than 4096 build tiles of 4096 samples: the per-level tile prefix comes from
    the one-CTA scan launch instead of each scatter CTA's own sum."""
    n, w = 4096 * 4096 + 4097, 101
    x = synth.rng(31).standard_normal(n).astype(np.float32)
    med, y = _run(F, x, w)
    r = synth.rng(32)
    at = np.unique(np.concatenate([np.arange(0, 100), np.arange(n - 100, n),
                                   np.arange(4096 * 4096 - 50, 4096 * 4096 + 50),
                                   r.integers(0, n, 2000)]))
    ref = oracle.running_median(x, w, at=at)
    np.testing.assert_array_equal(med[at], ref)
    np.testing.assert_array_equal(y[at], x[at] - ref)


def test_deredden_then_normalise(F):
    """The pre-processing of Sec. 5.2 on the device (de-redden, then normalise) against
    the oracle's (de-redden, then normalise in FP64)."""
    n, w = 30000, 2001
    x = synth.red_noise(n, 1e-3, seed=3)
    xd = torch.from_numpy(x).cuda()
    xn, mean, std = F.normalise(F.deredden(xd, w))
    m0, s0, ref = oracle.normalise(oracle.deredden(x, w))
    assert mean == pytest.approx(m0, rel=1e-12, abs=1e-12)
    assert std == pytest.approx(s0, rel=1e-12)
    np.testing.assert_allclose(xn.cpu().numpy(), ref, atol=1e-6)
