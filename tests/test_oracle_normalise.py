"""Pins of the oracle's normalisation (Sec. 3.1, Sec. 5.2): closed-form statistics of an
arithmetic sequence, zero mean / unit deviation of the output, invariance under positive
affine maps of the input."""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 65537])
def test_arithmetic_sequence_closed_form(n):
    x = np.arange(n, dtype=np.float32)
    mean, std, out = oracle.normalise(x)
    assert mean == pytest.approx((n - 1) / 2, rel=1e-14, abs=1e-14)
    assert std == pytest.approx(math.sqrt((n * n - 1) / 12.0), rel=1e-12, abs=1e-14)
    if n > 1:
        assert abs(out.mean()) < 1e-12 and out.std() == pytest.approx(1.0, rel=1e-12)


def test_output_moments_and_affine_invariance():
    x = synth.white_noise(100_000, seed=3).astype(np.float32)
    m1, s1, o1 = oracle.normalise(x)
    assert abs(o1.mean()) < 1e-12 and o1.std() == pytest.approx(1.0, rel=1e-12)
    y = (3.0 * x.astype(np.float64) + 40.0).astype(np.float32)
    m2, s2, o2 = oracle.normalise(y)
    assert m2 == pytest.approx(3 * m1 + 40, rel=1e-6)
    assert s2 == pytest.approx(3 * s1, rel=1e-6)
    np.testing.assert_allclose(o2, o1, atol=2e-5)


def test_constant_series():
    mean, std, out = oracle.normalise(np.full(10, 2.5, np.float32))
    assert mean == 2.5 and std == 0.0 and np.all(out == 0.0)
