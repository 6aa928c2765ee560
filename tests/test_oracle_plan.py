"""Pins of the oracle's search plan and trial periods (Sec. 2.3, Sec. 5.3, Sec. 5.6)
and of its end-to-end periodogram (recovery of injected pulses)."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_width_sets_follow_the_recurrence(paper_values):
    """Sec. 5.4: w_{k+1} = max(floor(f_sp w_k), w_k + 1) from w_0 = 1."""
    def seq(fsp, wmax):
        w = [paper_values["width_recurrence"]["w0"]]
        while True:
            nxt = max(int(math.floor(fsp * w[-1])), w[-1] + 1)
            if nxt > wmax:
                return tuple(w)
            w.append(nxt)
    assert seq(paper_values["width_recurrence"]["f_sp"], 63) == synth.WIDTHS_11
    assert seq(1.37, 120) == synth.WIDTHS_16


@pytest.mark.parametrize("m,p", [(2, 240), (3, 7), (26, 260), (2684, 240), (100, 1)])
def test_trial_periods(m, p, paper_values):
    tau = 1.7e-4
    P = np.array([oracle.trial_period(tau, p, m, s) for s in range(m)])
    assert P[0] == pytest.approx(p * tau, rel=1e-15)          # s = 0: base period
    assert np.all(np.diff(P) > 0)
    assert P[-1] > (p + 1) * tau                               # Sec. 2.3 remark
    # Eq. nu_s: trial frequencies are linear in s with step 1/((m-1) p^2 tau)
    nu = 1.0 / P
    expect = (1.0 / p - np.arange(m) / ((m - 1) * p * p)) / tau
    np.testing.assert_allclose(nu, expect, rtol=1e-13)


def test_plan_structure():
    n, tsamp, pmin, pmax, bmin, bmax = 2 ** 20, 64e-6, 0.1, 5.0, 240, 260
    pl = oracle.plan(n, tsamp, pmin, pmax, bmin, bmax)
    f = pl.oct_factor
    # Sec. 5.6: the first octave brings tau to Pmin / bmin
    assert bmin * tsamp * f[0] == pytest.approx(pmin, rel=1e-14)
    # Sec. 5.3: factors grow by (bmax + 1) / bmin; octave k+1 starts where k ends
    np.testing.assert_allclose(f[1:] / f[:-1], (bmax + 1) / bmin, rtol=1e-13)
    assert bmin * tsamp * f[-1] <= pmax < bmin * tsamp * f[-1] * (bmax + 1) / bmin
    np.testing.assert_array_equal(pl.oct_len, np.floor(n / f).astype(np.int64))
    # each transform: m = floor(N_k / p) rows, kept rows have P_s < (p + 1) tau_k
    for t in range(pl.n_transforms):
        k, p, m, kept = pl.tr_octave[t], int(pl.tr_p[t]), int(pl.tr_m[t]), int(pl.tr_kept[t])
        assert m == pl.oct_len[k] // p and m >= 2
        tau = tsamp * f[k]
        P = [oracle.trial_period(tau, p, m, s) for s in range(m)]
        assert all(P[s] < (p + 1) * tau for s in range(kept))
        assert all(P[s] >= (p + 1) * tau * (1 - 1e-15) for s in range(kept, m))
    assert pl.tr_first_trial[-1] + pl.tr_kept[-1] == pl.n_trials


def test_invalid_plans():
    with pytest.raises(ValueError):
        oracle.plan(1000, 1e-3, 0.1, 1.0, 240, 260)   # Pmin / bmin below tsamp
    with pytest.raises(ValueError):
        oracle.plan(1000, 1e-3, 2.0, 1.0, 240, 260)   # Pmax < Pmin
    with pytest.raises(ValueError):
        oracle.plan(1000, 1e-3, 1.0, 2.0, 260, 240)   # bmax < bmin


def _small_workload(seed, pulses):
    return synth.custom(2 ** 17, 1e-3, 0.5, 4.0, 60, 66, (1, 2, 3, 4, 6, 9), seed, pulses)


def test_periodogram_periods_strictly_increasing_and_contiguous():
    w = _small_workload(1, [])
    pg = oracle.periodogram(w.x, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    assert np.all(np.diff(pg.periods) > 0)
    assert pg.periods[0] == pytest.approx(w.pmin, rel=1e-14)
    assert pg.snr.shape == (len(pg.periods), len(w.widths))
    pl = oracle.plan(w.n, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax)
    assert len(pg.periods) == pl.n_trials


def test_periodogram_select_mask_matches_full():
    w = _small_workload(2, [])
    pl = oracle.plan(w.n, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax)
    full = oracle.periodogram(w.x, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    sel = np.zeros(pl.n_transforms, bool)
    sel[[0, 5, pl.n_transforms - 1]] = True
    part = oracle.periodogram(w.x, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths, sel)
    rows = np.concatenate([np.arange(pl.tr_first_trial[t], pl.tr_first_trial[t] + pl.tr_kept[t])
                           for t in np.flatnonzero(sel)])
    np.testing.assert_array_equal(part.periods, full.periods[rows])
    np.testing.assert_array_equal(part.snr, full.snr[rows])


def test_injected_pulse_recovery():
    """The noisy periodogram peaks within two trials of the injected period, with
    S/N within 3 of the noiseless expectation (Z ~ N(E a, 1), Sec. 3.5)."""
    P0, a = 1.234, 15.0
    pulse = synth.Pulse(P0, 0.03, a, 0.37)
    noisy = _small_workload(3, [pulse])
    clean_x = synth.pulse_train(noisy.n, noisy.tsamp, pulse).astype(np.float32)
    args = (noisy.tsamp, noisy.pmin, noisy.pmax, noisy.bmin, noisy.bmax, noisy.widths)
    pg = oracle.periodogram(noisy.x, *args)
    clean = oracle.periodogram(clean_x, *args)
    best = pg.snr.max(axis=1)
    i_true = int(np.argmin(np.abs(pg.periods - P0)))
    expected = clean.snr[max(0, i_true - 2): i_true + 3].max()
    i_peak = int(np.argmax(best))
    assert abs(i_peak - i_true) <= 2 or abs(pg.periods[i_peak] - P0) / P0 < 1e-4
    assert abs(best[i_peak] - expected) < 3.0
    assert expected > 0.85 * a
