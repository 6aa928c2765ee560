"""Parity of the GPU peak finder (Sec. 5.5, Fig. 6) with the oracle's, through the C ABI,
on the same periodogram arrays: the peaks (trial, period, S/N, width) are compared
exactly.  Inputs: synthetic periodograms with trends and bumps whose margins to the
threshold are far above the FP64 fitting error, the GPU's own periodogram of a series
with an injected pulse train, and the full survey-shaped periodogram (662,440 trials x
11 widths).  Edge cases: no control points, a single width, peak_cap truncation, and
periods out of order (rejected on the device, visible to ffa_check)."""
import math

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


def _gpu(F, P, S, tobs, **opts):
    S2 = S if S.ndim == 2 else S[:, None]
    pk, counts = F.find_peaks(torch.from_numpy(np.ascontiguousarray(P)).cuda(),
                              torch.from_numpy(np.ascontiguousarray(S2, dtype=np.float32)).cuda(),
                              tobs, **opts)
    return pk, counts


def _compare(P, S, tobs, pk, counts, **opts):
    S2 = S if S.ndim == 2 else S[:, None]
    ref = oracle.find_peaks(P, S2.astype(np.float32), tobs, **opts)
    assert list(counts) == [len(r.peaks) for r in ref]
    want = np.concatenate([r.peaks for r in ref]) if ref else np.zeros(0, np.int64)
    np.testing.assert_array_equal(pk["trial"], want)
    iw = np.concatenate([np.full(len(r.peaks), i) for i, r in enumerate(ref)])
    np.testing.assert_array_equal(pk["iw"], iw)
    np.testing.assert_array_equal(pk["period"], P[want])
    np.testing.assert_array_equal(pk["snr"], S2.astype(np.float32)[want, iw])
    return ref


def _grid(nseg, per_seg, tobs, nu0):
    w = 5.0 / tobs
    nu = np.concatenate([nu0 + (j + (np.arange(per_seg) + 0.5 + (0.2 if j else 0.0)) / per_seg) * w
                         for j in range(nseg)])
    nu = np.sort(nu)[::-1]
    return 1.0 / nu, nu


def test_trend_and_bumps_three_widths(F):
    tobs = 500.0
    P, nu = _grid(300, 250, tobs, 0.1)
    r = synth.rng(8)
    cols = []
    for iw in range(3):
        trend = 2.0 - (1.0 + iw) * np.log(nu) + 0.5 * np.log(nu) ** 2
        s = trend + r.standard_normal(len(P))
        for k in r.choice(len(P) - 5, 6, replace=False):
            s[k:k + 3] = trend[k:k + 3] + [10.0, 13.0 + iw, 9.5]
        cols.append(s)
    S = np.stack(cols, axis=1).astype(np.float32)
    pk, counts = _gpu(F, P, S, tobs)
    ref = _compare(P, S, tobs, pk, counts)
    assert all(len(x.peaks) >= 5 for x in ref)
    # no trial within 1e-6 of its width's threshold: the comparison is not on a knife edge
    for iw, x in enumerate(ref):
        assert np.abs(S[:, iw] - x.threshold).min() > 1e-6


@pytest.mark.parametrize("clrad", [0.1, 1.0, 4.0])
def test_cluster_radius(F, clrad):
    tobs = 500.0
    P, nu = _grid(100, 250, tobs, 0.1)
    s = synth.rng(4).standard_normal(len(P)) * 0.01
    i0 = 10000
    step = nu[i0] - nu[i0 + 1]
    s[i0:i0 + 3] = [12.0, 15.0, 11.0]
    s[i0 + int(math.ceil(2.0 / tobs / step)) + 3] = 9.0
    s[i0 + 2 + int(0.5 / tobs / step)] = 20.0
    s[i0 + 2 + int(0.5 / tobs / step) + 1] = 20.0     # equal S/N: the lower index wins
    pk, counts = _gpu(F, P, s, tobs, clrad=clrad)
    _compare(P, s, tobs, pk, counts, clrad=clrad)


def test_degree_and_segment_options(F):
    tobs = 300.0
    P, nu = _grid(120, 60, tobs, 0.3)
    s = (1.0 + 0.3 * np.log(nu) + synth.rng(6).standard_normal(len(P))).astype(np.float32)
    s[1234] += 12.0
    for opts in (dict(degree=0), dict(degree=1, dzseg=3.0), dict(degree=4, nsigma=5.0),
                 dict(min_seg=61), dict(degree=2, min_seg=20, dzseg=10.0)):
        pk, counts = _gpu(F, P, s, tobs, **opts)
        _compare(P, s, tobs, pk, counts, **opts)


def test_no_control_points_and_cap(F):
    tobs = 300.0
    P, nu = _grid(10, 5, tobs, 0.3)          # segments of 5 trials < min_seg 8
    s = np.zeros(len(P), np.float32)
    pk, counts = _gpu(F, P, s, tobs)
    assert len(pk) == 0 and list(counts) == [0]
    P, nu = _grid(100, 250, 500.0, 0.1)
    s = synth.rng(9).standard_normal(len(P)).astype(np.float32) * 0.01
    s[::997] = 30.0
    pd, sd = torch.from_numpy(P).cuda(), torch.from_numpy(s[:, None].copy()).cuda()
    Fp = F.PeakFinder(len(P), 1, 500.0, peak_cap=7)
    Fp(pd, sd)
    pk, counts = Fp.result()
    ref = oracle.find_peaks(P, s[:, None], 500.0)[0]
    assert counts[0] == len(ref.peaks) > 7
    np.testing.assert_array_equal(pk["trial"], ref.peaks[:7])


def test_periods_out_of_order_are_rejected(F):
    P, nu = _grid(20, 50, 300.0, 0.3)
    P = P.copy()
    P[[100, 101]] = P[[101, 100]]
    Fp = F.PeakFinder(len(P), 1, 300.0)
    Fp(torch.from_numpy(P).cuda(), torch.zeros(len(P), 1, device="cuda"))
    with pytest.raises(F.FFAError):
        Fp.check()
    pk, counts = Fp.result()
    assert len(pk) == 0 and list(counts) == [0]


def test_peaks_of_a_gpu_periodogram(F):
    """The library's own periodogram of a series with a 0.77 s pulse train: the GPU and
    the oracle find the same peaks on it, and the brightest is at the pulse period."""
    w = synth.custom(2 ** 17, 1e-3, 0.5, 3.0, 40, 44, (1, 2, 4, 8), seed=5,
                     pulses=[synth.Pulse(0.77, 0.05, 14.0, 0.2)])
    per, fb, snr = F.periodogram(torch.from_numpy(w.x).cuda(), w.tsamp, w.pmin, w.pmax,
                                 w.bmin, w.bmax, w.widths)
    torch.cuda.synchronize()
    tobs = len(w.x) * w.tsamp
    P, S = per.cpu().numpy(), snr.cpu().numpy()
    pk, counts = F.find_peaks(per, snr, tobs)
    _compare(P, S, tobs, pk, counts)
    best = pk[np.argmax(pk["snr"])]
    assert abs(best["period"] / 0.77 - 1.0) < 2e-3


def test_full_survey_periodogram(F):
    """The survey-shaped periodogram (2^23 samples at 64 us, 662,440 trials, 11 widths)
    searched on the GPU equals the oracle's search of the same arrays."""
    wl = synth.survey()
    S = F.Searcher(len(wl.x), wl.tsamp, wl.pmin, wl.pmax, wl.bmin, wl.bmax, wl.widths)
    S(torch.from_numpy(wl.x).cuda())
    torch.cuda.synchronize()
    per, snr = S.periods, S.snr
    tobs = len(wl.x) * wl.tsamp
    pk, counts = F.find_peaks(per, snr, tobs)
    ref = _compare(per.cpu().numpy(), snr.cpu().numpy(), tobs, pk, counts)
    # the two brighter injected trains (1.7 s at S/N 14, 7.9 s at S/N 20) are peaks
    for P0 in (1.7, 7.9):
        assert np.any(np.abs(pk["period"] / P0 - 1.0) < 2e-3), P0


def _check_fits(F, P, S, tobs, **opts):
    """Control points bit-identical to the oracle's; thresholds evaluated from the GPU's
    fitted polynomial within 1e-9 (relative) of the oracle's per-trial thresholds."""
    S2 = np.ascontiguousarray(S if S.ndim == 2 else S[:, None], dtype=np.float32)
    PF = F.PeakFinder(len(P), S2.shape[1], tobs, **opts)
    PF(torch.from_numpy(np.ascontiguousarray(P)).cuda(), torch.from_numpy(S2).cuda())
    PF.result()
    ctrl, fits = PF.fits()
    ref = oracle.find_peaks(P, S2, tobs, **opts)
    lnnu = np.log(1.0 / P)
    for iw, r in enumerate(ref):
        got = ctrl[:, iw]
        keep = ~np.isnan(got[:, 1])
        np.testing.assert_array_equal(got[keep, 0], r.ctrl_nu)
        np.testing.assert_array_equal(got[keep, 1], r.ctrl_s)
        xbar, xscale, valid = fits[iw, :3]
        if r.coef is None:
            assert valid == 0
            continue
        assert valid == 1
        u = (lnnu - xbar) / xscale
        thr = np.zeros_like(u)
        for a in range(6, -1, -1):
            thr = thr * u + fits[iw, 3 + a]
        np.testing.assert_allclose(thr, r.threshold, rtol=1e-9, atol=1e-9)
    return ref


def test_control_points_fits_and_thresholds(F):
    """Not only the selected peaks: the intermediate results that decide them."""
    tobs = 500.0
    P, nu = _grid(300, 250, tobs, 0.1)
    r = synth.rng(18)
    cols = []
    for iw in range(3):
        trend = 2.0 - (1.0 + iw) * np.log(nu) + 0.5 * np.log(nu) ** 2
        cols.append(trend + r.standard_normal(len(P)))
    S = np.stack(cols, axis=1).astype(np.float32)
    ref = _check_fits(F, P, S, tobs)
    assert all(len(x.ctrl_nu) > 100 for x in ref)
    for opts in (dict(degree=0), dict(degree=4, nsigma=5.0), dict(dzseg=10.0, min_seg=20)):
        _check_fits(F, P, S[:, :1], tobs, **opts)


def test_fits_without_control_points(F):
    tobs = 300.0
    P, nu = _grid(10, 5, tobs, 0.3)          # segments of 5 trials < min_seg 8
    _check_fits(F, P, np.zeros(len(P), np.float32), tobs)
