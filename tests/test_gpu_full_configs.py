"""Parity at the full sizes of the two batched workloads, in the launch configuration
that bench.py times (one BatchSearcher over the whole batch, 48 GB workspace budget per
chunk), checked on sampled outputs that the oracle computes one by one:

  * batch_uneven: 256 FP32 series of U[2^20, 2^23] samples, own period ranges;
  * batch_int8: 1024 series of 2^21 samples of white plus red noise, de-reddened by the
    library's running median (1 s) and normalised and stored as int8 by the library (the
    oracle searches the same dequantised values: pure accumulation error).

For three series of each batch (first, middle, last) a spread of transforms is
compared: periods and fold bins exactly, S/N within 1e-4 of the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SNR_TOL = 1e-4
BUDGET = 48 << 30


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_03701_gb300 as ffa
    ffa.build()
    ffa.library()
    return ffa


def _check_series(F, S, i, s, x, widths, seed):
    pl = oracle.plan(s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax)
    if pl.n_transforms == 0:
        return 0
    sel = np.zeros(pl.n_transforms, bool)
    sel[[0, pl.n_transforms - 1]] = True
    sel[int(np.argmax(pl.tr_m))] = True
    sel[synth.rng(seed).choice(pl.n_transforms, min(3, pl.n_transforms), replace=False)] = True
    ref = oracle.periodogram(x, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax, widths, select=sel)
    rows = np.concatenate([np.arange(pl.tr_first_trial[t], pl.tr_first_trial[t] + pl.tr_kept[t])
                           for t in np.flatnonzero(sel)])
    per, fb, snr = (t.cpu().numpy() for t in S.series_result(i))
    assert len(per) == pl.n_trials
    np.testing.assert_array_equal(per[rows], ref.periods)
    np.testing.assert_array_equal(fb[rows], ref.foldbins)
    err = np.abs(snr[rows].astype(np.float64) - ref.snr).max()
    assert err <= SNR_TOL, (i, err)
    assert np.isfinite(snr).all()
    return len(rows)


def _series(F, b):
    return [F.Series(s.offset, s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax) for s in b.series]


def test_batch_uneven_full_size(F):
    b = synth.batch_uneven()
    S = F.BatchSearcher(_series(F, b), b.widths, ws_budget=BUDGET)
    S(torch.from_numpy(b.x).cuda())
    torch.cuda.synchronize()
    S.check()
    n = 0
    for i in (0, len(b.series) // 2, len(b.series) - 1):
        n += _check_series(F, S, i, b.series[i], b.series_x(i), b.widths, seed=i)
    assert n > 0
    del S
    torch.cuda.empty_cache()


def test_batch_int8_full_size(F):
    b = synth.batch_int8_stress()
    x32 = torch.from_numpy(b.x).cuda()
    # red noise removed by the library's running median (1 s), then int8 storage
    width = F.median_width(synth.DEREDDEN_SECONDS, b.series[0].tsamp)
    q = F.prepare_batch(x32, [(s.offset, s.n) for s in b.series], width, torch.int8)
    del x32
    S = F.BatchSearcher(_series(F, b), b.widths, ws_budget=BUDGET)
    S(q)
    torch.cuda.synchronize()
    S.check()
    n = 0
    for i in (0, len(b.series) // 2, len(b.series) - 1):
        s = b.series[i]
        deq = q[s.offset:s.offset + s.n].cpu().numpy().astype(np.float32) / 16
        n += _check_series(F, S, i, s, deq, b.widths, seed=100 + i)
    assert n > 0
    del S, q
    torch.cuda.empty_cache()
