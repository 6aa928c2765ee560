"""Batched periodograms (many series of uneven length in one buffer, each with its own
period range) against the CPU oracle run on each series alone, through the C ABI.

Bars as for one series: periods and fold bins identical, S/N within 1e-4 of the FP64
oracle.  Also: a series' periodogram does not depend on the batch around it (its
prefix sums restart at its first sample), so it is bit-identical to the single-series
call for any cut of the batch into launch chunks and any place of the series in the
buffer; and a captured CUDA graph of the batch call replays it exactly."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SNR_TOL = 1e-4


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_03701_gb300 as ffa
    ffa.build()
    ffa.library()
    return ffa


@pytest.fixture(scope="module")
def batch():
    return synth.batch_uneven(7, 2 ** 15, 2 ** 17, seed=21, threads=4)


def _series(F, b, offsets=None):
    return [F.Series(s.offset if offsets is None else offsets[i], s.n, s.tsamp, s.pmin, s.pmax,
                     s.bmin, s.bmax) for i, s in enumerate(b.series)]


def _oracle(b, i, x=None):
    s = b.series[i]
    xs = b.series_x(i) if x is None else x
    return oracle.periodogram(xs, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax, b.widths)


def _compare(got, ref):
    per, fb, snr = (t.cpu().numpy() for t in got)
    np.testing.assert_array_equal(per, ref.periods)
    np.testing.assert_array_equal(fb, ref.foldbins)
    if len(per):
        err = np.abs(snr.astype(np.float64) - ref.snr).max()
        assert err <= SNR_TOL, err


@pytest.mark.parametrize("budget", [1 << 40, 1, 2 << 20])
def test_batch_matches_oracle_per_series(F, batch, budget):
    S = F.BatchSearcher(_series(F, batch), batch.widths, ws_budget=budget)
    if budget == 1:
        assert S.info.nchunks == len(batch.series)
    if budget == 1 << 40:
        assert S.info.nchunks == 1
    S(torch.from_numpy(batch.x).cuda())
    torch.cuda.synchronize()
    S.check()
    for i in range(len(batch.series)):
        _compare(S.series_result(i), _oracle(batch, i))


def test_batch_equals_single_series_calls(F, batch):
    x = torch.from_numpy(batch.x).cuda()
    ser = _series(F, batch)
    for budget in (1 << 40, 1, 3 << 20):
        S = F.BatchSearcher(ser, batch.widths, ws_budget=budget)
        S(x)
        torch.cuda.synchronize()
        for i, s in enumerate(batch.series):
            one = F.periodogram(x[s.offset:s.offset + s.n], s.tsamp, s.pmin, s.pmax, s.bmin,
                                s.bmax, batch.widths)
            for a, b in zip(S.series_result(i), one):
                assert torch.equal(a, b), (budget, i)


def test_batch_series_anywhere_in_the_buffer(F, batch):
    """Series stored out of order with gaps between them."""
    order = [3, 0, 6, 2, 5, 1, 4]
    offs, pos = [0] * len(order), 1000
    for k in order:
        offs[k] = pos
        pos += batch.series[k].n + 333
    buf = np.full(pos + 77, np.float32(1e30))   # gaps hold values no search may touch
    for k, s in enumerate(batch.series):
        buf[offs[k]:offs[k] + s.n] = batch.series_x(k)
    S = F.BatchSearcher(_series(F, batch, offs), batch.widths, ws_budget=2 << 20)
    S(torch.from_numpy(buf).cuda())
    torch.cuda.synchronize()
    S.check()
    for i in (0, 3, 6):
        _compare(S.series_result(i), _oracle(batch, i))


def test_batch_int8_storage(F, batch):
    """Each series normalised and stored as int8 (q/16) in one buffer: FP32 accumulation
    error against the FP64 oracle run on the dequantised values."""
    q = np.zeros(len(batch.x), np.int8)
    for i, s in enumerate(batch.series):
        x64 = batch.series_x(i).astype(np.float64)
        xn = (x64 - x64.mean()) / x64.std()
        q[s.offset:s.offset + s.n] = np.clip(np.rint(16 * xn), -128, 127).astype(np.int8)
    S = F.BatchSearcher(_series(F, batch), batch.widths, ws_budget=4 << 20)
    S(torch.from_numpy(q).cuda())
    torch.cuda.synchronize()
    S.check()
    for i in (1, 4):
        s = batch.series[i]
        deq = q[s.offset:s.offset + s.n].astype(np.float32) / 16
        _compare(S.series_result(i), _oracle(batch, i, deq))


def test_batch_cuda_graph_replay(F, batch):
    """The batch call captured once into a CUDA graph replays bit-identically to the
    eager call, on the data present in the input buffer at replay time."""
    S = F.BatchSearcher(_series(F, batch), batch.widths, ws_budget=1)  # a chunk per series
    assert S.info.nchunks == len(batch.series)
    x = torch.from_numpy(batch.x).cuda()
    S(x)                                   # eager, also the warm-up before capture
    torch.cuda.synchronize()
    eager = [t.clone() for t in (S.periods, S.foldbins, S.snr)]
    F.profile_enable(False)                # no event records inside the capture
    launches = F.launch_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S(x)
    captured = F.launch_count() - launches
    assert captured > 0
    S.snr.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert F.launch_count() - launches == captured   # replays launch nothing from the host
    for a, b in zip(eager, (S.periods, S.foldbins, S.snr)):
        assert torch.equal(a, b)
    # new data in the same buffer: the replay searches it
    x2 = torch.from_numpy(synth.batch_uneven(7, 2 ** 15, 2 ** 17, seed=21, threads=4).x[::-1]
                          .copy()).cuda()
    x.copy_(x2)
    g.replay()
    torch.cuda.synchronize()
    S.check()
    got = S.snr.clone()
    S(x)
    torch.cuda.synchronize()
    assert torch.equal(got, S.snr)
    assert not torch.equal(got, eager[2])


def test_batch_with_series_too_short_for_any_transform(F):
    """A series with no 2-row transform contributes no trials; its neighbours are
    unaffected."""
    b = synth.batch_uneven(3, 2 ** 15, 2 ** 16, seed=31, threads=2)
    short = np.random.default_rng(3).standard_normal(500).astype(np.float32)
    x = np.concatenate([b.series_x(0), short, b.series_x(1)])
    s0, s1 = b.series[0], b.series[1]
    ser = [F.Series(0, s0.n, s0.tsamp, s0.pmin, s0.pmax, s0.bmin, s0.bmax),
           F.Series(s0.n, 500, 64e-6, 0.5, 3.0, 240, 260),
           F.Series(s0.n + 500, s1.n, s1.tsamp, s1.pmin, s1.pmax, s1.bmin, s1.bmax)]
    for budget in (1 << 40, 1):
        S = F.BatchSearcher(ser, b.widths, ws_budget=budget)
        assert S.trial_offsets[1] == S.trial_offsets[2]   # no trials for the short series
        S(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        S.check()
        _compare(S.series_result(0), _oracle(b, 0))
        ref = oracle.periodogram(b.series_x(1), s1.tsamp, s1.pmin, s1.pmax, s1.bmin, s1.bmax,
                                 b.widths)
        _compare(S.series_result(2), ref)


def test_dynamic_duty_cycle_segments(F):
    """One series, three period segments with more bins at longer periods (the paper's
    dynamic duty-cycle resolution): each segment equals its own oracle periodogram."""
    w = synth.plain_small()
    segs = [(1.0, 2.5, 240, 260), (2.5, 6.0, 360, 390), (6.0, 10.0, 480, 520)]
    S = F.SegmentSearcher(w.n, w.tsamp, segs, w.widths)
    S(torch.from_numpy(w.x).cuda())
    torch.cuda.synchronize()
    S.batch.check()
    for k, (pmin, pmax, bmin, bmax) in enumerate(segs):
        ref = oracle.periodogram(w.x, w.tsamp, pmin, pmax, bmin, bmax, w.widths)
        _compare(S.segment_result(k), ref)
    # the injected 2.345 s pulse is the strongest trial of the segment that holds it
    per, _, snr = (t.cpu().numpy() for t in S.segment_result(0))
    assert abs(per[snr.max(axis=1).argmax()] - 2.345) / 2.345 < 2e-3


def test_segments_long_profiles_full_size(F):
    """The Sec. 5.6 segments of the 2^23-sample survey series at full size, in the
    bench's launch configuration; the 2-20 s segment folds at 1000-1100 bins (scored one
    profile per warp with compensated prefix sums).  In every segment the deepest
    transforms (the most rows) and the first and last are compared with the FP64 oracle:
    periods and fold bins exactly, S/N within 1e-4, and within 3e-5 at 1000-1100 bins."""
    b = synth.survey_segments()
    S = F.SegmentSearcher(b.n, b.series[0].tsamp,
                          [(t.pmin, t.pmax, t.bmin, t.bmax) for t in b.series], b.widths)
    S(torch.from_numpy(b.x).cuda())
    torch.cuda.synchronize()
    S.batch.check()
    assert max(t.bmin for t in b.series) >= 1000
    for k, s in enumerate(b.series):
        pl = oracle.plan(s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax)
        sel = np.zeros(pl.n_transforms, bool)
        sel[np.argsort(-pl.tr_m)[:3]] = True
        sel[[0, pl.n_transforms - 1]] = True
        ref = oracle.periodogram(b.x, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax, b.widths,
                                 select=sel)
        rows = np.concatenate([np.arange(pl.tr_first_trial[t], pl.tr_first_trial[t] + pl.tr_kept[t])
                               for t in np.flatnonzero(sel)])
        per, fb, snr = (t.cpu().numpy() for t in S.segment_result(k))
        np.testing.assert_array_equal(per[rows], ref.periods)
        np.testing.assert_array_equal(fb[rows], ref.foldbins)
        err = np.abs(snr[rows].astype(np.float64) - ref.snr).max()
        assert err <= (3e-5 if s.bmin >= 1000 else 1e-4), (k, s.bmin, err)
