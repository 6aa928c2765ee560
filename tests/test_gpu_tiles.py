"""Tile shapes of the persistent FFA launch (sub-tree rows, merge levels per top pass,
rows per top-pass item).  Every shape must give the same periodogram bit for bit (the
merges and the S/N of each row do not depend on how rows are grouped into work items),
and the tuner must pick one of its candidates."""
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


def test_tiles_bit_identical_and_match_oracle(F):
    w = synth.plain_small()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    x = torch.from_numpy(w.x).cuda()
    base = [t.clone() for t in F.Searcher(w.n, *args)(x)]
    auto = F.periodogram_plan(w.n, *args).tiles
    shapes = F.tile_candidates(auto) + [F.Tiles(8, 1, 4), F.Tiles(3, 1, 1), F.Tiles(24, 2, 16)]
    for t in shapes:
        got = F.Searcher(w.n, *args, tiles=t)(x)
        torch.cuda.synchronize()
        for a, b in zip(base, got):
            assert torch.equal(a, b), t
    ref = oracle.periodogram(w.x, *args)
    assert np.abs(base[2].cpu().numpy().astype(np.float64) - ref.snr).max() <= 1e-4


def test_batch_tiles_bit_identical(F):
    b = synth.batch_uneven(4, 2 ** 15, 2 ** 16, seed=8, threads=2)
    ser = [F.Series(s.offset, s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax) for s in b.series]
    x = torch.from_numpy(b.x).cuda()
    base = [t.clone() for t in F.BatchSearcher(ser, b.widths)(x)]
    got = F.BatchSearcher(ser, b.widths, tiles=F.Tiles(12, 2, 8))(x)
    torch.cuda.synchronize()
    for a, c in zip(base, got):
        assert torch.equal(a, c)


def test_tuner_picks_a_candidate(F):
    w = synth.plain_small()
    x = torch.from_numpy(w.x).cuda()
    best, timings = F.tune_periodogram(x, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths,
                                       repeats=2)
    assert best in [t for t, _ in timings] and len(timings) >= 2
    assert all(ms > 0 for _, ms in timings)
