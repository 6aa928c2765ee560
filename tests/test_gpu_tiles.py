"""Tile shapes of the persistent FFA launch (sub-tree rows, merge levels per top pass,
rows per top-pass item).  Every shape must give the same periodogram bit for bit (the
merges and the S/N of each row do not depend on how rows are grouped into work items),
and the tuners must pick one of their candidates.  Tile classes (per-(m, p) shapes inside
one launch) are covered the same way: every candidate of every class of the survey
search, and a mixed table, against the automatic shape."""
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


def test_every_class_shape_bit_identical(F):
    """The survey search (2^23 samples, 1155 transforms of m = 26 .. 2684 rows) with each
    candidate of each tile class in turn equals the automatic search bit for bit."""
    w = synth.survey()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    x = torch.from_numpy(w.x).cuda()
    base = [t.clone() for t in F.Searcher(w.n, *args)(x)]
    table = F.tile_classes()
    eff = F.periodogram_plan(w.n, *args, tiles=table).tiles
    tried = 0
    for i, c in enumerate(eff.classes):
        for f in F.class_candidates(c):
            got = F.Searcher(w.n, *args, tiles=table.with_class(i, **f))(x)
            torch.cuda.synchronize()
            for a, b in zip(base, got):
                assert torch.equal(a, b), (i, f)
            tried += 1
    assert tried >= 40
    # a mixed table: odd sizes in several classes at once
    mixed = table.with_class(1, subtree_rows=13, top_levels=1, top_rows=5) \
                 .with_class(4, subtree_rows=37, top_levels=2, top_rows=19) \
                 .with_class(6, top_rows=3)
    got = F.Searcher(w.n, *args, tiles=mixed)(x)
    torch.cuda.synchronize()
    for a, b in zip(base, got):
        assert torch.equal(a, b)


def test_class_tuner_returns_a_faster_or_equal_table(F):
    w = synth.plain_small()
    x = torch.from_numpy(w.x).cuda()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    best, log = F.tune_periodogram_classes(x, *args, repeats=2)
    assert len(best.classes) == len(F.CLASS_M_BOUNDS) and log[0][0] == -1
    assert min(ms for _, _, ms in log) <= log[0][2]
    base = F.Searcher(w.n, *args)(x)
    got = F.Searcher(w.n, *args, tiles=best)(x)
    torch.cuda.synchronize()
    for a, b in zip(base, got):
        assert torch.equal(a, b)
