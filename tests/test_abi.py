"""Host-side checks of libffa that need no GPU: the library loads, exports every
symbol include/ffa.h declares, plans searches exactly like the oracle's reading of
Sec. 5.3, and rejects bad arguments before launching anything."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2004_03701_gb300 as ffa
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ffa.build()
    return ffa.library()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(ffa_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_symbols_exported(lib):
    names = declared_functions()
    assert "ffa_periodogram" in names and "ffa_transform" in names
    for name in names:
        assert hasattr(lib, name), name


def test_version(lib):
    assert b"sm_103a" in lib.ffa_version()


@pytest.mark.parametrize("args", [
    (262144, 1e-3, 1.0, 10.0, 240, 260),
    (2 ** 23, 64e-6, 0.2, 20.0, 240, 260),
    (2 ** 21, 64e-6, 0.1, 10.0, 480, 520),
    (100_000, 1e-3, 0.5, 3.0, 40, 44),
    (5000, 1e-3, 0.5, 3.0, 40, 44),
    (2 ** 23, 64e-6, 1.0, 120.0, 983, 1065),
])
def test_plan_matches_oracle(lib, args):
    widths = (1, 2, 3, 4, 6, 9, 13, 19, 28)
    info = ffa.periodogram_plan(*args, widths)
    pl = oracle.plan(*args)
    assert info.ntrials == pl.n_trials
    assert info.noctaves == pl.n_octaves
    assert info.ntransforms == pl.n_transforms
    assert info.downsampled_samples == int(pl.oct_len.sum())
    assert info.folded_samples == int((pl.tr_m * pl.tr_p).sum())
    assert info.max_rows == (int(pl.tr_m.max()) if pl.n_transforms else 0)
    assert info.workspace_bytes > 0 and info.host_workspace_bytes >= info.workspace_bytes


@pytest.mark.parametrize("bad", [
    dict(n=0), dict(tsamp=0.0), dict(pmin=20.0), dict(bmin=1), dict(bmax=200),
    dict(pmin=0.1),                     # first downsampling factor below 1
    dict(widths=(1, 1)), dict(widths=(0, 2)), dict(widths=(1, 240)), dict(widths=()),
])
def test_plan_rejects_bad_arguments(lib, bad):
    a = dict(n=262144, tsamp=1e-3, pmin=1.0, pmax=10.0, bmin=240, bmax=260, widths=(1, 2, 4))
    a.update(bad)
    with pytest.raises(ffa.FFAError) as e:
        ffa.periodogram_plan(a["n"], a["tsamp"], a["pmin"], a["pmax"], a["bmin"], a["bmax"],
                             a["widths"])
    assert e.value.status == 1


def test_other_calls_reject_bad_arguments(lib):
    sz = ctypes.c_size_t()
    assert lib.ffa_transform_workspace(0, 5, ctypes.byref(sz)) == 1
    assert lib.ffa_transform_workspace(5, 5000, ctypes.byref(sz)) == 5
    assert lib.ffa_transform_workspace(5, 5, None) == 1
    assert lib.ffa_downsample_workspace(0, ctypes.byref(sz)) == 1
    n_out = ctypes.c_int64()
    assert lib.ffa_downsample(None, 10, 2.0, None, 5, ctypes.byref(n_out), None, 0, None) == 1
    fake = ctypes.c_void_p(256)   # never dereferenced: rejected on the host first
    assert lib.ffa_downsample(fake, 10, 0.5, fake, 5, ctypes.byref(n_out), fake, 1 << 20,
                              None) == 1
    assert lib.ffa_downsample(fake, 100, 3.0, fake, 5, ctypes.byref(n_out), fake, 1 << 20,
                              None) == 2
    assert n_out.value == 33
    w = np.array([1, 2], np.int32)
    assert lib.ffa_boxcar_snr(fake, 4, 8, w.ctypes.data, 2, 0.0, fake, None) == 1
    assert lib.ffa_boxcar_snr(fake, 4, 8, w.ctypes.data, 0, 1.0, fake, None) == 1
    assert lib.ffa_transform(fake, 4, 8, fake, fake, 1 << 20, None) == 1  # in/out overlap
    assert len(lib.ffa_last_error()) > 0
    assert lib.ffa_check(None, None) == 1


def test_kernel_kinds(lib):
    names = ffa.kernel_names()
    assert "ffa_bottom" in names and "ffa_top" in names and "downsample" in names
    assert "median_build" in names and "median_query" in names and "peaks" in names


def test_running_median_rejects_bad_arguments(lib):
    sz = ctypes.c_size_t()
    assert lib.ffa_running_median_workspace(0, ctypes.byref(sz)) == 1
    assert lib.ffa_running_median_workspace(1 << 31, ctypes.byref(sz)) == 1
    assert lib.ffa_running_median_workspace(5, None) == 1
    assert lib.ffa_running_median_workspace(2 ** 23, ctypes.byref(sz)) == 0
    need = sz.value
    assert 16 * 2 ** 23 <= need <= 17 * 2 ** 23
    fake = ctypes.c_void_p(256)   # never dereferenced: rejected on the host first
    n = 2 ** 23
    call = lib.ffa_running_median
    assert call(None, n, 15, fake, None, fake, need, None) == 1
    assert call(fake, n, 15, None, None, fake, need, None) == 1       # no output
    assert call(fake, n, 16, fake, None, fake, need, None) == 1       # even width
    assert call(fake, n, 0, fake, None, fake, need, None) == 1
    assert call(fake, n, -3, fake, None, fake, need, None) == 1
    assert call(fake, 0, 15, fake, None, fake, need, None) == 1
    assert call(fake, n, 15, fake, fake, fake, need, None) == 1       # med == y
    assert call(fake, n, 15, fake, None, ctypes.c_void_p(260), need, None) == 1  # alignment
    assert call(fake, n, 15, fake, None, fake, need - 1, None) == 2   # workspace too small
    assert len(lib.ffa_last_error()) > 0


def test_find_peaks_rejects_bad_arguments(lib):
    o = ffa._PeakOpts()
    lib.ffa_peak_opts_default(ctypes.byref(o))
    assert (o.dzseg, o.nsigma, o.clrad, o.degree, o.min_seg, o.max_segments) == \
        (5.0, 6.0, 1.0, 2, 8, 65536)
    sz = ctypes.c_size_t()
    assert lib.ffa_find_peaks_workspace(662440, 11, None, ctypes.byref(sz)) == 0
    need = sz.value
    assert need >= 12 * 662440 * 11
    assert lib.ffa_find_peaks_workspace(0, 11, None, ctypes.byref(sz)) == 1
    assert lib.ffa_find_peaks_workspace(10, 65, None, ctypes.byref(sz)) == 1
    for field, bad in (("dzseg", 0.0), ("clrad", -1.0), ("degree", 7), ("degree", -1),
                       ("min_seg", 0), ("max_segments", 0)):
        b = ffa._PeakOpts()
        lib.ffa_peak_opts_default(ctypes.byref(b))
        setattr(b, field, bad)
        assert lib.ffa_find_peaks_workspace(10, 2, ctypes.byref(b), ctypes.byref(sz)) == 1, field
    fake = ctypes.c_void_p(256)   # never dereferenced: rejected on the host first
    call = lib.ffa_find_peaks
    n = 662440
    assert call(None, fake, n, 11, 537.0, None, fake, 10, fake, fake, need, None) == 1
    assert call(fake, fake, n, 11, 0.0, None, fake, 10, fake, fake, need, None) == 1   # tobs
    assert call(fake, fake, n, 11, 537.0, None, None, 10, fake, fake, need, None) == 1  # no out
    assert call(fake, fake, n, 11, 537.0, None, fake, -1, fake, fake, need, None) == 1
    assert call(fake, fake, n, 11, 537.0, None, fake, 10, fake, ctypes.c_void_p(264), need,
                None) == 1                                                            # alignment
    assert call(fake, fake, n, 11, 537.0, None, fake, 10, fake, fake, need - 1, None) == 2


def test_median_width():
    assert ffa.median_width(1.0, 64e-6) == 15625
    assert ffa.median_width(0.5, 1e-3) == 501
    assert ffa.median_width(0.01, 1e-3) == 11
    assert ffa.median_width(1e-6, 1e-3) == 1


def test_width_sets_fit_the_plan(lib):
    for wl in (synth.WIDTHS_11, synth.WIDTHS_16):
        info = ffa.periodogram_plan(2 ** 21, 64e-6, 0.1, 10.0, 480, 520, wl)
        assert info.nwidths == len(wl)


def _batch_series(nseries=6, seed=11):
    b = synth.batch_uneven(nseries, 2 ** 15, 2 ** 17, seed=seed, threads=1)
    return b, [ffa.Series(s.offset, s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax)
               for s in b.series]


def test_batch_plan_matches_per_series_oracle_plans(lib):
    b, ser = _batch_series()
    info, offs = ffa.batch_plan(ser, b.widths)
    plans = [oracle.plan(s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax) for s in ser]
    assert list(np.diff(offs)) == [pl.n_trials for pl in plans]
    assert offs[0] == 0 and info.ntrials == offs[-1]
    assert info.ntransforms == sum(pl.n_transforms for pl in plans)
    assert info.folded_samples == sum(int((pl.tr_m * pl.tr_p).sum()) for pl in plans)
    assert info.input_samples == sum(s.n for s in ser)


def test_batch_chunks_follow_the_budget(lib):
    b, ser = _batch_series()
    one, offs1 = ffa.batch_plan(ser, b.widths, ws_budget=1 << 40)
    each, offs2 = ffa.batch_plan(ser, b.widths, ws_budget=1)
    assert one.nchunks == 1 and each.nchunks == len(ser)
    assert np.array_equal(offs1, offs2)
    alone = [ffa.periodogram_plan(s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax, b.widths)
             for s in ser]
    # one series per chunk: the workspace of the largest series searched alone
    assert each.workspace_bytes == max(a.workspace_bytes for a in alone)
    assert one.workspace_bytes >= each.workspace_bytes
    mid, _ = ffa.batch_plan(ser, b.widths, ws_budget=2 * each.workspace_bytes)
    assert 1 < mid.nchunks < len(ser)


def test_batch_rejects_bad_series(lib):
    b, ser = _batch_series(3)
    bad = list(ser)
    bad[1] = ffa.Series(-5, ser[1].n, ser[1].tsamp, ser[1].pmin, ser[1].pmax, 240, 260)
    with pytest.raises(ffa.FFAError):
        ffa.batch_plan(bad, b.widths)
    bad = list(ser)
    bad[2] = ffa.Series(ser[2].offset, ser[2].n, ser[2].tsamp, ser[2].pmin, ser[2].pmax, 40, 44)
    with pytest.raises(ffa.FFAError):   # width 63 is not below bmin = 40
        ffa.batch_plan(bad, b.widths)
    with pytest.raises(ffa.FFAError):
        ffa.batch_plan([], b.widths)


def test_tiles_cap_the_plan(lib):
    args = (2 ** 23, 64e-6, 0.2, 20.0, 240, 260, synth.WIDTHS_11)
    auto = ffa.periodogram_plan(*args)
    assert auto.tiles.subtree_rows >= 2 and 1 <= auto.tiles.top_levels <= 3
    for t in ffa.tile_candidates(auto.tiles) + [ffa.Tiles(16, 1, 8), ffa.Tiles(0, 2, 0)]:
        info = ffa.periodogram_plan(*args, tiles=t)
        # the same search, only the work items differ
        assert (info.ntrials, info.ntransforms, info.folded_samples) == \
            (auto.ntrials, auto.ntransforms, auto.folded_samples)
        for got, cap in zip((info.tiles.subtree_rows, info.tiles.top_levels, info.tiles.top_rows),
                            (t.subtree_rows, t.top_levels, t.top_rows)):
            assert cap == 0 or got <= cap


@pytest.mark.parametrize("bad", [ffa.Tiles(1, 0, 0), ffa.Tiles(2000, 0, 0), ffa.Tiles(0, 4, 0),
                                 ffa.Tiles(0, -1, 0), ffa.Tiles(0, 0, 129)])
def test_tiles_rejected(lib, bad):
    with pytest.raises(ffa.FFAError) as e:
        ffa.periodogram_plan(262144, 1e-3, 1.0, 10.0, 240, 260, (1, 2, 4), tiles=bad)
    assert e.value.status == 1


def test_tile_classes_apply_per_transform(lib):
    """A class table changes only the work items of the transforms it admits: the first
    matching class wins, its sizes cap that class's tiles, other classes keep theirs."""
    args = (2 ** 23, 64e-6, 0.2, 20.0, 240, 260, (1, 2, 3, 4, 6, 9, 13, 19, 28, 42, 63))
    auto = ffa.periodogram_plan(*args)
    base = ffa.periodogram_plan(*args, tiles=ffa.tile_classes())
    assert (base.ntrials, base.folded_samples) == (auto.ntrials, auto.folded_samples)
    # all-automatic classes: each class's effective tiles are within the plan-wide ones
    nonempty = [c for c in base.tiles.classes if c.subtree_rows]
    assert len(nonempty) >= 4
    for c in nonempty:
        assert c.subtree_rows <= auto.tiles.subtree_rows and c.top_levels <= auto.tiles.top_levels
    t = ffa.tile_classes().with_class(3, subtree_rows=16, top_levels=1, top_rows=8)
    info = ffa.periodogram_plan(*args, tiles=t)
    assert (info.ntrials, info.folded_samples) == (auto.ntrials, auto.folded_samples)
    c3 = info.tiles.classes[3]
    assert (c3.subtree_rows, c3.top_levels, c3.top_rows) == (16, 1, 8)
    for i, (a, b) in enumerate(zip(base.tiles.classes, info.tiles.classes)):
        if i != 3:
            assert a == b
    # a transform matches the first class that admits it: an earlier catch-all wins
    first = ffa.Tiles(classes=(ffa.TileClass(0, 0, 16, 1, 8),) + ffa.tile_classes().classes[:7])
    info = ffa.periodogram_plan(*args, tiles=first)
    assert info.tiles.classes[0].subtree_rows == 16
    assert all(c.subtree_rows == 0 for c in info.tiles.classes[1:])


@pytest.mark.parametrize("bad", [ffa.TileClass(-1, 0, 0, 0, 0), ffa.TileClass(0, -5, 0, 0, 0),
                                 ffa.TileClass(0, 0, 1, 0, 0), ffa.TileClass(0, 0, 0, 4, 0),
                                 ffa.TileClass(0, 0, 0, 0, 200)])
def test_tile_classes_rejected(lib, bad):
    with pytest.raises(ffa.FFAError) as e:
        ffa.periodogram_plan(262144, 1e-3, 1.0, 10.0, 240, 260, (1, 2, 4),
                             tiles=ffa.Tiles(classes=(bad,)))
    assert e.value.status == 1
    with pytest.raises(ValueError):
        ffa.periodogram_plan(262144, 1e-3, 1.0, 10.0, 240, 260, (1, 2, 4),
                             tiles=ffa.Tiles(classes=(ffa.TileClass(),) * 9))


def test_batch_tiles_rejected_and_accepted(lib):
    b, ser = _batch_series(2)
    with pytest.raises(ffa.FFAError):
        ffa.batch_plan(ser, b.widths, tiles=ffa.Tiles(0, 9, 0))
    info, offs = ffa.batch_plan(ser, b.widths, tiles=ffa.Tiles(12, 2, 8))
    ref, offs0 = ffa.batch_plan(ser, b.widths)
    assert np.array_equal(offs, offs0) and info.ntrials == ref.ntrials


def test_plan_arithmetic_counts(lib):
    """The plan's operation counts against an independent count over the oracle's plan:
    an n-row FFA produces n rows at its top node plus those of its two halves."""
    from functools import lru_cache

    @lru_cache(None)
    def rows(n):
        return 0 if n < 2 else n + rows(n // 2) + rows(n - n // 2)

    for args, widths in [((2 ** 23, 64e-6, 0.2, 20.0, 240, 260), synth.WIDTHS_11),
                         ((100_000, 1e-3, 0.5, 3.0, 40, 44), (1, 2, 3))]:
        info = ffa.periodogram_plan(*args, widths)
        pl = oracle.plan(*args)
        adds = sum(rows(int(m)) * int(p) for m, p in zip(pl.tr_m, pl.tr_p))
        ops = sum(int(k) * int(p) * (1 + 2 * len(widths)) for k, p in zip(pl.tr_kept, pl.tr_p))
        assert info.ffa_adds == adds and info.snr_ops == ops


def test_plan_options_boxcar_template(lib):
    args = (262144, 1e-3, 1.0, 10.0, 240, 260, (1, 2, 4))
    plain = ffa.periodogram_plan(*args)
    zm = ffa.periodogram_plan(*args, zero_mean=True)
    assert zm.ntrials == plain.ntrials and zm.workspace_bytes == plain.workspace_bytes
    opts = ffa._PlanOpts(0, 0, 0, 7)
    info = ffa._PlanInfo()
    w = np.array(args[-1], np.int32)
    st = lib.ffa_periodogram_plan_opts(*args[:-1], w.ctypes.data_as(ctypes.c_void_p), len(w),
                                       ctypes.cast(ctypes.byref(opts), ctypes.c_void_p),
                                       ctypes.byref(info))
    assert st == 1 and b"boxcar" in lib.ffa_last_error()


def test_downsample_length(lib):
    """The output length query: floor(n / f) complete windows (reading c5), for the
    binding to size its output; bad arguments rejected."""
    n_out = ctypes.c_int64()
    for n, f in [(1000, 1.0), (1000, 3.0), (1000, 3.7), (2 ** 23, 13.02), (5, 6.0)]:
        assert lib.ffa_downsample_length(n, f, ctypes.byref(n_out)) == 0
        assert n_out.value == int(np.floor(n / f)), (n, f)
    assert lib.ffa_downsample_length(0, 2.0, ctypes.byref(n_out)) == 1
    assert lib.ffa_downsample_length(10, 0.5, ctypes.byref(n_out)) == 1
    assert lib.ffa_downsample_length(10, float("nan"), ctypes.byref(n_out)) == 1
    assert lib.ffa_downsample_length(10, 2.0, None) == 1
