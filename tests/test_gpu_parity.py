"""GPU parity of every hot-path call against the CPU oracle, through libffa's C ABI.

Bars: FFA transforms bit-exact in FP32; downsampled series within 1e-6 of
sum_j |w_j x_j| per sample; S/N within 1e-4 (absolute) of the FP64 oracle; periods and
fold bins identical."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SNR_TOL = 1e-4
DS_TOL = 1e-6


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_03701_gb300 as ffa
    ffa.build()
    ffa.library()
    return ffa


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ----------------------------------------------------------------------------- FFA
TRANSFORM_SHAPES = [
    (1, 1), (1, 7), (2, 1), (2, 5), (3, 2), (5, 3), (7, 31), (8, 33), (13, 240), (64, 260),
    (100, 250), (111, 260), (112, 260), (127, 240), (128, 260), (129, 33), (257, 257),
    (1000, 240), (2684, 240), (5368, 250), (300, 1024), (17, 4096), (40000, 3), (2, 4096),
    (9683, 3), (4097, 7), (50, 4096), (100, 2048), (223, 260), (3000, 31), (1342, 520),
]


@pytest.mark.parametrize("m,p", TRANSFORM_SHAPES)
def test_transform_bit_exact(F, m, p):
    X = synth.normal_block(m, p, seed=m * 7919 + p)
    got = F.ffa_transform(dev(X)).cpu().numpy()
    ref = oracle.ffa(X)
    assert got.shape == ref.shape
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError("%d elements differ, first at %s" % (len(bad), bad[0]))


def test_transform_integer_brute_force(F):
    """Small-integer data: exact in any order, checked against direct path sums."""
    from tests.test_oracle_ffa import brute_force_fold
    m, p = 37, 11
    X = synth.small_integer_block(m, p, seed=3)
    got = F.ffa_transform(dev(X)).cpu().numpy().astype(np.float64)
    for s in range(m):
        np.testing.assert_array_equal(got[s], brute_force_fold(X, s))


# ----------------------------------------------------------------------- downsample
@pytest.mark.parametrize("n", [1, 7, 1000, 262144, 2 ** 23])
@pytest.mark.parametrize("f", [1.0, 2.0, 3.0, math.pi, 4.1666666666666667, 13.020833333333334,
                               1302.0833333333333])
def test_downsample(F, n, f):
    x = synth.white_noise(n, seed=n + int(f * 1000)).astype(np.float32)
    x[::97] += 5.0
    nout = int(math.floor(n / f))
    got = F.downsample(dev(x), f).cpu().numpy().astype(np.float64)
    assert len(got) == nout
    if nout == 0:
        return
    ref = oracle.downsample(x, f)
    scale = oracle.downsample(np.abs(x), f)      # sum_j |w_j x_j| per output sample
    err = np.abs(got - ref) / np.maximum(scale, 1e-30)
    assert err.max() <= DS_TOL, (err.max(), int(err.argmax()))


# ----------------------------------------------------------------------- boxcar S/N
@pytest.mark.parametrize("rows,cols,widths", [
    (1, 1, (1,)), (3, 7, (1, 2, 7)), (1000, 240, synth.WIDTHS_11), (777, 260, synth.WIDTHS_11),
    (300, 520, synth.WIDTHS_16), (50, 64, tuple(range(1, 33))),
    # the last half-warp size (Q = 35), the first warp-per-row size, and long profiles
    (41, 560, synth.WIDTHS_16), (41, 561, synth.WIDTHS_16), (20, 1024, synth.WIDTHS_16),
    (5, 4096, (1, 64, 1000)),
])
def test_boxcar_snr(F, rows, cols, widths):
    m = 500
    prof = (synth.normal_block(rows, cols, seed=rows + cols) * math.sqrt(m)).astype(np.float32)
    prof[:, 3 % cols] += 40.0
    std = math.sqrt(m * 1.0)
    got = F.boxcar_snr(dev(prof), widths, std).cpu().numpy().astype(np.float64)
    ref = oracle.boxcar_snr(prof.astype(np.float64), widths, std)
    assert np.abs(got - ref).max() <= SNR_TOL


# ---------------------------------------------------------------------- periodogram
def compare_periodogram(got, ref, rows=None):
    per, fb, snr = (t.cpu().numpy() for t in got)
    if rows is not None:
        per, fb, snr = per[rows], fb[rows], snr[rows]
    np.testing.assert_array_equal(per, ref.periods)
    np.testing.assert_array_equal(fb, ref.foldbins)
    err = np.abs(snr.astype(np.float64) - ref.snr)
    assert err.max() <= SNR_TOL, (err.max(), np.unravel_index(err.argmax(), err.shape))
    return float(err.max())


def test_periodogram_plain_small_full(F):
    """2^18 samples at 1 ms, periods 1-10 s, bins 240-260, 11 widths: every trial."""
    w = synth.plain_small()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    got = F.periodogram(dev(w.x), *args)
    ref = oracle.periodogram(w.x, *args)
    compare_periodogram(got, ref)
    # the injected 2.345 s pulse is the strongest trial
    best = ref.snr.max(axis=1)
    assert abs(ref.periods[best.argmax()] - 2.345) / 2.345 < 2e-3


def _sampled_rows(pl, sel):
    return np.concatenate([np.arange(pl.tr_first_trial[t], pl.tr_first_trial[t] + pl.tr_kept[t])
                           for t in np.flatnonzero(sel)])


def test_periodogram_survey_sampled(F):
    """2^23 samples at 64 us, periods 0.2-20 s: the full GPU periodogram, checked on a
    spread of transforms (every octave's deepest tree and a random sample)."""
    w = synth.survey()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    got = F.periodogram(dev(w.x), *args)
    torch.cuda.synchronize()
    pl = oracle.plan(w.n, *args[:-1])
    sel = np.zeros(pl.n_transforms, bool)
    sel[[0, 1, 20, pl.n_transforms - 1]] = True
    sel[synth.rng(9).choice(pl.n_transforms, 12, replace=False)] = True
    ref = oracle.periodogram(w.x, *args, select=sel)
    compare_periodogram(got, ref, _sampled_rows(pl, sel))
    # all S/N finite, periods strictly increasing over the whole periodogram
    per = got[0].cpu().numpy()
    assert np.all(np.diff(per) > 0)
    assert torch.isfinite(got[2]).all()


def _quantised(x):
    x64 = x.astype(np.float64)
    xn = (x64 - x64.mean()) / x64.std()
    f16 = xn.astype(np.float16)
    q = np.clip(np.rint(16 * xn), -128, 127).astype(np.int8)
    return f16, q


def test_periodogram_fp16_int8_storage(F):
    """Normalised series stored as FP16 and as int8 (q/16): FP32 accumulation error
    against the FP64 oracle run on the same dequantised values."""
    w = synth.plain_small()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    f16, q = _quantised(w.x)
    for stored, deq in ((f16, f16.astype(np.float32)), (q, q.astype(np.float32) / 16)):
        got = F.periodogram(dev(stored), *args)
        pl = oracle.plan(w.n, *args[:-1])
        sel = np.zeros(pl.n_transforms, bool)
        sel[::7] = True
        ref = oracle.periodogram(deq, *args, select=sel)
        compare_periodogram(got, ref, _sampled_rows(pl, sel))


def test_periodogram_no_transforms(F):
    """A series too short for any 2-row transform gives an empty periodogram."""
    x = synth.white_noise(300, seed=1).astype(np.float32)
    per, fb, snr = F.periodogram(dev(x), 1e-3, 0.5, 3.0, 240, 260, (1, 2))
    assert per.numel() == 0 and snr.shape == (0, 2)


def test_periodogram_ragged_small(F):
    """Odd sizes: few rows per transform, integer and non-integer factors."""
    for n, tsamp, pmin, pmax, bmin, bmax, widths in [
        (5000, 1e-3, 0.5, 3.0, 40, 44, (1, 2, 3)),
        (12345, 1e-3, 0.1, 0.9, 50, 99, (1, 2, 4, 8, 16, 32, 49)),
        (77777, 2e-3, 0.2, 5.0, 20, 23, (1, 3, 9, 19)),
    ]:
        x = synth.white_noise(n, seed=n).astype(np.float32)
        got = F.periodogram(dev(x), tsamp, pmin, pmax, bmin, bmax, widths)
        ref = oracle.periodogram(x, tsamp, pmin, pmax, bmin, bmax, widths)
        compare_periodogram(got, ref)


@pytest.mark.parametrize("bins,widths", [
    ((545, 560), (1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144)),   # half-warp S/N, Q = 35
    ((983, 1065), (1, 2, 4, 8, 16, 32, 64, 128, 200)),       # the paper's context bins
])
def test_periodogram_long_profiles(F, bins, widths):
    """Base periods above the half-warp S/N limit score stored rows one warp each;
    sampled transforms of a 2^20-sample series at 64 us, P 1-10 s."""
    n, tsamp, pmin, pmax = 2 ** 20, 64e-6, 1.0, 10.0
    x = synth.make_series(n, tsamp, seed=bins[0], pulses=[synth.Pulse(2.2, 0.03, 12.0, 0.3)])
    args = (tsamp, pmin, pmax, bins[0], bins[1], widths)
    got = F.periodogram(dev(x), *args)
    pl = oracle.plan(n, *args[:-1])
    sel = np.zeros(pl.n_transforms, bool)
    sel[[0, pl.n_transforms - 1, int(np.argmax(pl.tr_m))]] = True
    sel[synth.rng(bins[0]).choice(pl.n_transforms, 5, replace=False)] = True
    ref = oracle.periodogram(x, *args, select=sel)
    compare_periodogram(got, ref, _sampled_rows(pl, sel))


@pytest.mark.parametrize("rows,cols,widths", [
    (300, 250, synth.WIDTHS_11), (77, 17, (1, 2, 3, 16)), (41, 560, synth.WIDTHS_16),
    (20, 1024, synth.WIDTHS_16),
])
def test_boxcar_snr_zero_mean(F, rows, cols, widths):
    """The zero-mean boxcar template (zero sum, unit square sum) on both S/N paths,
    against the FP64 oracle, on profiles with a common offset (which it ignores).  The
    offset is kept modest: sums are FP32, and an offset of c per bin costs an absolute
    error of about c * cols * 2^-24 in every prefix sum, with either template."""
    prof = synth.normal_block(rows, cols, seed=cols) + np.float32(0.5)
    got = F.boxcar_snr(dev(prof), widths, 2.5, zero_mean=True).cpu().numpy()
    ref = oracle.boxcar_snr(prof.astype(np.float64), widths, 2.5, zero_mean=True)
    assert np.abs(got - ref).max() <= SNR_TOL


def test_periodogram_zero_mean_full(F):
    """plain_small scored with the zero-mean boxcar: every trial against the oracle."""
    w = synth.plain_small()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    got = F.periodogram(dev(w.x), *args, zero_mean=True)
    ref = oracle.periodogram(w.x, *args, zero_mean=True)
    compare_periodogram(got, ref)


def test_status_and_launch_accounting(F):
    w = synth.plain_small()
    s = F.Searcher(w.n, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    before = F.launch_count()
    s(dev(w.x))
    s.check()
    assert F.launch_count() > before


def test_host_buffer_entry_point(F):
    w = synth.plain_small()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    per, fb, snr = F.periodogram_host(w.x, *args)
    d = F.periodogram(dev(w.x), *args)
    np.testing.assert_array_equal(per, d[0].cpu().numpy())
    np.testing.assert_array_equal(fb, d[1].cpu().numpy())
    np.testing.assert_array_equal(snr, d[2].cpu().numpy())


# ------------------------------------------------------------------------ normalise
@pytest.mark.parametrize("n", [1, 1000, 262144, 2 ** 23])
def test_normalise(F, n):
    """Whole-series normalisation (Sec. 3.1, 5.2): FP64 statistics within 1e-12 of the
    oracle; float output within rounding of the oracle's FP64 value; half and int8 codes
    identical to the same FP64 decision taken with the device's mean and deviation."""
    x = (synth.white_noise(n, seed=n) * 3.0 + 7.0).astype(np.float32)
    x[::101] += 20.0
    om, osd, ref = oracle.normalise(x)
    out, m, s = F.normalise(dev(x))
    assert m == pytest.approx(om, rel=1e-12, abs=1e-12)
    assert s == pytest.approx(osd, rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(out.cpu().numpy(), ref.astype(np.float32), rtol=2.5e-7, atol=1e-9)
    h, m2, s2 = F.normalise(dev(x), torch.float16)
    q, m3, s3 = F.normalise(dev(x), torch.int8)
    assert (m2, s2) == (m, s) and (m3, s3) == (m, s)      # deterministic statistics
    v = (x.astype(np.float64) - m) / s if s > 0 else np.zeros(n)
    np.testing.assert_array_equal(h.cpu().numpy(), v.astype(np.float16))
    np.testing.assert_array_equal(q.cpu().numpy(), np.clip(np.rint(16 * v), -128, 127).astype(np.int8))


def test_normalised_int8_periodogram_chain(F):
    """normalise -> int8 storage -> periodogram, all on the device: S/N of the injected
    pulse within 0.5 of the FP32 periodogram of the same series."""
    w = synth.plain_small()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    x = dev(w.x)
    xf, _, _ = F.normalise(x)
    xq, _, _ = F.normalise(x, torch.int8)
    sf = F.periodogram(xf, *args)[2].max().item()
    sq = F.periodogram(xq, *args)[2].max().item()
    assert sf > 12 and abs(sf - sq) < 0.5
