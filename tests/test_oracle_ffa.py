"""Pins of the oracle's FFA (Sec. 2 of the paper) against facts that do not come
from the oracle itself: the folding transform's definition evaluated by brute force,
the Fig. 1 worked example, closed forms for the s = 0 and s = m-1 rows, an
independent breadth-first (Staelin) evaluation for power-of-two m, and invariants
(sum conservation, linearity, bounded path deviation, b in {0, 1})."""
import math

import numpy as np
import pytest

import oracle
import synth


# --- integration paths, derived here from the merge rule on row indices only -----

def _nint(a, d):
    return (2 * a + d) // (2 * d)


def path(m, s):
    """Column offset of each input row on the integration path with drift s:
    head rows follow the head's path with drift i, tail rows the tail's path with
    drift j, started i + b bins further right (Sec. 2.2)."""
    if m == 1:
        return [0]
    mh = m // 2
    mt = m - mh
    i = _nint((mh - 1) * s, m - 1)
    j = _nint((mt - 1) * s, m - 1)
    b = s - i - j
    return path(mh, i) + [i + b + v for v in path(mt, j)]


def brute_force_fold(X, s):
    """Sum of the rows along one integration path: O(m p) per output row, O(p m^2)
    for the whole transform (Sec. 2.1)."""
    m, p = X.shape
    sh = path(m, s)
    out = np.zeros(p, np.float64)
    for r in range(m):
        out += np.roll(X[r].astype(np.float64), -sh[r])  # out[x] += X[r][(x + sh) mod p]
    return out


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8, 9, 13, 16, 17, 31, 32, 33, 40])
@pytest.mark.parametrize("p", [1, 2, 3, 6, 17])
def test_ffa_matches_brute_force_fold(m, p):
    X = synth.small_integer_block(m, p, seed=1000 * m + p)
    F = oracle.ffa(X)                      # float32 path: exact on small integers
    F64 = oracle.ffa(X.astype(np.float64))
    for s in range(m):
        ref = brute_force_fold(X, s)
        np.testing.assert_array_equal(F[s].astype(np.float64), ref)
        np.testing.assert_array_equal(F64[s], ref)


def test_fig1_worked_example(paper_values):
    """Fig. 1: a width-1 pulse train at initial phase 1 drifting 4 bins over 8 rows
    of 6 samples folds into a single peak at row 4, column 1."""
    g = paper_values["fig1_folding_transform"]
    m, p, phase, s = g["m"], g["p"], g["phase"], g["drift"]
    period = p + s / (m - 1)                # samples; drift s over m-1 periods
    X = np.zeros(m * p, np.float32)
    for k in range(m):
        X[int(math.floor(phase + k * period + 0.5))] = 1.0
    F = oracle.ffa(X.reshape(m, p))
    r, c = np.unravel_index(np.argmax(F), F.shape)
    assert (r, c) == (g["peak_row"], g["peak_col"])
    assert F[r, c] == g["peak_value"]
    assert np.count_nonzero(F == F.max()) == 1


@pytest.mark.parametrize("m,p", [(2, 5), (3, 4), (7, 9), (64, 33), (100, 250), (257, 7)])
def test_row_zero_is_plain_fold(m, p):
    """s = 0 is folding at exactly p samples: f_j = sum_i x_{pi+j} (Sec. 3.4)."""
    X = synth.small_integer_block(m, p, seed=7 + m)
    F = oracle.ffa(X)
    np.testing.assert_array_equal(F[0], X.sum(axis=0))


@pytest.mark.parametrize("m,p", [(2, 5), (3, 4), (7, 9), (64, 33), (100, 250), (257, 7)])
def test_last_row_is_unit_slope_diagonal(m, p):
    """s = m-1 drifts exactly one bin per row: F_{m-1}[x] = sum_r X_r[(x + r) mod p]."""
    X = synth.small_integer_block(m, p, seed=11 + m)
    F = oracle.ffa(X)
    ref = np.zeros(p)
    for r in range(m):
        ref += np.roll(X[r].astype(np.float64), -r)
    np.testing.assert_array_equal(F[m - 1].astype(np.float64), ref)


def test_two_rows_textbook():
    X = synth.small_integer_block(2, 11, seed=3)
    F = oracle.ffa(X)
    np.testing.assert_array_equal(F[0], X[0] + X[1])
    np.testing.assert_array_equal(F[1], X[0] + np.roll(X[1], -1))


def test_one_row_identity():
    X = synth.normal_block(1, 13, seed=5)
    np.testing.assert_array_equal(oracle.ffa(X), X)


def staelin_breadth_first(X):
    """Independent bottom-up evaluation for m = 2^k (Sec. 2.2, last paragraph):
    transform all 2-row blocks, then all 4-row blocks, ... in place of recursion."""
    m, p = X.shape
    level = [X[r:r + 1].copy() for r in range(m)]   # 1-row blocks are their transforms
    while len(level) > 1:
        nxt = []
        for a in range(0, len(level), 2):
            H, T = level[a], level[a + 1]
            n = 2 * H.shape[0]
            out = np.empty((n, p), X.dtype)
            for s in range(n):
                i = _nint((n // 2 - 1) * s, n - 1)
                j = i
                b = s - 2 * i
                out[s] = H[i] + np.roll(T[j], -(i + b))
            nxt.append(out)
        level = nxt
    return level[0]


@pytest.mark.parametrize("k,p", [(1, 7), (3, 6), (5, 33), (7, 250), (8, 13)])
def test_power_of_two_matches_breadth_first_bitwise(k, p):
    X = synth.normal_block(2 ** k, p, seed=100 + k)
    np.testing.assert_array_equal(oracle.ffa(X), staelin_breadth_first(X))


@pytest.mark.parametrize("m", [5, 37, 100, 263, 1000])
def test_sum_conservation(m):
    """Every folded profile adds each input sample exactly once."""
    p = 29
    X = synth.small_integer_block(m, p, seed=m)
    F = oracle.ffa(X).astype(np.float64)
    np.testing.assert_array_equal(F.sum(axis=1), np.full(m, X.astype(np.float64).sum()))


def test_linearity():
    m, p = 45, 19
    A = synth.small_integer_block(m, p, seed=1)
    B = synth.small_integer_block(m, p, seed=2)
    np.testing.assert_array_equal(oracle.ffa(A + 2 * B), oracle.ffa(A) + 2 * oracle.ffa(B))


def test_paths_are_near_straight_lines(paper_values):
    """The integration path of drift s starts at 0, ends at s, never moves left, and
    stays within half a bin per tree level of the straight line r s / (m-1); the
    phase jump b is 0 or 1 (Sec. 2.2)."""
    allowed_b = set(paper_values["merge_phase_jump"]["allowed_values"])
    for m in range(2, 160):
        depth = math.ceil(math.log2(m))
        for s in range(m):
            sh = np.array(path(m, s))
            assert sh[0] == 0 and sh[-1] == s
            assert np.all(np.diff(sh) >= 0)
            assert np.abs(sh - np.arange(m) * s / (m - 1)).max() <= 0.5 * depth + 1e-12
            i, j, b = oracle.ffa_split(m, s)
            assert b in allowed_b
            assert (i, j, b) == (_nint((m // 2 - 1) * s, m - 1),
                                 _nint((m - m // 2 - 1) * s, m - 1),
                                 s - _nint((m // 2 - 1) * s, m - 1)
                                 - _nint((m - m // 2 - 1) * s, m - 1))


def test_fp32_and_fp64_agree_to_rounding():
    m, p = 300, 41
    X = synth.normal_block(m, p, seed=9)
    F32 = oracle.ffa(X).astype(np.float64)
    F64 = oracle.ffa(X.astype(np.float64))
    depth = math.ceil(math.log2(m))
    bound = depth * np.finfo(np.float32).eps * np.abs(X).sum(axis=0).max() * 2
    assert np.abs(F32 - F64).max() <= bound


def test_drifting_pulse_train_peaks_at_its_drift():
    """Width-1 pulses drifting s bins over m = 2^k rows (as in Fig. 1) fold into a
    maximum at row s and the initial phase column."""
    rng = synth.rng(77)
    for _ in range(20):
        m = 2 ** int(rng.integers(2, 6))
        p = int(rng.integers(m + 2, 3 * m))
        s = int(rng.integers(0, m))
        phase = int(rng.integers(0, p))
        X = np.zeros((m, p), np.float32)
        for r in range(m):
            X[r, int((phase + math.floor(r * s / (m - 1) + 0.5)) % p)] += 1.0
        F = oracle.ffa(X)
        assert F[s, phase] == F.max()
