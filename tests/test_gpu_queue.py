"""The work queue of the persistent FFA launch, as the device built it: the per-position
item records (`ffa_periodogram_queue`) read back after a search.  CTAs claim queue
positions in order and an item waits only on a completion counter, so every wait ends if
all the items that release a counter come earlier in the queue than its waiters and
their number is the count the waiters need.  Checked on the survey search (one batch
ring of six slots), on plain_small, and with small tiles that make many more batches and
deeper top-pass chains."""
import collections

import numpy as np
import pytest

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


def _check_queue(rec):
    tr, pas, batch, wait, need, rel = rec[:, 0], rec[:, 2], rec[:, 3], rec[:, 4], rec[:, 5], rec[:, 6]
    n = len(rec)
    assert n > 0
    first_wait = {}
    releasers = collections.defaultdict(list)
    for q in range(n):
        if rel[q] >= 0:
            releasers[int(rel[q])].append(q)
        if wait[q] >= 0:
            first_wait.setdefault(int(wait[q]), q)
    needs = collections.defaultdict(set)
    for q in range(n):
        if wait[q] >= 0:
            needs[int(wait[q])].add(int(need[q]))
    for c, qs in needs.items():
        assert len(qs) == 1, c               # every waiter of a counter needs the same count
        k = qs.pop()
        r = releasers[c]
        assert len(r) == k, (c, len(r), k)   # exactly the items that release it
        assert max(r) < first_wait[c], c     # ... all of them queued before its first waiter
    for c, r in releasers.items():
        assert c in needs, c                 # nothing is released that no item waits for
    # stages of a transform: sub-trees, then its top passes in order
    stage = np.where(pas < 0, 0, pas + 1)
    last = {}
    for q in range(n):
        t, s = int(tr[q]), int(stage[q])
        prev = last.get(t, (-1, -1))
        assert s >= prev[0], (q, t, s, prev)
        last[t] = (s, q)
    # a sub-tree that reuses a ring slot waits for the counter released by the last
    # passes of one earlier batch
    for q in range(n):
        if pas[q] == -1 and wait[q] >= 0:
            rb = {int(batch[x]) for x in releasers[int(wait[q])]}
            assert len(rb) == 1 and rb.pop() < batch[q], q
    return int((wait >= 0).sum())


def _run(F, w, tiles=None):
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    S = F.Searcher(w.n, *args, tiles=tiles)
    S(torch.from_numpy(w.x).cuda())
    S.check()
    return S.queue_records()


def test_survey_queue(F):
    rec = _run(F, synth.survey())
    assert len(rec) == 20177  # 8442 sub-trees, 11378 top-pass items, 357 whole trees
    assert _check_queue(rec) > 10000
    assert rec[:, 3].max() >= 6          # more batches than ring slots: slots are reused


def test_plain_small_queue(F):
    _check_queue(_run(F, synth.plain_small()))


def test_small_tiles_queue(F):
    """Sub-trees of 12 rows and one merge level per top pass: deep chains of stages."""
    rec = _run(F, synth.survey(), F.Tiles(12, 1, 16))
    assert _check_queue(rec) > 0
    assert rec[:, 2].max() >= 4
