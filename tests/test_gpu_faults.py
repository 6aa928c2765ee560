"""The device-side failure path, made without a GPU fault: one transform's second stage
is told to wait for one item more than exist (FFA_FAULT=stage), so that wait runs out
after a 1 ms limit.  The launch then ends early by itself, ffa_check reports
FFA_ERR_TIMEOUT, and the next normal call on the same workspace is bit-identical to one
made before the fault."""
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


def test_stage_wait_runs_out_and_the_workspace_recovers(F, monkeypatch):
    w = synth.plain_small()
    S = F.Searcher(w.n, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths)
    assert S.info.tiles.top_levels > 0  # the plan has top passes, hence stage waits
    x = torch.from_numpy(w.x).cuda()
    ref = [t.clone() for t in S(x)]
    S.check()
    try:
        F.set_wait_limit_ms(1.0)
        monkeypatch.setenv("FFA_FAULT", "stage")
        S(x)
        with pytest.raises(F.FFAError) as err:
            S.check()
        assert err.value.status == 4  # FFA_ERR_TIMEOUT
    finally:
        monkeypatch.delenv("FFA_FAULT", raising=False)
        F.set_wait_limit_ms(1000.0)
    got = S(x)
    S.check()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
