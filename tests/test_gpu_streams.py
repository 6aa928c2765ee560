"""The one-shot calls of the binding on a stream other than the current one: their
workspace and outputs are allocated on the stream the kernels run on, so allocations
made meanwhile on the current stream never receive that memory while the kernels may
still use it.  Results are compared bit for bit with the same calls on the current
stream."""
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


def _busy_current_stream(n=8):
    """Allocations and writes on the current stream while the side stream works."""
    junk = []
    for k in range(n):
        t = torch.empty(1 << 22, dtype=torch.float32, device="cuda")
        t.fill_(float(k))
        junk.append(t)
    return junk


def test_one_shot_calls_on_a_side_stream(F):
    block = torch.from_numpy(synth.normal_block(2684, 250, seed=3)).cuda()
    x = torch.from_numpy(synth.red_noise(1 << 18, 1e-3, seed=4)).cuda()
    ref_t = F.ffa_transform(block)
    ref_d = F.downsample(x, 3.7)
    ref_n = F.normalise(x)[0]
    ref_m = F.running_median(x, 101)
    ref_s = F.boxcar_snr(ref_t[:64], (1, 2, 4, 8), 50.0)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    got_t = F.ffa_transform(block, stream=side)
    got_d = F.downsample(x, 3.7, stream=side)
    got_n, mean, std = F.normalise(x, stream=side)
    got_m = F.running_median(x, 101, stream=side)
    got_s = F.boxcar_snr(ref_t[:64], (1, 2, 4, 8), 50.0, stream=side)
    # freed workspaces of the calls above must not be handed out here while side runs
    junk = _busy_current_stream()
    side.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(got_t, ref_t)
    assert torch.equal(got_d, ref_d)
    assert torch.equal(got_n, ref_n) and np.isfinite(mean) and std > 0
    assert torch.equal(got_m, ref_m)
    assert torch.equal(got_s, ref_s)
    for k, t in enumerate(junk):
        assert bool((t == float(k)).all())
