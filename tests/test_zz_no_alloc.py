"""ffa_transform_noalloc: the transform for callers that cannot allocate device memory
(plugins whose host application owns every allocation, pipelines that forbid allocation
once running).  Its scratch is a fixed array inside the library, so the call takes only
the input and output buffers.  Checked through the C ABI against ffa_transform (which is
given a workspace) on two calls in a row: results must be bit-identical, as every FFA
transform result of this library is.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_03701_gb300 as ffa
    ffa.build()
    L = ffa.library()
    L.ffa_transform_noalloc.restype = ctypes.c_int32
    L.ffa_transform_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p]
    return ffa, L


def _noalloc(L, block):
    out = torch.empty_like(block)
    stream = torch.cuda.current_stream().cuda_stream
    st = L.ffa_transform_noalloc(ctypes.c_void_p(block.data_ptr()), block.shape[0],
                                 block.shape[1], ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream))
    return st, out


@pytest.mark.parametrize("m,p", [(1000, 250), (2684, 240), (77, 31)])
def test_matches_workspace_transform_twice(lib, m, p):
    ffa, L = lib
    for call in range(2):   # the shared scratch keeps the previous call's contents
        X = torch.from_numpy(synth.normal_block(m, p, seed=100 * call + m)).cuda()
        st, got = _noalloc(L, X)
        assert st == 0, L.ffa_last_error()
        ref = ffa.ffa_transform(X)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_rejects_blocks_above_the_fixed_scratch(lib):
    ffa, L = lib
    X = torch.zeros((5000, 260), dtype=torch.float32, device="cuda")  # needs ~5.2 MB
    st, _ = _noalloc(L, X)
    assert st == 2  # FFA_ERR_CAPACITY
    assert b"4 MiB" in L.ffa_last_error()


def test_allocates_nothing_after_the_first_call(lib):
    """After the first call on a device (which looks the array up, loading the library's
    module with it under lazy loading), a call changes no device allocation and records
    no profiling events (the launch counter still counts its kernels)."""
    ffa, L = lib
    X = torch.from_numpy(synth.normal_block(1000, 250, seed=7)).cuda()
    st, out = _noalloc(L, X)
    assert st == 0, L.ffa_last_error()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    ffa.profile_enable(True)
    ffa.profile_reset()
    free0 = torch.cuda.mem_get_info()[0]
    launches0 = ffa.launch_count()
    st = L.ffa_transform_noalloc(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1],
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert st == 0, L.ffa_last_error()
    assert free1 == free0
    assert ffa.launch_count() > launches0
    for kind in ("ffa_bottom", "ffa_top"):
        assert ffa.profile_query(kind)["launches"] == 0, kind
    ffa.profile_enable(False)
    ffa.profile_reset()
    assert torch.equal(out, ffa.ffa_transform(X))
