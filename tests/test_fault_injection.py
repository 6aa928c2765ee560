"""Host-side fault injection (environment variable FFA_FAULT), checked without a GPU:
each injected failure returns its status with a message naming it, before any CUDA
call, and nothing is left behind (the next call without the variable succeeds)."""
import ctypes

import numpy as np
import pytest

import paper_2004_03701_gb300 as ffa

W = np.array([1, 2, 4, 8], np.int32)
ARGS = (1 << 16, 1e-3, 0.5, 4.0, 40, 44)


@pytest.fixture(scope="module")
def lib():
    ffa.build()
    return ffa.library()


def _plan(lib):
    info = ffa._PlanInfo()
    st = lib.ffa_periodogram_plan(*ARGS, ctypes.c_void_p(W.ctypes.data), len(W),
                                  ctypes.byref(info))
    return st, info


def test_plan_fault(lib, monkeypatch):
    monkeypatch.setenv("FFA_FAULT", "plan")
    st, _ = _plan(lib)
    assert st == 5 and b"injected fault: plan" in lib.ffa_last_error()
    series = (ffa._Series * 1)(ffa._Series(0, 1 << 16, 1e-3, 0.5, 4.0, 40, 44))
    binfo = ffa._BatchInfo()
    st = lib.ffa_batch_plan(ctypes.cast(series, ctypes.c_void_p), 1,
                            ctypes.c_void_p(W.ctypes.data), len(W), 1 << 30, None,
                            ctypes.byref(binfo))
    assert st == 5 and b"injected fault: plan" in lib.ffa_last_error()
    monkeypatch.delenv("FFA_FAULT")
    st, info = _plan(lib)
    assert st == 0 and info.ntrials > 0


@pytest.mark.parametrize("what", ["alloc", "launch"])
def test_execution_faults_before_any_cuda_call(lib, monkeypatch, what):
    st, info = _plan(lib)
    assert st == 0
    monkeypatch.setenv("FFA_FAULT", what)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the call fails first
    st = lib.ffa_periodogram(fake, 0, *ARGS, ctypes.c_void_p(W.ctypes.data), len(W), fake,
                             fake, fake, info.ntrials, fake, info.workspace_bytes, None)
    assert st == 3, lib.ffa_last_error()
    assert ("injected fault: " + what).encode() in lib.ffa_last_error()


def test_wait_limit_arguments(lib):
    assert lib.ffa_set_wait_limit_ms(0.0) == 1
    assert lib.ffa_set_wait_limit_ms(-1.0) == 1
    assert lib.ffa_set_wait_limit_ms(1e9) == 1
    assert lib.ffa_set_wait_limit_ms(1000.0) == 0
