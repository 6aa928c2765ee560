"""The bounds-checked debug build (libffa_checked.so, compiled with FFA_CHECKED) run over
the small and odd shapes of the parity, median, peaks, tile and batch tests.

Every shared-memory range and global index that the persistent FFA, S/N, prefix,
downsampling, median and peak kernels compute from runtime data is checked in that
build; a violation skips the access and records a status bit.  The selected tests run in
a child pytest process with FFA_LIBRARY=checked: they must pass with the same results as
the normal library (their own comparisons with the oracle) and, after each test, the
recorded violation bits must be zero (tests/conftest.py)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FILES = ["tests/test_gpu_parity.py", "tests/test_gpu_median.py", "tests/test_gpu_peaks.py",
         "tests/test_gpu_tiles.py", "tests/test_gpu_batch.py"]
# the full-size cases take minutes in the checked build and add no new shapes
DESELECT = ("not survey_sampled and not 8388608 and not full_size and not longer_than_4096 "
            "and not full_survey and not cuda_graph")


@pytest.mark.gpu
def test_checked_build_small_and_odd_shapes():
    from paper_2004_03701_gb300 import _build
    _build.build(checked=True)
    env = dict(os.environ, FFA_LIBRARY="checked")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "-k", DESELECT, *FILES]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout[-6000:] + "\n" + r.stderr[-3000:])
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail


@pytest.mark.gpu
def test_normal_build_reports_unchecked():
    import paper_2004_03701_gb300 as ffa
    if os.environ.get("FFA_LIBRARY") == "checked":
        pytest.skip("runs against the normal library")
    checked, bits = ffa.checked_status()
    assert not checked and bits == 0
