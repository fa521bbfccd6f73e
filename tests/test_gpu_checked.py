"""The index-checked library (libsdgr_checked.so, built with -DSDGR_CHECKED)
on the GPU.  In child processes with SDGR_CHECKED=1: tiny scenes (1-4
Gaussians, 8x8 and 9x7 images, every raster schedule) and the forward,
backward, schedule and batching parity suites.  Every index the binning and
raster stages produce must stay inside its buffer -- a violation sets
SDGR_ERR_BOUNDS in the status word, skips the access and makes the run
fail -- and the results must match the oracle as with the default build."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(args, timeout=900):
    env = dict(os.environ, SDGR_CHECKED="1")
    p = subprocess.run([sys.executable] + args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-3000:]
    return p.stdout


def test_checked_library_is_built():
    from paper_2506_21633_b300 import build
    assert os.path.exists(build.LIB_CHECKED), "build() makes libsdgr_checked.so"


def test_tiny_cases_checked():
    out = _child([os.path.join("tests", "checked_cases.py")])
    assert "checked tiny cases ok: 12" in out


def test_parity_suites_checked():
    _child(["-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
            "tests/test_gpu_forward.py", "tests/test_gpu_backward.py", "tests/test_gpu_schedule.py",
            "tests/test_gpu_batch.py"])
