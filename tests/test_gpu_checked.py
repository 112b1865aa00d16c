"""The bounds-checked build (nvcc -DAMPED_CHECKS=1), the stand-in for a memory
sanitizer: every gather coordinate, output row id, stream position and
row-table window that the MTTKRP and sampled-model kernels use is checked on
the device; the first failure is recorded in the handle's error word, the
access is clamped in bounds (nothing faults) and the entry point returns
AMPED_ERR_INDEX naming the check.

The checked library is compiled into a temporary directory and loaded in child
processes (AMPED_LIB).  On valid inputs no check fires and every kernel path
matches the FP64 oracle; with one coordinate of a mode copy corrupted on the
host after validation (AMPED_FAULT=coord:K, an injector compiled into checked
builds only) the call reports the failed check instead of reading out of bounds,
and the modes whose copies are intact still compute.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = os.path.join(ROOT, "tests", "checked_child.py")


@pytest.fixture(scope="module")
def checked_lib(tmp_path_factory):
    sys.path.insert(0, ROOT)
    from paper_2507_15121_gb300 import build as lib_build
    d = tmp_path_factory.mktemp("checked")
    return lib_build.build(flags=["-DAMPED_CHECKS=1"], lib_path=str(d / "libamped_checked.so"),
                           build_dir=str(d / "_build"))


def _child(lib, case, **env):
    e = {k: v for k, v in os.environ.items() if k != "AMPED_FAULT"}
    e.update(AMPED_LIB=lib, **env)
    r = subprocess.run([sys.executable, CHILD, case], env=e, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return r.stdout


def test_checked_build_valid_inputs_match_oracle(checked_lib):
    assert "valid inputs: ok" in _child(checked_lib, "valid")


def test_checked_build_reports_corrupted_coordinate(checked_lib):
    assert "corrupted copy: reported" in _child(checked_lib, "corrupt", AMPED_FAULT="coord:7")
