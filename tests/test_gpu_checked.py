"""The checked build (libsgn_checked.so, -DSGN_CHECKED) runs the parity suites:
its stage kernels fill every shared-memory tile with NaN before staging it and
check every global index of the tile loads, so a halo entry that is read but
never written, or an index that leaves its plane (flagged, and reported as
SGN_E_INVAL), fails these tests.  This stands in for a memory checker.  The
suites run in a child process with SGN_LIBRARY=checked, the switch that makes
the binding load the checked library."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_parity_suites_pass_on_the_checked_build():
    assert os.path.exists(os.path.join(ROOT, "paper_2601_02540_b300", "libsgn_checked.so"))
    env = dict(os.environ, SGN_LIBRARY="checked")
    suites = ["test_gpu_parity.py", "test_gpu_precision.py", "test_gpu_df64.py", "test_gpu_monitor.py",
              "test_gpu_adaptive.py", "test_gpu_mms.py", "test_gpu_sponge.py", "test_gpu_batch.py",
              "test_gpu_adjoint.py"]
    probe = ("import paper_2601_02540_b300.sgn as s; s.lib(); "
             "assert s.LIB_PATH.endswith('libsgn_checked.so'), s.LIB_PATH")
    subprocess.run([sys.executable, "-c", probe], cwd=ROOT, env=env, check=True)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        *[os.path.join(HERE, f) for f in suites]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
