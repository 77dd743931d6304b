"""The checked build: libicm_checked.so, compiled with -DICM_INDEX_CHECKS=1, checks the
indices of the blob stencils (gathers, spreads, the blob work inside the x passes) and
of the tiles of the TMA z pass on the device; a failed check raises ICM_EINDEX at the
next icm_sync and skips the access instead of faulting.  The per-step parity cases of
tests/test_gpu_step.py (odd, radix-3, non-cubic and ragged grids, blobs on the periodic
seams, dense bins) run against it in a child process: no check fires and every result
matches the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_step_parity_cases_pass_under_the_index_checks():
    from paper_1212_6427_gb300 import build
    build.build_library()
    lib = build.build_library(checked=True)
    assert lib.endswith("libicm_checked.so") and os.path.exists(lib)
    env = dict(os.environ, ICM_CHECKED="1")
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join("tests", "test_gpu_step.py"), "-k", "test_step_parity"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert res.returncode == 0, res.stdout[-4000:] + res.stderr[-2000:]
    assert " passed" in res.stdout


def test_checked_library_is_the_one_loaded():
    """ICM_CHECKED=1 selects libicm_checked.so in the binding (and nothing else)."""
    code = "import paper_1212_6427_gb300.binding as b; print(os.path.basename(b.LIB_PATH))"
    out = subprocess.run([sys.executable, "-c", "import os; " + code], cwd=ROOT,
                         env=dict(os.environ, ICM_CHECKED="1"), capture_output=True, text=True, timeout=600)
    assert out.stdout.strip() == "libicm_checked.so"
