"""The bounds-checked build (libcmx_check.so, CMX_CHECK = 1) on the ragged, holed and
two-sublattice grids of the parity tests and on the dense boxes of the tensor-copy path (needs a
B300).

Every stage kernel of that build checks its shared- and global-memory indices; a failed check
stops the run with CMX_ECHECK instead of touching memory.  The parity tests below run in a child
process that loads the checked library: they must pass, i.e. no check fires and the results
still match the oracle.
"""
import os
import subprocess
import sys

import pytest

from paper_2603_03706_b300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_runs_clean_on_the_checked_build():
    lib = build.build(checked=True)
    selection = ("rhs or replay_ragged or replay_afm or single_block or deterministic or "
                 "unit_norm or nan_state")
    script = (
        "import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from paper_2603_03706_b300 import cmx\n"
        "assert cmx.load().cmx_checked_build() == 1\n"
        "import pytest\n"
        "sys.exit(pytest.main(['-q', '-p', 'no:cacheprovider', '-x', %r, %r, '-k', %r]))\n"
        % (ROOT, os.path.join(ROOT, "tests"), os.path.join(ROOT, "tests", "test_gpu_parity.py"),
           os.path.join(ROOT, "tests", "test_gpu_dense.py"), selection))
    env = dict(os.environ, CMX_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", script], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
