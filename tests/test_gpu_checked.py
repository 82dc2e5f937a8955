"""The range-checked build (-DDR_CHECKED=1): every kernel family checks each
global address against the bounds of its piece (and the alignment of 16-byte
accesses) and records DR_E_BOUNDS instead of touching memory outside it.  This
test builds that variant of the library into its own directory and runs small
cases of every kernel family through it (tests/checked_cases.py, in a fresh
process so the two builds never share one process); each case must leave the
status word clean and match the oracle."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_checked_build_runs_every_kernel_clean():
    pytest.importorskip("torch")
    from paper_2406_00158_gb300 import build
    pkg = os.path.join(ROOT, "paper_2406_00158_gb300")
    lib = build.build(extra_flags=["-DDR_CHECKED=1"], out=os.path.join(pkg, "libdr_gb300_checked.so"),
                      build_dir=os.path.join(pkg, "_build_checked"))
    env = dict(os.environ, DR_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "checked cases ok" in r.stdout
