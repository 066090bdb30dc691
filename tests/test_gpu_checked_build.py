"""The bounds-checked debug build (liblbib_checked.so, compiled with
-DLBIB_CHECKED) under the parity tests of the lattice, coupled, moving-least-
squares, batched and launch-shape paths.  In that build every population, node,
tile and marker index the kernels form is checked against its array; an index
outside sets a status bit (the access is redirected to the array's first
element, nothing traps) that the next sync reports as LBIB_ERR_STATE, so any
such index fails the tests it occurs in.  The tests run in a child process with
LBIB_CHECKED=1, which makes lbib.load() build and load the checked library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_lattice.py", "tests/test_gpu_coupled.py", "tests/test_gpu_mls.py",
          "tests/test_gpu_batch.py", "tests/test_gpu_tuning.py"]


def test_parity_suites_pass_on_the_bounds_checked_build():
    env = dict(os.environ, LBIB_CHECKED="1")
    probe = subprocess.run([sys.executable, "-c", "from paper_2210_06043_gb300 import lbib; lbib.load(); "
                            "print(lbib.library_path())"], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=1200)
    assert probe.returncode == 0, probe.stderr[-3000:]
    assert probe.stdout.strip().endswith("liblbib_checked.so")
    r = subprocess.run([sys.executable, "-m", "pytest", *SUITES, "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
