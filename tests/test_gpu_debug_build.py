"""The MG_DEBUG build: the library compiled with its device-side index checks
(neighbour sites and blocks, blocks of a colour, coarse sites and neighbours,
aggregates, kernel block indices, bulk-copy alignment; include/sapmg.h,
mg_debug_failures).

1. The reporting path: a one-thread kernel checks a value against a bound,
   touching no memory; an out-of-range value must come back as one failed
   check with its kind, value and source, an in-range one as none, and the
   record must clear once read.
2. The parity tests of the Dirac operator, the Schwarz pass and the
   multilevel cycle (test_gpu_dirac_sap.py, test_gpu_mg.py) run again on the
   debug build, with every test required to end with no failed check
   (tests/conftest.py).

Both run in child processes with SAPMG_LIBRARY=debug, because a process
loads one of the two libraries.  Neither makes a kernel touch memory out of
bounds: no check fails in the parity run, and the self-check kernel only
compares two integers."""

import os
import subprocess
import sys

import pytest

from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SELFTEST = r"""
from paper_1202_2462_gb300 import binding as B
assert B.LIB_PATH.endswith("libsapmg_debug.so"), B.LIB_PATH
assert B.mg_debug_failures() == 0
B.mg_debug_check(2, 3)
assert B.mg_debug_failures() == 0
B.mg_debug_check(5, 3)
n = B.mg_debug_failures()
msg = B.lib().mg_last_error().decode()
assert n == 1, (n, msg)
assert "solver.cu" in msg and "block 5 out of range" in msg, msg
B.mg_debug_check(-1, 3)
B.mg_debug_check(7, 3)
n = B.mg_debug_failures()
msg = B.lib().mg_last_error().decode()
assert n == 2, (n, msg)
assert B.mg_debug_failures() == 0
print("selftest ok:", msg)
"""


def _debug_env():
    from paper_1202_2462_gb300 import _build
    _build.build(debug=True)
    torch = torch_cuda()
    torch.cuda.empty_cache()                  # leave the device memory to the child
    return dict(os.environ, SAPMG_LIBRARY="debug")


def test_debug_build_reports_a_failed_check():
    r = subprocess.run([sys.executable, "-c", _SELFTEST], cwd=ROOT, env=_debug_env(), capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "selftest ok" in r.stdout


def test_parity_tests_pass_on_the_debug_build_without_a_failed_check():
    cmd = [sys.executable, "-m", "pytest", "tests/test_gpu_dirac_sap.py", "tests/test_gpu_mg.py", "-m", "gpu",
           "-x", "-q", "-p", "no:cacheprovider"]
    r = subprocess.run(cmd, cwd=ROOT, env=_debug_env(), capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-6000:] + r.stderr[-4000:]
