"""The GPU parity suites rerun on the bounds-checking build of the library (liblcl_debug.so,
compiled with LCL_DEBUG_BOUNDS): every index a kernel computes into a plane, layer, list, depth map
or table is checked before its access, an out-of-range index is skipped and recorded, and after
each test lcl_last_device_status must report LCL_OK (tests/conftest.py).  The suites run in a child
process so that the loaded library is the debug one; results must still match the oracle."""
import os
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SUITES = ["test_gpu_parity.py", "test_gpu_numeric.py", "test_gpu_batch.py", "test_gpu_pool.py", "test_gpu_serve.py"]


def test_parity_suites_pass_with_bounds_checks_and_clean_device_status():
    from paper_2501_14807_gb300 import build, lcl
    if not os.path.exists(lcl.DEBUG_LIB_PATH):
        build.build(debug=True)
    env = dict(os.environ, LCL_DEBUG_BOUNDS="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider"] + \
          [os.path.join(HERE, s) for s in SUITES]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 150 and "failed" not in r.stdout.splitlines()[-1], tail
