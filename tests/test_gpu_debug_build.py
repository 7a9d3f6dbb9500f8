"""The parity suites against the debug build of the library.

The debug build (build_lib.build(debug=True), loaded when ZD_DEBUG=1) checks
the kernels' index arithmetic before every guarded access and records
ZD_ERR_INTERNAL instead of touching memory it does not own; every parity
test ends with zd_check() == ZD_OK, so a failed check fails the test that
triggered it.  The extra build takes about a minute, so this runs only when
ZD_TEST_DEBUG_BUILD=1 is set.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_dynamic.py", "tests/test_gpu_batched.py",
          "tests/test_gpu_large_k.py", "tests/test_gpu_backward.py", "tests/test_gpu_failure.py",
          "tests/test_gpu_small_updates.py"]


@pytest.mark.skipif(os.environ.get("ZD_TEST_DEBUG_BUILD") != "1", reason="set ZD_TEST_DEBUG_BUILD=1")
def test_parity_suites_pass_under_the_debug_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04182_gb300 import build_lib
    build_lib.build(debug=True)
    env = dict(os.environ, ZD_DEBUG="1", ZD_TEST_DEBUG_BUILD="0")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + SUITES,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    # the debug library, not the release one, served those tests
    chk = subprocess.run([sys.executable, "-c", "from paper_2111_04182_gb300 import zd; "
                          "assert zd.LIB_PATH.endswith('libzd_debug.so'); zd._lib()"],
                         cwd=ROOT, env=env, capture_output=True, text=True)
    assert chk.returncode == 0, chk.stderr
