"""The bounds-checked build of the library (libpgs_checked.so, compiled with
PGS_CHECKED): every list, range, record and pixel index of the blend, sort,
emission and range kernels is checked against the scene's allocations, and a
failing check raises PGS_ERR_BOUNDS and skips the access instead of touching
memory out of range.  This runs the GPU parity and failure-path tests in a
child process on that build; any check that fails surfaces as PGS_ERR_BOUNDS
from pgs_read_status and fails them."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _env():
    return dict(os.environ, PGS_LIB="checked")


def test_parity_and_failure_paths_pass_on_the_bounds_checked_build():
    from paper_2503_23044_b300 import build
    if not os.path.exists(build.LIB_CHECKED):
        build.build(checked=True)
    probe = subprocess.run([sys.executable, "-c", "from paper_2503_23044_b300 import binding as B; "
                            "print(B.lib().pgs_checked_build())"], env=_env(), cwd=ROOT, capture_output=True,
                           text=True, timeout=300)
    assert probe.stdout.strip().endswith("1"), probe.stdout + probe.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_parity_gpu.py", "tests/test_failure_paths_gpu.py",
                        "tests/test_bf16_decode.py", "-x", "-q", "-m", "gpu"], env=_env(), cwd=ROOT,
                       capture_output=True, text=True, timeout=1800)
    print(r.stdout[-2000:])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
