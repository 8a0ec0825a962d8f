"""Index safety: the GPU test files that drive every kernel (every summing
arm, both gridding kernels, every storage type, random shapes and lists) run
again against the bounds-checking build of the library, in which every index
the coordinate step produces is checked against the extent of what it
addresses before any access, and a violation makes degrid_get_status return
DG_ERR_BOUNDS (which fails those tests).  Stands in for a memory checker
(GPU only)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernels_pass_their_tests_under_index_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2102_12739_gb300 import build
    build.build_variant("bounds")
    env = dict(os.environ, DEGRID_LIBRARY_VARIANT="bounds")
    files = ["tests/test_gpu_fuzz.py", "tests/test_gpu_gather.py", "tests/test_gpu_parity.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        *files, "-k", "not central_differences and not full_size and not batched512"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-25:])
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail
