"""The bounds-checked build (-DNIF_BOUNDS=1, include/nif.h: nif_bounds_check)
runs the oracle parity suites with no failed index check.

The build compiles the same sources with index checks at the gathers and
scatters (the grid cell of every encoder access, label triangles, the
rest-space point order, the per-ray segment rows); a failed check is counted
in a device word and the access redirected or skipped, nothing traps. The
suites run in a child process that loads libnif_bounds.so
(NIF_BOUNDS_BUILD=1); tests/conftest.py then checks after every GPU test that
no index check failed. A planted mistake belongs in the oracle, on the CPU,
so no test here makes a check fail on purpose.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_parity_full.py", "tests/test_gpu_query_fused.py",
          "tests/test_gpu_train_steps.py", "tests/test_gpu_mixed_train.py", "tests/test_gpu_query_async.py"]


def test_parity_suites_pass_under_the_bounds_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_24666_gb300 import build as Bld
    lib = Bld.build(bounds=True)
    assert lib.endswith("libnif_bounds.so") and os.path.exists(lib)
    env = dict(os.environ, NIF_BOUNDS_BUILD="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *SUITES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail.split("\n")[-2], tail
