"""The parity suite on small cases under the bounds-checked build (needs a
GB300).  In that build every checked kernel access -- encoder stages and
tile rings, workspace arrays, decoder offsets, block heads -- is tested
against its buffer; a failed check records ZC_ERR_BOUNDS (and skips the
access), which every parity test's status assertion catches.  The suite runs
in a child process that loads the checked library (ZC_LIBRARY=debug)."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_under_the_bounds_checked_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05199_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, ZC_LIBRARY="debug")
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_batch.py", "tests/test_gpu_heads.py",
             "tests/test_gpu_pipeline.py", "tests/test_gpu_collectives.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p",
                        "no:cacheprovider"] + files, capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in tail
