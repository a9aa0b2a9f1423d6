"""The bounds-checking build of the library (-DHS_CHECK_BOUNDS): every
shared-memory index of the staged kernel is tested against its own level's
span in the stage and every global index of its exact pass against its table
or plane; the harmonic-fraction kernels test every shared-memory read against
its term's box (staged) or every plane read against the plane (gather), and
each threshold read against the table.  An index outside would be skipped
and reported as HS_ERR_BOUNDS, which the binding raises.  The GPU parity
tests of the small shapes (every level sum, candidate sets, band edges, other
shapes, 16-bit storage, signed inputs, tile orders, the harmonic-fraction
map) run against that build in a child process and must pass unchanged: no
index leaves its buffer and the records still equal the FP64 oracle's.
(compute-sanitizer is not available to these tests.)"""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_tests_pass_on_the_bounds_checking_build():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1805_12258_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, HS_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           os.path.join("tests", "test_gpu_parity.py"), "-k", "not ska_plane"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout[-3000:] + "\n" + r.stderr[-2000:]).strip()
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
