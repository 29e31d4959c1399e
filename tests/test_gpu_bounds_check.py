"""The bounds-checked build (QG_BOUNDS_CHECK): every index the fine-stage,
solve, matrix-form, transfer, multigrid, diagnostics and adjoint kernels
use is compared with its buffer's extent before the access; a failure is
recorded instead of trapping.  This
stands in for a memory checker: the library's main paths (every solve
engine, every tile height, the transfers, two layers, multigrid, the
adjoint, the batched ensemble, the allocation-free solve) run under that
build, in a process of their own, and no check may fail."""
import os
import subprocess
import sys

import pytest

from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_index_leaves_its_buffer_in_the_checked_build():
    require_gpu()
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_workload.py")],
                       capture_output=True, text=True, timeout=1500)
    print(r.stdout[-3000:], r.stderr[-3000:])
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "FIRST_FAILED_SITE 0" in r.stdout
