"""Helpers of the GPU parity tests: run the CUDA path through the C ABI
binding and the oracle on the same seeded inputs."""
import numpy as np
import pytest

from paper_1308_3290_gb300 import build, qg


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    build.build()
    qg.load()
    return torch


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_np(t):
    return t.detach().double().cpu().numpy()


def seam_lines(n, period):
    """Indices (0-based, exchange layout) of the interior lines next to the
    walls and on both sides of every multiple of `period` nodes: where a
    mistake at a wall or at a tile edge of the fine-grid kernels or of the
    restriction's partial-sum planes would sit."""
    j = np.arange(1, n + 1)          # node index of exchange index j - 1
    sel = (j == 1) | (j == n) | (j % period <= 1) | (j % period == period - 1)
    return np.nonzero(sel)[0]


def field_errors(got, ref, xper=64, yper=8):
    """Relative L2 error over the whole field and over the wall and seam
    rows and columns alone, and the largest element error relative to the
    field's largest value."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rows = seam_lines(ref.shape[0], yper)
    cols = seam_lines(ref.shape[1], xper)
    return {
        "l2": rel_l2(got, ref),
        "l2_seam_rows": rel_l2(got[rows], ref[rows]),
        "l2_seam_cols": rel_l2(got[:, cols], ref[:, cols]),
        "max": float(np.abs(got - ref).max() / np.abs(ref).max()),
    }


def assert_fields_close(got, ref, l2_tol, max_tol=None, **kw):
    """Element-wise parity: the relative L2 bound holds on the whole field
    and on the wall and seam lines separately (a local error is not diluted
    by the rest of the field), and no element is off by more than max_tol
    (default l2_tol) of the field's largest value."""
    e = field_errors(got, ref, **kw)
    mt = l2_tol if max_tol is None else max_tol
    assert e["l2"] <= l2_tol, e
    assert e["l2_seam_rows"] <= l2_tol, e
    assert e["l2_seam_cols"] <= l2_tol, e
    assert e["max"] <= mt, e
    return e
