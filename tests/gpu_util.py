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
