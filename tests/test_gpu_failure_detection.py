"""Failure detection on the GPU without a GPU fault: a grid barrier of the
elliptic solve is made to wait for an arrival that never comes, its bounded
wait runs out, and the host sees QG_ERR_TIMEOUT; the handle and the CUDA
context stay usable and the next steps match the oracle again."""
import time

import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu


def test_stalled_barrier_is_reported_and_recovered():
    torch = require_gpu()
    nx, ny = 64, 128
    w0 = inputs.perturbation(nx, ny, seed=11) * 50.0
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-4, dtype="f64")
    b.set_state(w0)
    b.step(2)
    b.synchronize()

    qg.qg_inject_fault(b.h, qg.QG_FAULT_BARRIER_STALL)
    t0 = time.perf_counter()
    b.step(1)
    with pytest.raises(qg.QGError) as e:
        b.synchronize()
    assert e.value.status == qg.QG_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0      # every wait is bounded

    # the stand-alone solve reports it too
    rhs = inputs.random_field(nx, ny, seed=12)
    psi = torch.empty((ny - 1, nx - 1), dtype=torch.float64, device="cuda")
    r = torch.as_tensor(rhs, device="cuda")
    qg.qg_poisson_solve(b.h, r, psi, 0)
    with pytest.raises(qg.QGError) as e:
        b.synchronize()
    assert e.value.status == qg.QG_ERR_TIMEOUT

    # back to normal: the same handle, the same context
    qg.qg_inject_fault(b.h, qg.QG_FAULT_NONE)
    b.set_state(w0)
    b.step(10)
    got = to_np(b.state())
    b.synchronize()
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-4)
    assert rel_l2(got, O.run(w0, ob, 10)) <= 1e-12
    qg.qg_poisson_solve(b.h, r, psi, 0)
    b.synchronize()
    assert rel_l2(to_np(psi), O.poisson_solve(rhs, nx, ny, 1.0 / nx, 2.0 / ny)) <= 1e-12
    b.close()
    assert np.isfinite(torch.ones(4, device="cuda").sum().item())


def test_allocation_failure_is_reported_and_released(monkeypatch):
    """An allocation past the injected limit fails like a failed cudaMalloc:
    qg_create returns QG_ERR_OOM, frees what it had allocated, and a handle
    can be created once the limit is lifted."""
    torch = require_gpu()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("QG_ALLOC_LIMIT_BYTES", str(16 << 20))   # the basin needs ~50 MB
    for _ in range(3):
        with pytest.raises(qg.QGError) as e:
            qg.Basin(1024, 2048, Re=200.0, Ro=0.0016, levels=1, dt=1e-5, dtype="f32")
        assert e.value.status == qg.QG_ERR_OOM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (32 << 20)   # nothing held back
    monkeypatch.delenv("QG_ALLOC_LIMIT_BYTES")
    b = qg.Basin(1024, 2048, Re=200.0, Ro=0.0016, levels=1, dt=1e-5, dtype="f32")
    b.step(1)
    b.synchronize()
    b.close()
