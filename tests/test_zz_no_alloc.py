"""qg_poisson_solve_noalloc, the Poisson solve for callers that must not
allocate device memory, against the FP64 oracle and the handle-based solve.

Its workspace is one fixed library-owned device array shared by all calls,
so every case makes two calls in a row with different right-hand sides (a
stale workspace would show up in the second) and compares each with the
oracle's solve (Section 4.3: Eqs. ifft-1, ialpha, ffft-1) and with
qg_poisson_solve.  The shapes cover both FFT engines the call can pick:
radix 4 on small grids, radix 16 at 2^21 nodes and on a 4096-long side that
radix 4 cannot take.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}

CASES = [
    ("f64", 64, 128, -1.0, 1.0),
    ("f32", 64, 128, -1.0, 1.0),
    ("f64", 256, 128, -0.5, 0.5),
    ("f32", 256, 128, -0.5, 0.5),
    ("f32", 4096, 128, -1.0, 1.0),     # radix 4 cannot take the 4096-long side
    ("f32", 1024, 2048, -1.0, 1.0),    # 2^21 nodes: radix 16
    ("f64", 1024, 1024, -0.5, 0.5),    # close to the workspace limit in FP64
]


def _call(torch, nx, ny, dx, dy, dtype, rhs):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    code = qg.QG_F64 if dtype == "f64" else qg.QG_F32
    r = torch.as_tensor(rhs, dtype=tdt, device="cuda").contiguous()
    out = torch.full((ny - 1, nx - 1), float("nan"), dtype=tdt, device="cuda")
    qg.qg_poisson_solve_noalloc(nx, ny, dx, dy, code, r, out,
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return to_np(out)


@pytest.mark.parametrize("dtype,nx,ny,y0,y1", CASES)
def test_noalloc_matches_oracle_and_handle_solve_twice(dtype, nx, ny, y0, y1):
    torch = require_gpu()
    dx, dy = 1.0 / nx, (y1 - y0) / ny
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype, y0=y0, y1=y1)
    for seed in (1, 2):
        rhs = inputs.smooth_field(nx, ny, seed=seed, noise=0.3 * seed)
        want = O.poisson_solve(rhs, nx, ny, dx, dy)
        got = _call(torch, nx, ny, dx, dy, dtype, rhs)
        assert np.isfinite(got).all()
        assert rel_l2(got, want) <= TOL[dtype], (seed, rel_l2(got, want))
        ref = to_np(b.poisson_solve(rhs))
        assert rel_l2(got, ref) <= TOL[dtype], (seed, rel_l2(got, ref))
    b.close()


def test_noalloc_rejects_requests_beyond_its_workspace():
    torch = require_gpu()
    r = torch.zeros((4095, 2047), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(r)
    with pytest.raises(qg.QGError) as e:
        qg.qg_poisson_solve_noalloc(2048, 4096, 1 / 2048, 2 / 4096, qg.QG_F32, r, out,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 2


def test_noalloc_reports_a_timed_out_wait(monkeypatch):
    """With the stall switch the solve's grid barrier waits for an arrival
    that never comes; the bounded wait runs out (about a second), the call
    returns QG_ERR_TIMEOUT and leaves psi alone, and the next call without
    the switch solves correctly again."""
    torch = require_gpu()
    nx, ny = 64, 128
    dx, dy = 1.0 / nx, 2.0 / ny
    rhs = inputs.smooth_field(nx, ny, seed=3, noise=0.2)
    monkeypatch.setenv("QG_NOALLOC_STALL", "1")
    r = torch.as_tensor(rhs, dtype=torch.float64, device="cuda").contiguous()
    out = torch.full((ny - 1, nx - 1), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(qg.QGError) as e:
        qg.qg_poisson_solve_noalloc(nx, ny, dx, dy, qg.QG_F64, r, out,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 7
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    monkeypatch.delenv("QG_NOALLOC_STALL")
    got = _call(torch, nx, ny, dx, dy, "f64", rhs)
    assert rel_l2(got, O.poisson_solve(rhs, nx, ny, dx, dy)) <= TOL["f64"]
