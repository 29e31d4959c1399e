"""qg_poisson_solve_noalloc, the Poisson solve for callers that must not
allocate device memory, gives the same answer as qg_poisson_solve.

Its workspace is one fixed library-owned device array shared by all calls,
so the test makes two calls in a row with different right-hand sides (a
stale workspace would show up in the second) and compares each with the
handle-based solve.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,y0,y1", [(64, 128, -1.0, 1.0), (256, 128, -0.5, 0.5)])
def test_noalloc_matches_handle_solve_twice(dtype, nx, ny, y0, y1):
    torch = require_gpu()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dx, dy = 1.0 / nx, (y1 - y0) / ny
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype, y0=y0, y1=y1)
    code = qg.QG_F64 if dtype == "f64" else qg.QG_F32
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (1, 2):
        rhs = inputs.smooth_field(nx, ny, seed=seed, noise=0.3 * seed)
        ref = to_np(b.poisson_solve(rhs))
        r = torch.as_tensor(rhs, dtype=tdt, device="cuda").contiguous()
        out = torch.full((ny - 1, nx - 1), float("nan"), dtype=tdt, device="cuda")
        qg.qg_poisson_solve_noalloc(nx, ny, dx, dy, code, r, out, stream)
        torch.cuda.synchronize()
        got = to_np(out)
        assert np.isfinite(got).all()
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
