"""Checkpoint / resume through the state exchange calls, and the non-finite
state watchdog of qg_diagnostics."""
import numpy as np
import pytest

from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("levels,dtype,tol", [(0, "f32", 0.0), (0, "f64", 0.0),
                                              (2, "f32", 1e-6), (2, "f64", 1e-13)])
def test_resume_from_a_saved_state(levels, dtype, tol):
    """40 steps in one go against 20 steps, the state saved to host memory, a
    new handle started from it and 20 more steps.  At l = 0 the step is a
    function of the state alone, so the resumed run is bitwise the same;
    at l >= 1 the new handle restricts the state afresh where the running
    one carries the restriction's partial sums from its last fine stage
    (a different summation order), so the runs agree to rounding."""
    torch = require_gpu()
    nx, ny = 256, 512
    w0 = inputs.perturbation(nx, ny, seed=21) * 30.0
    kw = dict(Re=200.0, Ro=0.0016, levels=levels, dt=2e-5, dtype=dtype)
    a = qg.Basin(nx, ny, **kw)
    a.set_state(w0)
    a.step(40)
    ref = to_np(a.state())
    a.close()
    b = qg.Basin(nx, ny, **kw)
    b.set_state(w0)
    b.step(20)
    saved = b.state().cpu().numpy()          # host copy: the checkpoint
    b.close()
    c = qg.Basin(nx, ny, **kw)
    c.set_state(saved)
    c.step(20)
    got = to_np(c.state())
    c.close()
    if tol == 0.0:
        assert np.array_equal(got, ref)
    else:
        assert rel_l2(got, ref) <= tol
    del torch


def test_nonfinite_state_is_reported():
    require_gpu()
    nx, ny = 64, 128
    w = inputs.perturbation(nx, ny, seed=3)
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-4, dtype="f32")
    bad = w.copy()
    bad[10, 20] = np.nan
    b.set_state(bad)
    with pytest.raises(qg.QGError) as e:
        b.diagnostics()
    assert e.value.status == qg.QG_ERR_NONFINITE
    assert qg.qg_last_error(b.h) == qg.QG_ERR_NONFINITE     # read and cleared
    b.set_state(w)
    ke, z, u = b.diagnostics()
    assert np.isfinite(ke) and np.isfinite(z) and np.isfinite(u)
    bad[10, 20] = np.inf
    b.set_state(bad)
    b.step(2)                                   # spreads through the step
    with pytest.raises(qg.QGError) as e:
        b.diagnostics()
    assert e.value.status == qg.QG_ERR_NONFINITE
    b.close()
