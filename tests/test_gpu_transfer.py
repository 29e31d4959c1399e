"""GPU parity of the mapping operators (Section 3.1, Eqs. res and pro) with
the oracle's level-by-level composition."""
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-14), ("f32", 2e-7)])
@pytest.mark.parametrize("levels", [1, 2, 3])
def test_restrict_and_prolong(dtype, tol, levels):
    require_gpu()
    nx, ny = 128, 256
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype)
    f = inputs.random_field(nx, ny, seed=levels)
    got = to_np(b.restrict(f, levels))
    ref = O.interior(O.restrict_levels(O.embed(f), levels))
    assert rel_l2(got, ref) <= tol
    mx, my = nx >> levels, ny >> levels
    c = inputs.random_field(mx, my, seed=10 + levels)
    got = to_np(b.prolong(c, levels))
    ref = O.interior(O.prolong_levels(O.embed(c), levels))
    assert rel_l2(got, ref) <= tol
    b.close()
