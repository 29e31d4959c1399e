"""Long-run time-mean kinetic energy of the chaotic flow (Section 5.1's
statistically steady state, Section 5.2's energy) against the FP64 oracle.

The 64 x 128, l = 1 basin of Experiment I runs from rest (plus the seeded
perturbation) to t = 50.  The oracle's energy history and its mean over
t in [10, 50] come from tests/golden/mean_ke_64x128_l1.txt (written by
tests/golden/make_mean_ke.py from the oracle alone).

The flow is chaotic: FP32 and FP64 trajectories, and FP64 trajectories that
sum in different orders, part at the end of the spin-up burst (t ~ 1.3), and
the energy of one realization varies slowly by tens of percent (the oracle's
10-unit means over [10, 50] span 169-367).  So the 1 % tolerance applies
where a time mean is a property of the trajectory itself: the mean over
the first 12 000 steps (t < 1.2, before the trajectories part); the mean
over [10, 50] is checked against the oracle's sampling band instead.
"""
import numpy as np
import pytest

from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def golden():
    mean, quarters, hist = None, None, {}
    from tests.golden.load import HERE
    import os
    with open(os.path.join(HERE, "mean_ke_64x128_l1.txt")) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if not parts:
                continue
            if parts[0] == "mean_ke":
                mean = float(parts[1])
            elif parts[0] == "quarter_means":
                quarters = [float(v) for v in parts[1:]]
            elif parts[0] == "ke_at":
                hist[int(parts[1])] = float(parts[2])
    return mean, quarters, hist


def run(dtype, last_step, every, keep):
    """KE every `every` steps up to last_step; returns {step: KE} for the
    steps where keep(step)."""
    b = qg.Basin(64, 128, Re=200.0, Ro=0.0016, levels=1, dt=1e-4, dtype=dtype)
    b.set_state(inputs.perturbation(64, 128, seed=1))
    out = {}
    for n in range(0, last_step + 1, every):
        if keep(n):
            out[n] = b.diagnostics()[0]
        if n < last_step:
            b.step(every)
    b.close()
    return out


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-2)])
def test_mean_energy_over_the_first_12000_steps(dtype, tol):
    """Mean of the kinetic energy history (every 200 steps) over t < 1.2:
    within the stated 1 % in FP32 (and to rounding in FP64)."""
    require_gpu()
    _, _, hist = golden()
    steps = [n for n in sorted(hist) if n < 12000]
    got = run(dtype, 11800, 200, lambda n: True)
    ref = np.mean([hist[n] for n in steps])
    val = np.mean([got[n] for n in steps])
    assert abs(val - ref) <= tol * ref, (val, ref)


def test_long_window_mean_energy_within_the_sampling_band():
    """FP32, t in [10, 50] sampled every 20 steps (Section 5.1's window):
    the mean lies within the spread of the oracle's own 10-unit means, the
    sampling band of a 40-unit mean of this chaotic flow."""
    require_gpu()
    mean, quarters, _ = golden()
    got = run("f32", 500000, 20, lambda n: 100000 <= n < 500000)
    val = float(np.mean(list(got.values())))
    assert len(got) == 20000
    assert min(quarters) <= val <= max(quarters), (val, mean, quarters)
