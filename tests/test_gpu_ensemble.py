"""GPU parity of the ensemble: independent one-layer basins of different
sizes, Reynolds and Rossby numbers, forcing amplitudes, time steps and CGP
levels (Sections 2.1 and 3) stepped together by one graph per step."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu

MEMBERS = [
    dict(nx=32, ny=64, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, amp=1.0),
    dict(nx=32, ny=64, Re=450.0, Ro=0.0036, levels=1, dt=1e-4, amp=0.7),
    dict(nx=64, ny=128, Re=312.5, Ro=0.0025, levels=1, dt=1e-4, amp=1.3),
    dict(nx=64, ny=128, Re=200.0, Ro=0.0016, levels=2, dt=5e-5, amp=1.0),
    dict(nx=128, ny=256, Re=800.0, Ro=0.0016, levels=2, dt=5e-5, amp=0.5),
    dict(nx=64, ny=64, Re=200.0, Ro=0.0016, levels=1, dt=1e-4, amp=1.5),
    dict(nx=256, ny=128, Re=200.0, Ro=0.0016, levels=3, dt=2e-5, amp=1.0),
]


def oracle_basin(m, forcing=None):
    return O.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"],
                   dt=m["dt"], amp=m["amp"], forcing=forcing)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-4)])
def test_ensemble_matches_oracle(dtype, tol):
    require_gpu()
    ens = qg.Ensemble(MEMBERS, dtype=dtype)
    w0 = [inputs.perturbation(m["nx"], m["ny"], seed=20 + i) * 50.0
          for i, m in enumerate(MEMBERS)]
    for i, w in enumerate(w0):
        ens.member(i).set_state(w)
    # one member with a forcing field (its captured step changes)
    f = inputs.perturbed_forcing_field(64, 128, seed=5, Ro=0.0016)
    ens.member(3).set_forcing(f)
    ens.step(20)
    ens.synchronize()
    for i, m in enumerate(MEMBERS):
        ref = O.run(w0[i], oracle_basin(m, forcing=f if i == 3 else None), 20)
        got = to_np(ens.member(i).state())
        assert rel_l2(got, ref) <= tol, (i, rel_l2(got, ref))
    ens.close()


def _groups(members):
    """Launches per TVDRK3 stage of a batched ensemble step: the members
    whose elliptic grids share shape and spacings form a group with one
    solve launch, and one fine-stage launch per CGP level among its
    members.  Returns (solve launches, fine launches)."""
    groups = {}
    for m in members:
        key = (m["nx"] >> m["levels"], m["ny"] >> m["levels"],
               (1.0 / m["nx"]) * 2 ** m["levels"], (2.0 / m["ny"]) * 2 ** m["levels"])
        groups.setdefault(key, set()).add(m["levels"])
    return len(groups), sum(len(v) for v in groups.values())


@pytest.mark.parametrize("engine", [34, 40, 4])
def test_ensemble_equals_standalone_handles(engine, monkeypatch):
    """The batched step (one solve launch per group of equal elliptic grids,
    one fine-stage launch per level) does the same arithmetic as stand-alone
    handles: with the same solve engine the states are bitwise equal.  With
    the warp-group engine (34) and the matrix form (40) the solves are
    batched; the shared-memory engine (4) does not batch, so each member
    solves with its own three launches."""
    require_gpu()
    monkeypatch.setenv("QG_SOLVE_ENGINE", str(engine))
    # members sweep 64-row tiles (the batched launch's); the stand-alone
    # handles are given the same tile
    monkeypatch.setenv("QG_FINE_ROWS", "64")
    ens = qg.Ensemble(MEMBERS, dtype="f32")
    solo = [qg.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"], dt=m["dt"],
                     amp=m["amp"], dtype="f32") for m in MEMBERS]
    for b in solo:
        assert qg.qg_solve_engine(b.h) == engine
    for i, m in enumerate(MEMBERS):
        w = inputs.perturbation(m["nx"], m["ny"], seed=40 + i) * 50.0
        ens.member(i).set_state(w)
        solo[i].set_state(w)
    ens.step(7)
    for b in solo:
        b.step(7)
    ens.synchronize()
    for i, b in enumerate(solo):
        b.synchronize()
        assert np.array_equal(to_np(ens.member(i).state()), to_np(b.state())), i
    for b in solo:
        b.close()
    n_solve, n_fine = _groups(MEMBERS)
    per_stage = n_solve + n_fine if engine != 4 else 3 * len(MEMBERS) + n_fine
    assert ens.kernel_count() == 3 * per_stage
    ens.close()


def test_ensemble_of_96_basins_steps():
    """The ensemble workload's shape (96 basins of four sizes, l in {1, 2}):
    every member advances and stays finite."""
    require_gpu()
    rng = np.random.default_rng(4)
    sizes = [(128, 256), (256, 512), (512, 1024), (1024, 2048)]
    members = []
    for _ in range(96):
        nx, ny = sizes[rng.integers(0, 4)]
        members.append(dict(nx=nx, ny=ny, Re=float(rng.uniform(200, 1000)), Ro=0.0016,
                            levels=int(rng.integers(1, 3)), dt=1e-5,
                            amp=float(rng.uniform(0.5, 1.5))))
    ens = qg.Ensemble(members, dtype="f32")
    for i, m in enumerate(members):
        ens.member(i).set_state(inputs.perturbation(m["nx"], m["ny"], seed=1000 + i))
    # batched: one solve launch per elliptic-grid group, one fine launch per
    # level, per stage
    n_solve, n_fine = _groups(members)
    assert n_solve + n_fine == 13
    assert ens.kernel_count() <= 3 * (n_solve + n_fine) <= 40
    ens.step(5)
    ens.synchronize()
    for i in (0, 17, 95):
        ke, z, u = ens.member(i).diagnostics()
        assert np.isfinite(ke) and ke > 0 and np.isfinite(z)
    ens.close()


def test_ensemble_member_time_mean_matches_oracle():
    """Time-mean psi (Section 5.1's statistic) accumulated on ensemble
    members, as the long-run study of the 16 x 32 elliptic set does: members
    with l = 0, 1, 2 started from rest, the mean over steps n0..n1-1 against
    the oracle's."""
    torch = require_gpu()
    runs = [(16, 32, 0), (32, 64, 1), (64, 128, 2)]
    members = [dict(nx=nx, ny=ny, Re=200.0, Ro=0.0016, levels=lv, dt=1e-4)
               for nx, ny, lv in runs]
    n0, n1 = 10, 40
    ens = qg.Ensemble(members, dtype="f64")
    for i, m in enumerate(members):
        ens.member(i).set_state(np.zeros((m["ny"] - 1, m["nx"] - 1)))
    ens.step(n0)
    ens.synchronize()
    for i in range(len(members)):
        qg.qg_stats_begin(ens.member(i).h)
    ens.step(n1 - n0)
    ens.synchronize()
    for i, m in enumerate(members):
        v = ens.member(i)
        out = torch.empty((m["ny"] - 1, m["nx"] - 1), dtype=torch.float64, device="cuda")
        assert qg.qg_stats_mean_psi(v.h, out) == n1 - n0
        ens.synchronize()
        w0 = np.zeros((m["ny"] - 1, m["nx"] - 1))
        ob = O.Basin(m["nx"], m["ny"], Re=200.0, Ro=0.0016, levels=m["levels"], dt=1e-4)
        ref = O.mean_psi(w0, ob, n0, n1)
        assert rel_l2(to_np(out), ref) <= 1e-12, (i, rel_l2(to_np(out), ref))
    ens.close()


_CACHE_SCRIPT = r"""
import json, os, sys
import numpy as np
from paper_1308_3290_gb300 import inputs, qg
members = json.loads(sys.argv[1])
force = sys.argv[2]
ens = qg.Ensemble(members, dtype="f32")
for i, m in enumerate(members):
    ens.member(i).set_state(inputs.perturbation(m["nx"], m["ny"], seed=70 + i) * 50.0)
ens.step(3)
ens.synchronize()
same = True
if force != "-":
    # stand-alone handles on the engine the cache file names for the group
    os.environ["QG_SOLVE_ENGINE"] = force
    os.environ.pop("QG_TUNE_CACHE")
    for i, m in enumerate(members):
        b = qg.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"], dt=m["dt"],
                     amp=m["amp"], dtype="f32")
        assert qg.qg_solve_engine(b.h) == int(force)
        b.set_state(inputs.perturbation(m["nx"], m["ny"], seed=70 + i) * 50.0)
        b.step(3)
        b.synchronize()
        same = same and np.array_equal(b.state().cpu().numpy(), ens.member(i).state().cpu().numpy())
        b.close()
ens.close()
print(json.dumps({"same": bool(same)}))
"""


def test_group_engine_from_the_tune_cache_file(tmp_path):
    """An ensemble group's engine choice goes to the QG_TUNE_CACHE file and a
    later process takes it from there: the file's group line, rewritten to
    another engine that batches the grid, decides the engine of a fresh
    process's group (bitwise the states of stand-alone handles on that
    engine)."""
    require_gpu()
    import json
    import os
    import subprocess
    import sys
    members = [dict(nx=512, ny=1024, Re=200.0, Ro=0.0016, levels=1, dt=2e-5, amp=1.0),
               dict(nx=512, ny=1024, Re=450.0, Ro=0.0036, levels=1, dt=2e-5, amp=0.7)]
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, QG_TUNE_CACHE=str(cache), QG_FINE_ROWS="64")
    env.pop("QG_SOLVE_ENGINE", None)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

    def run(force):
        r = subprocess.run([sys.executable, "-c", _CACHE_SCRIPT, json.dumps(members), force],
                           env=env, cwd=root, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        return json.loads(r.stdout.strip().splitlines()[-1])

    run("-")
    lines = [ln.split() for ln in cache.read_text().splitlines() if ln.startswith("group ")]
    assert len(lines) == 1, cache.read_text()
    g = lines[0]
    # group mx my dx dy members esz engine
    assert g[1:3] == ["256", "512"] and float(g[3]) == 1.0 / 256 and float(g[4]) == 2.0 / 512
    assert g[5:7] == ["2", "4"] and int(g[7]) in (32, 33, 34, 50)
    other = "33" if g[7] != "33" else "34"
    cache.write_text(cache.read_text().replace(" ".join(g), " ".join(g[:7] + [other])))
    assert run(other)["same"]
