"""Run the library's main paths at small sizes under the bounds-checked
build (libqgcgp_bounds.so, compiled with QG_BOUNDS_CHECK) and print the
site of the first failed index check (0: none).

Executed in a process of its own by tests/test_gpu_bounds_check.py: the
checked library must be the only one the process loads.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1308_3290_gb300 import adjoint, build, inputs, qg  # noqa: E402


def basin(nx, ny, levels, dtype, **kw):
    return qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=5e-5, dtype=dtype, **kw)


def run_steps(b, nx, ny, n=3, seed=1):
    b.set_state(inputs.perturbation(nx, ny, seed=seed) * 20.0)
    b.step(n)
    b.diagnostics()
    b.psi()


def main():
    qg.load(build.build(variant="bounds"))
    site = {}

    def check(name):
        s = qg.qg_bounds_check_result()
        site[name] = s
        print(f"{name}: {s}", flush=True)

    # every solve engine on one- and two-layer grids, FP32 and FP64, l = 0..3
    for engine in (4, 16, 32, 33, 34, 40):
        os.environ["QG_SOLVE_ENGINE"] = str(engine)
        for dtype in ("f32", "f64"):
            for nx, ny, lv in ((64, 128, 0), (64, 128, 1), (128, 64, 2), (128, 256, 3)):
                b = basin(nx, ny, lv, dtype)
                run_steps(b, nx, ny)
                b.poisson_solve(inputs.smooth_field(nx >> lv, ny >> lv, seed=2), lv)
                b.close()
        check(f"engine {engine}")
    # engine 41 (tcgen05, sides of 16 to 64 intervals), one basin and a batch
    os.environ["QG_SOLVE_ENGINE"] = "41"
    for nx, ny, lv in ((32, 64, 0), (64, 128, 1), (64, 64, 0), (128, 256, 2)):
        b = basin(nx, ny, lv, "f32")
        run_steps(b, nx, ny)
        b.poisson_solve(inputs.smooth_field(nx >> lv, ny >> lv, seed=2), lv)
        b.close()
    ens = qg.Ensemble([dict(nx=32, ny=64, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, amp=1.0),
                       dict(nx=64, ny=128, Re=300.0, Ro=0.0016, levels=1, dt=1e-4, amp=1.0)],
                      dtype="f32")
    for i, (nx, ny) in enumerate(((32, 64), (64, 128))):
        ens.member(i).set_state(inputs.perturbation(nx, ny, seed=7 + i) * 20.0)
    ens.step(3)
    ens.synchronize()
    ens.close()
    check("engine 41")
    # engine 50 (sides of 512 intervals and more): remainder passes of radix
    # 2, 4 and 8 and none, 1, 2 and 4 pairs per CTA, one and two layers
    os.environ["QG_SOLVE_ENGINE"] = "50"
    for dtype in ("f32", "f64"):
        for nx, ny, lv in ((512, 1024, 0), (1024, 2048, 1), (2048, 512, 0), (512, 4096, 0)):
            b = basin(nx, ny, lv, dtype)
            run_steps(b, nx, ny)
            b.poisson_solve(inputs.smooth_field(nx >> lv, ny >> lv, seed=2), lv)
            b.close()
        b = qg.Basin(512, 512, Re=697.16, Ro=2.49e-4, levels=0, dt=1e-5, dtype=dtype, layers=2,
                     Fr=0.087, delta=0.2, sigma=1.43e-3, y0=-0.5, y1=0.5)
        b.set_state(inputs.smooth_field(512, 512, seed=5, amp=0.05), 0)
        b.set_state(inputs.smooth_field(512, 512, seed=6, amp=0.02), 1)
        b.step(3)
        b.synchronize()
        b.close()
    check("engine 50")
    del os.environ["QG_SOLVE_ENGINE"]
    # every fine-stage tile height, with a forcing field and the adaptive step
    for tile in ("128", "64", "32", "64x4", "32x4"):
        os.environ["QG_FINE_ROWS"] = tile
        for lv in ((0, 1, 2) if "x4" in tile else (0, 1, 2, 3, 4)):
            b = basin(256, 512, lv, "f32")
            b.set_forcing(inputs.perturbed_forcing_field(256, 512, seed=3, Ro=0.0016))
            qg.qg_set_cfl(b.h, 0.5)
            run_steps(b, 256, 512)
            b.close()
        check(f"tile {tile}")
    del os.environ["QG_FINE_ROWS"]
    # transfers
    b = basin(128, 256, 3, "f32")
    for lv in (1, 2, 3):
        c = b.restrict(inputs.random_field(128, 256, seed=4), lv)
        b.prolong(c, lv)
    b.close()
    check("transfers")
    # two layers (Section 2.2), l = 0 and 1
    for lv in (0, 1):
        b = qg.Basin(64, 64, Re=697.16, Ro=2.49e-4, levels=lv, dt=1e-5, dtype="f32", layers=2,
                     Fr=0.087, delta=0.2, sigma=1.43e-3, y0=-0.5, y1=0.5)
        b.set_state(inputs.smooth_field(64, 64, seed=5, amp=0.05), 0)
        b.set_state(inputs.smooth_field(64, 64, seed=6, amp=0.02), 1)
        b.step(3)
        b.synchronize()
        b.close()
    check("two layers")
    # multigrid solver
    b = basin(128, 256, 1, "f32")
    qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 3)
    run_steps(b, 128, 256)
    b.close()
    check("multigrid")
    # adjoint through the autograd wrapper, checkpointed tape
    b = basin(64, 128, 1, "f32")
    F = torch.as_tensor(inputs.perturbed_forcing_field(64, 128, seed=5, Ro=0.0016),
                        dtype=torch.float32, device="cuda").contiguous().requires_grad_(True)
    w0 = torch.as_tensor(inputs.perturbation(64, 128, seed=5), dtype=torch.float32, device="cuda")
    adjoint.mean_kinetic_energy(F, b, w0, 20, 10, 4).backward()
    b.close()
    check("adjoint")
    # batched ensemble of uneven members (warp-group and matrix-form solves)
    members = [dict(nx=nx, ny=ny, Re=200.0, Ro=0.0016, levels=lv, dt=5e-5)
               for nx, ny, lv in ((32, 64, 0), (64, 128, 1), (128, 256, 2), (256, 128, 3),
                                  (128, 256, 1), (256, 512, 2))]
    for dtype in ("f32", "f64"):
        ens = qg.Ensemble(members, dtype=dtype)
        for i, m in enumerate(members):
            ens.member(i).set_state(inputs.perturbation(m["nx"], m["ny"], seed=10 + i))
        ens.step(3)
        ens.synchronize()
        ens.close()
    check("ensemble")
    # the allocation-free solve
    rhs = torch.as_tensor(inputs.smooth_field(64, 128, seed=7), dtype=torch.float32,
                          device="cuda").contiguous()
    out = torch.empty_like(rhs)
    qg.qg_poisson_solve_noalloc(64, 128, 1 / 64, 2 / 128, qg.QG_F32, rhs, out,
                                torch.cuda.current_stream().cuda_stream)
    check("noalloc")
    bad = {k: v for k, v in site.items() if v != 0}
    print("FIRST_FAILED_SITE", next(iter(bad.values())) if bad else 0)
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
