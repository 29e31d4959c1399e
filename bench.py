#!/usr/bin/env python
"""Throughput benchmark of the CGP quasigeostrophic time step on GB300.

Metric: fine-grid CGPRK3 steps per second (one step = the three TVDRK3 stages
of Section 3.2, each restricting, solving on the elliptic grid, prolonging
and updating the fine grid), for the one-layer double-gyre basin of
Experiment I (Re = 200, Ro = 0.0016) on a 2048 x 4096 fine grid with two
levels of coarsening (elliptic grid 512 x 1024), FP32 fields with FP64
tables and reductions.  Variants (full grid, one level, FP64) are reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed steps, then K steps each bracketed by CUDA events on the
library's stream, with a 256 MiB write between steps to flush the 129 MB
L2 (outside the timed intervals); barrier + synchronize around the region;
the maximum over ranks.  With N > 1 each rank advances its own basin
(independent replicas; a basin does not shard), so the value is the sum of
the ranks' steps over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX, NY, LEVELS = 2048, 4096, 2
RE, RO, DT = 200.0, 0.0016, 2e-6
SEED = 2
METRIC = "fine-grid CGPRK3 steps/s, one-layer 2048x4096 basin, CGP l=2 (elliptic 512x1024), FP32"
UNIT = "steps/s"
WORKLOAD = ("one-layer barotropic double-gyre basin, x in [0,1], y in [-1,1], 2048x4096 "
            "fine intervals, CGP coarsening l=2 (elliptic grid 512x1024), Experiment I "
            "Re=200 Ro=0.0016, dt=2e-6, seeded gyre-like state")
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true",
                    help="run W + K steps of the workload and exit (for ncu captures)")
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--levels", type=int, default=LEVELS)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--study", choices=["mean-fields"],
                    help="long-run time-mean study of Section 5.1 instead of the benchmark")
    ap.add_argument("--experiments", default="I,II")
    ap.add_argument("--t0", type=float, default=10.0)
    ap.add_argument("--t1", type=float, default=50.0)
    ap.add_argument("--study-dt", type=float, default=1e-5)
    ap.add_argument("--study-out", default="")
    ap.add_argument("--realizations", type=int, default=3)
    ap.add_argument("--ensemble", action="store_true",
                    help="with --profile-only: the 96-basin ensemble instead of one basin")
    ap.add_argument("--member-alone", action="store_true",
                    help="with --profile-only: the basin as the one member of an ensemble, "
                         "stepped alone (its solves run as three split launches, one per pass)")
    return ap.parse_args()


def profile_only(args):
    """W + K plain steps of one basin (or, with --ensemble, of the 96-basin
    ensemble), for profiler captures."""
    import torch
    from paper_1308_3290_gb300 import build, inputs, qg
    build.build()
    qg.load()
    if args.ensemble:
        members = ensemble_members()
        ens = qg.Ensemble(members, dtype="f32")
        for i, m in enumerate(members):
            ens.member(i).set_state(inputs.perturbation(m["nx"], m["ny"], seed=1000 + i) * 50.0)
        ens.step(args.warmup + args.steps)
        ens.synchronize()
        print(json.dumps({"profile_only": True, "ensemble": len(members),
                          "kernels_per_step": ens.kernel_count(),
                          "steps": args.warmup + args.steps}))
        ens.close()
        return
    ens = None
    if args.member_alone:
        ens = qg.Ensemble([dict(nx=args.nx, ny=args.ny, Re=RE, Ro=RO, levels=args.levels, dt=DT,
                                amp=1.0)], dtype=args.dtype)
        b = ens.member(0)
    else:
        b = qg.Basin(args.nx, args.ny, Re=RE, Ro=RO, levels=args.levels, dt=DT, dtype=args.dtype)
    b.set_state(inputs.gyre_state(args.nx, args.ny, seed=SEED))
    b.step(args.warmup + args.steps)
    b.synchronize()
    torch.cuda.synchronize()
    print(json.dumps({"profile_only": True, "nx": args.nx, "ny": args.ny,
                      "levels": args.levels, "dtype": args.dtype,
                      "member_alone": args.member_alone, "solve_engine": qg.qg_solve_engine(b.h),
                      "steps": args.warmup + args.steps}))
    if ens is not None:
        ens.close()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def n_unknowns(nx, ny):
    return (nx - 1) * (ny - 1)


def alg_bytes_per_launch(cls, nx, ny, levels, esz):
    """Algorithmic bytes of one launch of each kernel class of the step: every
    field the kernel must read or write once, halos from cache."""
    N = n_unknowns(nx, ny)
    Nc = n_unknowns(nx >> levels, ny >> levels)
    if cls == "fine":
        # fused stage: read w^(s), write w^(s+1), read w^n in stages 2 and 3;
        # l >= 1: read the elliptic-grid psi, write the restricted field;
        # l = 0: read the fine psi
        fine = esz * N * (2 + 3 + 3) / 3.0
        return fine + (esz * N if levels == 0 else 2 * esz * Nc)
    if cls == "restrict":
        return esz * (N + Nc)
    if cls == "prolong":
        return esz * (N + Nc)
    if cls == "solve":
        # x pass (read rhs, write transposed), y pass (read, write), inverse
        # x pass (read, write): six passes over the elliptic grid
        return esz * 6 * Nc
    if cls == "cfl":
        # the adaptive step's reduction reads the step's first streamfunction
        return esz * (N if levels == 0 else Nc)
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the source files each kernel class is built from
KERNEL_SOURCES = {
    "fine": ["fused.cu", "qg_internal.cuh"],
    "solve": ["solve32.cu", "solve.cu", "dst_engine.cuh", "qg_internal.cuh"],
}


def kernel_source_hash(cls):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES.get(cls, []):
        with open(os.path.join(ROOT, "paper_1308_3290_gb300", "csrc", name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(cls):
    """DRAM bytes per launch of kernel class `cls` from the committed ncu
    summary, if it was taken on the current sources of that kernel."""
    p = os.path.join(ROOT, "profiles", "dram_traffic_2048x4096_l2.txt")
    if not os.path.exists(p) or cls not in KERNEL_SOURCES:
        return None
    with open(p) as f:
        d = json.load(f)
    ent = d.get("kernels", {}).get(cls)
    if ent is None or ent.get("source_hash") != kernel_source_hash(cls):
        return None
    return ent.get("bytes_per_launch_full_size")


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def slowest_rank_ms(total_ms, world, device):
    """The job's time: the largest timed total over all ranks."""
    if world == 1:
        return float(total_ms)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, job_ms):
    """Whole-job steps/s: every rank advances its own basin by `steps`."""
    return world * steps / (job_ms / 1e3)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs
b = O.Basin({nx}, {ny}, Re={re}, Ro={ro}, levels={lv}, dt={dt})
w = O.embed(inputs.gyre_state({nx}, {ny}, seed={seed}))
for _ in range({warm}):
    w = O.cgprk3_step(w, b)
t0 = time.perf_counter()
n = 0
while True:
    w = O.cgprk3_step(w, b)
    n += 1
    el = time.perf_counter() - t0
    if n >= {kmax} or el >= {budget}:
        break
print(json.dumps({{"steps": n, "seconds": el}}))
"""


def run_oracle(nx, ny, levels, warm, kmax, budget, threads=1):
    """Time the FP64 oracle in a fresh process with `threads` BLAS threads
    (its sine transforms are matrix products)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    code = ORACLE_SNIPPET.format(root=ROOT, nx=nx, ny=ny, re=RE, ro=RO, lv=levels, dt=DT,
                                 seed=SEED, warm=warm, kmax=kmax, budget=budget)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle run failed: {r.stderr[-2000:]}")
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["steps"], d["seconds"]


def reference_arm(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    kmax = max(1, args.steps)
    steps, sec = run_oracle(NX, NY, LEVELS, warm=min(args.warmup, 1), kmax=kmax, budget=120.0)
    v = steps / sec
    sample = (f"{steps} of the requested {args.steps} CGPRK3 steps of the same 2048x4096 l=2 "
              f"workload after {min(args.warmup, 1)} warm-up step(s), FP64 numpy oracle, "
              f"1 thread (BLAS and numpy)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
        "n_gpus": args.gpus, "steps": steps, "warmup": min(args.warmup, 1),
        "ms_per_step": 1e3 * sec / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "levels": LEVELS, "dt": DT},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def time_steps(torch, qg, h, stream, K, flush):
    """K single steps, each bracketed by CUDA events, L2 flushed between."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    for k in range(K):
        evs[k][0].record(stream)
        qg.qg_step(h, 1)
        evs[k][1].record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def kernel_timing(torch, qg, h, stream, K, flush):
    """Per kernel class: summed device time and launches over K steps.  One
    class is bracketed by events at a time (events between kernels take away
    the next kernel's programmatic early start)."""
    acc = {}
    for cls in qg.KERNEL_CLASSES:
        qg.qg_set_timing_mask(h, [cls])
        for _ in range(K):
            qg.qg_step(h, 1)
            ms, n = qg.qg_read_timing(h)[cls]
            a = acc.setdefault(cls, [0.0, 0])
            a[0] += ms
            a[1] += n
            flush.zero_()
        torch.cuda.synchronize()
    qg.qg_set_timing(h, False)
    return acc


def small_basin_variant(torch, qg, inputs, stream, flush):
    """The 64x128, l = 1 basin (elliptic grid 32x64) in FP32 with the
    autotuned solve and with each kind of solve kernel forced: shared-memory
    FFT (4), warp-group FFT (34) and the matrix form on the tensor cores
    with mma.sync (40) and with tcgen05 (41).  Steps/s of the whole step and
    the mean solve launch."""
    out = {}
    prev = os.environ.get("QG_SOLVE_ENGINE")
    w = inputs.gyre_state(64, 128, seed=SEED)
    try:
        for eng in ("auto", "4", "34", "40", "41"):
            if eng == "auto":
                os.environ.pop("QG_SOLVE_ENGINE", None)
            else:
                os.environ["QG_SOLVE_ENGINE"] = eng
            b = qg.Basin(64, 128, Re=RE, Ro=RO, levels=1, dt=2e-5, dtype="f32", stream=stream)
            b.set_state(w)
            for _ in range(20):
                qg.qg_step(b.h, 1)
            K = 1000
            ts = time_steps(torch, qg, b.h, stream, K, flush)
            kt = kernel_timing(torch, qg, b.h, stream, 50, flush)
            ms, n = kt["solve"]
            out[eng] = {"engine": qg.qg_solve_engine(b.h), "steps_per_s": K / (sum(ts) / 1e3),
                        "ms_per_step": sum(ts) / K, "solve_us": 1e3 * ms / max(1, n)}
            b.close()
    finally:
        if prev is None:
            os.environ.pop("QG_SOLVE_ENGINE", None)
        else:
            os.environ["QG_SOLVE_ENGINE"] = prev
    return out


def ensemble_members(count=96, seed=4):
    """Independent one-layer basins of four sizes, Re ~ U[200, 1000], forcing
    amplitude ~ U[0.5, 1.5], Ro = 0.0016, CGP level 1 or 2, seeded."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = [(128, 256), (256, 512), (512, 1024), (1024, 2048)]
    out = []
    for _ in range(count):
        nx, ny = sizes[rng.integers(0, 4)]
        out.append(dict(nx=int(nx), ny=int(ny), Re=float(rng.uniform(200, 1000)), Ro=RO,
                        levels=int(rng.integers(1, 3)), dt=1e-5,
                        amp=float(rng.uniform(0.5, 1.5))))
    return out


def ensemble_variant(torch, qg, inputs, stream, flush, K=50):
    members = ensemble_members()
    ens = qg.Ensemble(members, dtype="f32", stream=stream)
    for i, m in enumerate(members):
        ens.member(i).set_state(inputs.perturbation(m["nx"], m["ny"], seed=1000 + i) * 50.0)
    ens.step(3)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    for k in range(K):
        evs[k][0].record(stream)
        ens.step(1)
        evs[k][1].record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ens.synchronize()
    points = sum((m["nx"] - 1) * (m["ny"] - 1) for m in members)
    out = {"basins": len(members), "steps_per_s": K / (ms / 1e3), "ms_per_step": ms / K,
           "basin_steps_per_s": len(members) * K / (ms / 1e3),
           "fine_point_steps_per_s": points * K / (ms / 1e3),
           "kernels_per_step": ens.kernel_count()}
    ens.close()
    return out


def ensemble_vs_single(ens, variants):
    """The ensemble's fine point-steps/s against the single 2048x4096 basin's
    in the same run: against the l = 2 rate alone, and against the time its
    members would take at the single basin's per-point rate of their own
    level (l = 1 members do twice the elliptic work per fine point)."""
    pts = (NX - 1) * (NY - 1)
    rate = {lv: variants[f"cgp_l{lv}_f32"]["steps_per_s"] * pts for lv in (1, 2)}
    members = ensemble_members()
    want_s = sum((m["nx"] - 1) * (m["ny"] - 1) / rate[m["levels"]] for m in members)
    return {"fine_point_rate_frac_of_l2": ens["fine_point_steps_per_s"] / rate[2],
            "level_matched_frac": want_s / (ens["ms_per_step"] / 1e3)}


def adjoint_variant(torch, qg, inputs, stream, N=2000, first=1500):
    """Gradient of the kinetic energy averaged over steps 1500..2000 with
    respect to the forcing field, 256x512 basin, l = 1, FP32: forward sweep
    with every state kept, then the reverse sweep (wall-clock seconds)."""
    from paper_1308_3290_gb300 import adjoint
    nx, ny = 256, 512
    b = qg.Basin(nx, ny, Re=RE, Ro=RO, levels=1, dt=5e-5, dtype="f32", stream=stream)
    F = torch.as_tensor(inputs.perturbed_forcing_field(nx, ny, seed=5, Ro=RO),
                        dtype=torch.float32, device="cuda").contiguous().requires_grad_(True)
    w0 = torch.as_tensor(inputs.perturbation(nx, ny, seed=5), dtype=torch.float32, device="cuda")
    # warm-up: a short forward and reverse sweep first (the first reverse
    # sweep of a process pays one-time costs of about 0.7 s)
    Fw = F.detach().clone().requires_grad_(True)
    adjoint.mean_kinetic_energy(Fw, b, w0, 40, 20, 1).backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = adjoint.mean_kinetic_energy(F, b, w0, N, first, 1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"steps": N, "window": [first, N], "J": float(J.detach()), "forward_s": t1 - t0,
           "backward_s": t2 - t1, "grad_norm": float(F.grad.norm())}
    b.close()
    return out


def ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1308_3290_gb300 import build, inputs, qg
    build.build()
    qg.load()

    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    w0 = inputs.gyre_state(NX, NY, seed=SEED + rank)

    def make(levels, dtype):
        b = qg.Basin(NX, NY, Re=RE, Ro=RO, levels=levels, dt=DT, dtype=dtype, stream=stream)
        b.set_state(w0)
        return b

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    basin = make(LEVELS, "f32")
    h = basin.h
    for _ in range(args.warmup):
        qg.qg_step(h, 1)
        flush.zero_()
    torch.cuda.synchronize()
    per_step_kernels = qg.qg_step_kernel_count(h)
    solve_engine = qg.qg_solve_engine(h)
    stencil_tile = qg.qg_stencil_tile(h)

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.2)
    barrier()
    torch.cuda.synchronize()
    times = time_steps(torch, qg, h, stream, args.steps, flush)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    total_ms = slowest_rank_ms(sum(times), world, "cuda")
    value = job_throughput(world, args.steps, total_ms)
    ms_per_step = total_ms / args.steps

    # per-kernel timing (graph with event nodes), for the roofline
    Kt = min(args.steps, 200)
    ktimes = kernel_timing(torch, qg, h, stream, Kt, flush)
    peak, peak_kind = measured_peaks()

    def kernel_roofline(c, kt, levels, K):
        ms, n = kt[c]
        if alg_bytes_per_launch(c, NX, NY, levels, 4) is None:
            return None
        avg_ms = ms / max(1, n)
        algb = alg_bytes_per_launch(c, NX, NY, levels, 4)
        ach = algb / (avg_ms * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": c, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_kind, "traffic": ncu_traffic(c),
                "alg_bytes_per_launch": algb, "avg_launch_ms": avg_ms,
                "ms_per_step": ms / K, "launches_per_step": n / K}

    live = [c for c in ktimes if ktimes[c][1] > 0]
    dom = max(live, key=lambda c: ktimes[c][0])
    roofline = kernel_roofline(dom, ktimes, LEVELS, Kt)
    rooflines = {c: kernel_roofline(c, ktimes, LEVELS, Kt) for c in live}
    rooflines = {c: r for c, r in rooflines.items() if r is not None}

    # end to end through the C ABI with host buffers: every step uploads its
    # input state from page-locked host memory and downloads its result into
    # page-locked host memory; the library's DMA transfers overlap the
    # neighbouring steps (one synchronisation at the end)
    K_e2e = min(args.steps, 100)
    host = torch.empty((NY - 1, NX - 1), dtype=torch.float32, pin_memory=True)
    host.copy_(torch.from_numpy(w0.astype(np.float32)))
    host_out = torch.empty_like(host).pin_memory()
    for _ in range(3):                     # first use makes the staging buffers
        qg.qg_set_state(h, host, 0)
        qg.qg_step(h, 1)
        qg.qg_get_state_async(h, host_out, 0)
    qg.qg_synchronize(h)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K_e2e):
        qg.qg_set_state(h, host, 0)
        qg.qg_step(h, 1)
        qg.qg_get_state_async(h, host_out, 0)
    qg.qg_synchronize(h)
    e2e_s = time.perf_counter() - t0
    barrier()
    # the same exchange with the host waiting for every step's result
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K_e2e):
        qg.qg_set_state(h, host, 0)
        qg.qg_step(h, 1)
        qg.qg_get_state(h, host_out, 0)
        stream.synchronize()
    serial_s = time.perf_counter() - t0
    nbytes = 4 * (NX - 1) * (NY - 1)
    e2e = {"value": world * K_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes,
           "how": "per step: qg_set_state from page-locked host (DMA upload overlapping the "
                  "step before), qg_step(1), qg_get_state_async to page-locked host (DMA "
                  "download overlapping the step after); one qg_synchronize at the end",
           "serial_steps_per_s": world * K_e2e / serial_s}
    basin.close()

    variants = {}
    if not args.no_variants:
        for name, lv, dt in (("cgp_l2_f32", 2, "f32"), ("cgp_l1_f32", 1, "f32"),
                             ("full_grid_l0_f32", 0, "f32"), ("cgp_l2_f64", 2, "f64"),
                             ("full_grid_l0_f64", 0, "f64")):
            b = make(lv, dt)
            for _ in range(5):
                qg.qg_step(b.h, 1)
            K = 200 if dt == "f32" else 20
            ts = time_steps(torch, qg, b.h, stream, K, flush)
            variants[name] = {"steps_per_s": K / (sum(ts) / 1e3), "ms_per_step": sum(ts) / K,
                              "solve_engine": qg.qg_solve_engine(b.h)}
            if name == "full_grid_l0_f32":
                # the full-grid solve streams from HBM (its fields exceed L2)
                kt = kernel_timing(torch, qg, b.h, stream, 50, flush)
                variants[name]["rooflines"] = {
                    c: kernel_roofline(c, kt, 0, 50) for c in kt if kt[c][1] > 0}
            b.close()
        # the same workload with the adaptive step of Eq. dt (c = 0.5, capped
        # by dt) and with the time-mean streamfunction accumulated
        for name, setup in (("cgp_l2_f32_adaptive_dt", lambda h: qg.qg_set_cfl(h, 0.5)),
                            ("cgp_l2_f32_time_mean_psi", lambda h: qg.qg_stats_begin(h))):
            b = make(LEVELS, "f32")
            setup(b.h)
            for _ in range(5):
                qg.qg_step(b.h, 1)
            ts = time_steps(torch, qg, b.h, stream, 200, flush)
            variants[name] = {"steps_per_s": 200 / (sum(ts) / 1e3), "ms_per_step": sum(ts) / 200}
            b.close()
        # CGP with a costlier elliptic solver (Section 3: CGP does not depend
        # on the solver): 3 warm-started V(2,2) multigrid cycles per solve
        for name, lv in (("cgp_l2_f32_multigrid", 2), ("cgp_l1_f32_multigrid", 1),
                         ("full_grid_l0_f32_multigrid", 0)):
            b = make(lv, "f32")
            qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 3)
            b.set_state(w0)
            for _ in range(5):
                qg.qg_step(b.h, 1)
            K = 100 if lv > 0 else 20
            ts = time_steps(torch, qg, b.h, stream, K, flush)
            variants[name] = {"steps_per_s": K / (sum(ts) / 1e3), "ms_per_step": sum(ts) / K,
                              "kernels_per_step": qg.qg_step_kernel_count(b.h)}
            b.close()
        # two-layer basin of Table 2 Experiment 1 (Section 2.2): square
        # basin, 1024x2048 intervals per layer, l = 1, FP32
        tl = dict(Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3)
        b = qg.Basin(1024, 2048, Re=tl["Ro"] / 3.57e-7, levels=1, dt=1e-5, dtype="f32",
                     layers=2, y0=-0.5, y1=0.5, stream=stream, **tl)
        b.set_state(inputs.smooth_field(1024, 2048, seed=3, amp=0.05, noise=0.01), 0)
        b.set_state(inputs.smooth_field(1024, 2048, seed=4, amp=0.02, noise=0.01), 1)
        for _ in range(5):
            qg.qg_step(b.h, 1)
        ts = time_steps(torch, qg, b.h, stream, 100, flush)
        variants["two_layer_1024x2048_l1_f32"] = {"steps_per_s": 100 / (sum(ts) / 1e3),
                                                  "ms_per_step": sum(ts) / 100}
        b.close()
        variants["small_64x128_l1_f32"] = small_basin_variant(torch, qg, inputs, stream, flush)
        variants["ensemble_96_f32"] = ens = ensemble_variant(torch, qg, inputs, stream, flush)
        ens["vs_single_basin"] = ensemble_vs_single(ens, variants)
        variants["adjoint_256x512_l1_f32"] = adjoint_variant(torch, qg, inputs, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        steps, sec = run_oracle(NX, NY, LEVELS, warm=0, kmax=2, budget=25.0)
        cpu = {"value": steps / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{steps} CGPRK3 step(s) of the same 2048x4096 l=2 workload, "
                         f"FP64 numpy oracle, 1 thread"}
        ncores = os.cpu_count() or 1
        if ncores > 1:
            steps, sec = run_oracle(NX, NY, LEVELS, warm=1, kmax=4, budget=15.0, threads=ncores)
            cpu["all_cores"] = {"value": steps / sec, "unit": UNIT, "cores": ncores,
                                "sample": f"{steps} step(s) after 1 warm-up step, {ncores} BLAS threads"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "levels": LEVELS,
                       "Re": RE, "Ro": RO, "dt": DT,
                       "l2": "256 MiB write between timed steps (outside the timed intervals)",
                       "parallelism": f"{world} independent replica(s)"},
            "roofline": roofline, "rooflines": rooflines, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": per_step_kernels * args.steps,
            "solve_engine": solve_engine,
            "stencil_tile": {"rows_per_cta": stencil_tile[0], "rows_per_thread": stencil_tile[1]},
            "clocks": clocks, "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# long-run statistics (Section 5.1)
# ---------------------------------------------------------------------------

# (label, nx, ny, levels): the 256 x 512 DNS, CGP of it at l = 1, 2, 3, and
# the three runs whose elliptic grid is 16 x 32 (Figs. of the 16 x 32 set).
# Every run is repeated from `--realizations` starts: realization 0 from
# rest (the paper's start), realization r >= 1 from a seeded 1e-3
# perturbation of rest; the spread of the DNS realizations' means is the
# sampling noise of a time mean over the window.
STUDY_RUNS = [
    ("DNS 256x512:256x512", 256, 512, 0),
    ("CGP 256x512:128x256", 256, 512, 1),
    ("CGP 256x512:64x128", 256, 512, 2),
    ("CGP 256x512:32x64", 256, 512, 3),
    ("coarse 16x32:16x32", 16, 32, 0),
    ("CGP 32x64:16x32", 32, 64, 1),
    ("CGP 64x128:16x32", 64, 128, 2),
]
STUDY_EXPERIMENTS = {"I": (200.0, 0.0016), "II": (312.5, 0.0025)}


def study_mean_fields(args):
    """Time-mean streamfunction and potential vorticity of each run in
    STUDY_RUNS over t in [t0, t1] (Section 5.1: t in [10, 50], Exp I and
    II), every realization of every run one member of an ensemble stepped
    together at a fixed dt.  Each run's mean over its realizations is
    compared with the DNS mean over its realizations at the run's own nodes
    (relative L2), next to the spread of single DNS realizations."""
    import numpy as np
    import torch
    from paper_1308_3290_gb300 import build, inputs, qg
    build.build()
    qg.load()
    n0 = int(round(args.t0 / args.study_dt))
    n1 = int(round(args.t1 / args.study_dt))
    R = args.realizations
    chunk = 20000
    report = {"study": "time-mean psi and q, Section 5.1", "t0": args.t0, "t1": args.t1,
              "dt": args.study_dt, "steps": n1, "mean_over_steps": n1 - n0, "dtype": "f32",
              "realizations": R, "experiments": {}}
    names = args.experiments.split(",")
    members, owner = [], []
    for name in names:
        Re, Ro = STUDY_EXPERIMENTS[name]
        for ri, run in enumerate(STUDY_RUNS):
            for r in range(R):
                members.append(dict(nx=run[1], ny=run[2], Re=Re, Ro=Ro, levels=run[3],
                                    dt=args.study_dt))
                owner.append((name, ri, r))
    ens = qg.Ensemble(members, dtype="f32")
    for i, m in enumerate(members):
        r = owner[i][2]
        w0 = np.zeros((m["ny"] - 1, m["nx"] - 1))
        if r > 0:
            w0 = 1e-3 * inputs.perturbation(m["nx"], m["ny"], seed=100 + r)
        ens.member(i).set_state(w0)
    t_start = time.perf_counter()
    done = 0
    while done < n0:
        k = min(chunk, n0 - done)
        ens.step(k)
        done += k
    ens.synchronize()
    for i in range(len(members)):
        qg.qg_stats_begin(ens.member(i).h)
    while done < n1:
        k = min(chunk, n1 - done)
        ens.step(k)
        done += k
    ens.synchronize()
    wall = time.perf_counter() - t_start
    report["wall_s"] = wall
    report["ensemble_members"] = len(members)
    report["ensemble_steps_per_s"] = n1 / wall

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    for name in names:
        Re, Ro = STUDY_EXPERIMENTS[name]
        means = {}   # run index -> list of (psi mean, q mean)
        for i, (nm, ri, r) in enumerate(owner):
            if nm != name:
                continue
            v = ens.member(i)
            outp = torch.empty((v.ny - 1, v.nx - 1), dtype=torch.float32, device="cuda")
            outq = torch.empty_like(outp)
            qg.qg_stats_mean_psi(v.h, outp)
            qg.qg_stats_mean_q(v.h, outq)
            ens.synchronize()
            means.setdefault(ri, []).append((outp.double().cpu().numpy(), outq.double().cpu().numpy()))
        dns_p = np.mean([m[0] for m in means[0]], axis=0)
        dns_q = np.mean([m[1] for m in means[0]], axis=0)
        runs = []
        for ri, (label, nx, ny, lv) in enumerate(STUDY_RUNS):
            s = 256 // nx
            ref_p, ref_q = dns_p[s - 1::s, s - 1::s], dns_q[s - 1::s, s - 1::s]
            mp = np.mean([m[0] for m in means[ri]], axis=0)
            mq = np.mean([m[1] for m in means[ri]], axis=0)
            entry = {"run": label, "levels": lv,
                     "rel_l2_psi_vs_dns": rel(mp, ref_p), "rel_l2_q_vs_dns": rel(mq, ref_q),
                     "psi_min": float(mp.min()), "psi_max": float(mp.max()),
                     "single_realization_rel_l2_psi":
                         [rel(m[0], ref_p) for m in means[ri]]}
            runs.append(entry)
        spread = [rel(m[0], dns_p) for m in means[0]]
        report["experiments"][name] = {
            "Re": Re, "Ro": Ro, "runs": runs,
            "dns_single_realization_spread_psi": spread,
            "noise_floor_psi": float(np.sqrt(2.0 / R) * np.sqrt(np.mean(np.square(spread))) *
                                     np.sqrt(R / max(R - 1, 1))),
        }
        print(json.dumps({"experiment": name, **report["experiments"][name]}), flush=True)
    print(json.dumps({"wall_s": wall, "ensemble_steps_per_s": n1 / wall}), flush=True)
    ens.close()
    if args.study_out:
        with open(args.study_out, "w") as f:
            json.dump(report, f, indent=1)


def main():
    args = parse()
    if args.study:
        study_mean_fields(args)
    elif args.profile_only:
        profile_only(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
