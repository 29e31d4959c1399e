"""Write mean_ke_64x128_l1.txt: the time-mean basin kinetic energy of the
one-layer Experiment I basin computed by the FP64 oracle.

Workload: Table 1's Experiment I (Re = 200, Ro = 0.0016), basin
[0, 1] x [-1, 1] with 64 x 128 intervals, CGP at level 1 (elliptic grid
32 x 64, Section 3), fixed dt = 1e-4 (TVDRK3, Section 4.2), started from rest
plus the seeded N(0, 1e-2) perturbation (seed 1).  The kinetic energy is
Section 5.2's E = 1/2 iint |grad psi|^2 of psi^n, the CGP streamfunction of
the step's first stage; it is sampled every 20 steps over t in [10, 50], the
window of Section 5.1 (20 000 snapshots, as there).  The file also holds the
means over the four 10-unit sub-windows, a measure of the sampling noise of
the chaotic flow, and the energy history every 200 steps from t = 0.

This script calls only the oracle and the seeded input generator:

    OMP_NUM_THREADS=1 python tests/golden/make_mean_ke.py     # about 35 min
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import qg_oracle as O  # noqa: E402
from paper_1308_3290_gb300 import inputs  # noqa: E402

NX, NY, LEVELS, DT, SEED = 64, 128, 1, 1e-4, 1
RE, RO = 200.0, 0.0016
T0, T1, EVERY = 10.0, 50.0, 20
SERIES = 200         # the energy history is kept every 200 steps (t = 0.02)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mean_ke_64x128_l1.txt")


def main():
    b = O.Basin(NX, NY, Re=RE, Ro=RO, levels=LEVELS, dt=DT)
    w = O.embed(inputs.perturbation(NX, NY, seed=SEED))
    n0, n1 = int(round(T0 / DT)), int(round(T1 / DT))
    ke = []
    series = []          # (step, KE) every SERIES steps from the start
    t_start = time.time()
    for n in range(n1 + 1):
        take = n >= n0 and (n - n0) % EVERY == 0 and n < n1
        if take or n % SERIES == 0:
            e = O.kinetic_energy(O.cgp_psi(w, b), b.dx, b.dy)
            if take:
                ke.append(e)
            if n % SERIES == 0:
                series.append((n, e))
        if n == n1:
            break
        w = O.cgprk3_step(w, b)
        if n % 50000 == 0:
            print(f"step {n} of {n1}, {time.time() - t_start:.0f} s", flush=True)
    ke = np.array(ke)
    quarters = [float(np.mean(q)) for q in np.array_split(ke, 4)]
    with open(OUT, "w") as f:
        f.write("# Time-mean kinetic energy (Section 5.2) of the one-layer Experiment I basin\n")
        f.write("# (Table 1: Re = 200, Ro = 0.0016), 64 x 128 intervals, CGP level 1, dt = 1e-4,\n")
        f.write("# from rest + seeded N(0, 1e-2) perturbation (seed 1), psi^n sampled every\n")
        f.write("# 20 steps over t in [10, 50] (Section 5.1's window).  Written by\n")
        f.write("# tests/golden/make_mean_ke.py from the FP64 oracle alone.\n")
        f.write(f"nx {NX}\nny {NY}\nlevels {LEVELS}\ndt {DT!r}\nseed {SEED}\n")
        f.write(f"t0 {T0!r}\nt1 {T1!r}\nevery {EVERY}\nsamples {ke.size}\n")
        f.write(f"mean_ke {float(np.mean(ke))!r}\n")
        f.write(f"std_ke {float(np.std(ke))!r}\n")
        f.write("quarter_means " + " ".join(repr(q) for q in quarters) + "\n")
        f.write(f"final_ke {float(ke[-1])!r}\n")
        f.write("# energy history: step  KE, every 200 steps from rest\n")
        for n, e in series:
            f.write(f"ke_at {n} {e!r}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
