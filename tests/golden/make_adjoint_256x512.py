"""Write adjoint_256x512_l1.txt: the time-mean kinetic energy J and its
gradient with respect to the wind-forcing field, computed by the FP64
oracle's adjoint, for the adjoint workload at its own size.

Workload: one-layer basin [0, 1] x [-1, 1] with 256 x 512 intervals, CGP at
level 1, Experiment I parameters (Table 1: Re = 200, Ro = 0.0016), fixed
dt = 5e-5 (TVDRK3, Section 4.2), forcing sin(pi y)/Ro plus a seeded smooth
perturbation (seed 5), initial state the seeded N(0, 1e-2) perturbation of
rest (seed 5); J = mean of the kinetic energy (Section 5.2) of psi^n over
the steps n = 1500..2000.  The gradient dJ/dF is stored through its inner
products with 16 seeded directions of unit root-mean-square value (seed 51)
and its L2 norm.  The oracle's adjoint is pinned to differences of the
forward oracle by tests/test_oracle_adjoint.py.

This script calls only the oracle and the seeded input generator:

    OMP_NUM_THREADS=4 python tests/golden/make_adjoint_256x512.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import qg_adjoint as AD  # noqa: E402
from oracle import qg_oracle as O  # noqa: E402
from paper_1308_3290_gb300 import inputs  # noqa: E402

NX, NY, LEVELS, DT, N, FIRST = 256, 512, 1, 5e-5, 2000, 1500
RE, RO = 200.0, 0.0016
SEED, DIR_SEED, NDIR = 5, 51, 16
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_256x512_l1.txt")


def main():
    t0 = time.time()
    b = O.Basin(NX, NY, Re=RE, Ro=RO, levels=LEVELS, dt=DT)
    F = inputs.perturbed_forcing_field(NX, NY, seed=SEED, Ro=RO)
    w0 = inputs.perturbation(NX, NY, seed=SEED)
    J, g = AD.mean_energy_gradient(w0, b, F, N, FIRST)
    d = inputs.unit_directions(NX, NY, NDIR, seed=DIR_SEED)
    proj = [float(np.sum(g * d[k])) for k in range(NDIR)]
    with open(OUT, "w") as f:
        f.write("# Time-mean kinetic energy J (Section 5.2) over steps 1500..2000 of the\n")
        f.write("# 256 x 512, l = 1 Experiment I basin (Table 1), dt = 5e-5, forcing\n")
        f.write("# sin(pi y)/Ro + seeded perturbation (seed 5), state seed 5, and dJ/dF as\n")
        f.write("# inner products with 16 unit-RMS directions (seed 51) and its L2 norm.\n")
        f.write("# Written by tests/golden/make_adjoint_256x512.py from the FP64 oracle.\n")
        f.write(f"J {J!r}\n")
        f.write(f"grad_norm {float(np.linalg.norm(g))!r}\n")
        f.write("projections " + " ".join(repr(p) for p in proj) + "\n")
    print(open(OUT).read())
    print(f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
