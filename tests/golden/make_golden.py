"""Writes the stored expected values under tests/golden/ by calling only the
oracle (and the seeded input generators).  Run: python tests/golden/make_golden.py

tg32_fp64.txt: Taylor-Green vortex (the initial field of Sec. 4, Eq. TG) on
a 32^3 mesh, nu = 0.01, dt = 0.01, 100 classical RK4 steps of Eq. NSfinal
with 2/3-rule dealiasing; kinetic energy E and dissipation eps after every
step, from the FP64 oracle."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1607_00850_gb300 import inputs  # noqa: E402


def tg32(path):
    o = oracle.load()
    N, nu, dt, steps = 32, 0.01, 0.01, 100
    u = inputs.taylor_green(N)
    rows = [(0, 0.0, o.energy(u), o.dissipation(u, nu))]
    for n in range(1, steps + 1):
        u = o.rk4(u, nu, dt, 1)
        rows.append((n, n * dt, o.energy(u), o.dissipation(u, nu)))
    with open(path, "w") as f:
        f.write("# Taylor-Green vortex (Sec. 4, Eq. TG), N=32, nu=0.01, dt=0.01, classical RK4 of\n")
        f.write("# Eq. NSfinal with 2/3-rule dealiasing; written by tests/golden/make_golden.py (FP64 oracle)\n")
        f.write("# step t E eps\n")
        for r in rows:
            f.write(f"{r[0]:d} {r[1]:.2f} {r[2]:.17e} {r[3]:.17e}\n")


if __name__ == "__main__":
    tg32(os.path.join(HERE, "tg32_fp64.txt"))
