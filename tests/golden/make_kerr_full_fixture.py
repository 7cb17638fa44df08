"""Write tests/golden/kerr_a0.9_8192x128_1e5.txt with the FP64 oracle only.

The Kerr workload in full: a = 0.9, s = -2, m = 2, 8192 x 128, r* in
[-100, 600], prograde orbit r0 = 10 with a Gaussian source of width 0.05,
zero initial data, 1e5 steps of Eqs. (3)-(4) with dt from the time-step rule
(c_r = 0.5, c_theta = 0.1).  Stored (text, complex as re im pairs):
  * the waveform at r* = 20 every 100 steps, projected on -2Y_22 (1000 values);
  * the final Phi and Pi on rows i = 200, 1300, 4096, 7000 (4 x 128 values each).

    python tests/golden/make_kerr_full_fixture.py      # ~10 min on 8 cores
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kerr_a0.9_8192x128_1e5.txt")
ROWS = (200, 1300, 4096, 7000)
NR, NTH, RMIN, RMAX, A, S, M = 8192, 128, -100.0, 600.0, 0.9, -2, 2
STEPS, EVERY, REXT = 100000, 100, 20.0


def y22(nth):
    # -2Y_22 theta-part, sqrt(5 / (64 pi)) (1 + cos theta)^2, midpoint weights
    th = (np.arange(nth) + 0.5) * np.pi / nth
    return 2 * np.pi * np.sqrt(5 / (64 * np.pi)) * (1 + np.cos(th)) ** 2 * np.sin(th) * (np.pi / nth)


def main():
    dt = O.stable_dt(NR, NTH, RMIN, RMAX, A, S, M, 0.5, 0.1)
    sol = O.Solver(NR, NTH, RMIN, RMAX, dt, A, S, M)
    sol.set_initial(np.zeros((NR, NTH), complex))
    sol.set_source(r0=10.0, sigma=0.05, amplitude=1.0, prograde=True)
    sol.set_extraction(REXT, EVERY)
    sol.step(STEPS)
    t, rows = sol.samples()
    proj = rows @ y22(NTH)
    phi, pi = sol.state()
    with open(OUT, "w") as f:
        f.write("# FP64 oracle, Kerr a=0.9 s=-2 m=2 8192x128 r*[-100,600] r0=10 sigma=0.05, 1e5 steps\n")
        f.write("# dt %.17g\n" % dt)
        f.write("# waveform r*=20 every 100 steps projected on -2Y22: t re im\n")
        for tk, z in zip(t, proj):
            f.write("W %.17g %.17g %.17g\n" % (tk, z.real, z.imag))
        for i in ROWS:
            for j in range(NTH):
                f.write("S %d %d %.17g %.17g %.17g %.17g\n" % (i, j, phi[i, j].real, phi[i, j].imag,
                                                            pi[i, j].real, pi[i, j].imag))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
