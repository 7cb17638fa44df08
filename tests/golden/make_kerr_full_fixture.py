"""Write tests/golden/kerr_a0.9_8192x128_1e5.txt with the FP64 oracle only.

The Kerr workload in full: a = 0.9, s = -2, m = 2, 8192 x 128, r* in
[-100, 1000], prograde orbit r0 = 10 with a Gaussian source of width 0.05,
zero initial data, 1e5 steps of Eqs. (3)-(4) with the time-step rule
(c_r = 0.5, c_theta = 0.8) and the angular Kreiss-Oliger dissipation
(eps = 1) of the workload.  Stored (text, complex as re im pairs):
  * the waveform at r* = 500 every 100 steps projected on -2Y_22 (1000 values);
  * max |Phi| and max |Pi| over the grid every 1000 steps (100 pairs);
  * the final Phi and Pi on rows i = 200, 1300, 4096, 7000 (4 x 128 values each).

    python tests/golden/make_kerr_full_fixture.py      # ~50 min on 8 cores
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1206_0270_gb300 import inputs  # noqa: E402  (workload parameters only)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kerr_a0.9_8192x128_1e5.txt")
ROWS = (200, 1300, 4096, 7000)
EVERY, REXT, CHUNK = 100, 500.0, 1000


def y22(nth):
    # -2Y_22 theta-part, sqrt(5 / (64 pi)) (1 + cos theta)^2, midpoint weights
    th = (np.arange(nth) + 0.5) * np.pi / nth
    return 2 * np.pi * np.sqrt(5 / (64 * np.pi)) * (1 + np.cos(th)) ** 2 * np.sin(th) * (np.pi / nth)


def main():
    w = inputs.WORKLOADS["kerr_a0.9_s-2_m2_8192x128_r0_10"]
    nr, nth, rmin, rmax = w["nr"], w["nth"], w["rstar_min"], w["rstar_max"]
    dt = O.stable_dt(nr, nth, rmin, rmax, w["a"], w["s"], w["m"], w["c_r"], w["c_theta"])
    sol = O.Solver(nr, nth, rmin, rmax, dt, w["a"], w["s"], w["m"])
    sol.set_dissipation(w["eps"])
    sol.set_initial(np.zeros((nr, nth), complex))
    sol.set_source(**w["source"])
    sol.set_extraction(REXT, EVERY)
    hist = []
    while sol.step_count < w["steps"]:
        sol.step(CHUNK)
        phi, pi = sol.state()
        hist.append((sol.step_count, abs(phi).max(), abs(pi).max()))
    t, rows = sol.samples()
    proj = rows @ y22(nth)
    phi, pi = sol.state()
    with open(OUT, "w") as f:
        f.write("# FP64 oracle, Kerr a=%g s=%d m=%d %dx%d r*[%g,%g] r0=%g sigma=%g, %d steps, c_theta %g eps %g\n"
                % (w["a"], w["s"], w["m"], nr, nth, rmin, rmax, w["source"]["r0"], w["source"]["sigma"],
                   w["steps"], w["c_theta"], w["eps"]))
        f.write("# dt %.17g\n" % dt)
        f.write("# W: waveform r*=%g every %d steps projected on -2Y22: t re im\n" % (REXT, EVERY))
        for tk, z in zip(t, proj):
            f.write("W %.17g %.17g %.17g\n" % (tk, z.real, z.imag))
        f.write("# H: step max|Phi| max|Pi| every %d steps\n" % CHUNK)
        for n, a, b in hist:
            f.write("H %d %.17g %.17g\n" % (n, a, b))
        f.write("# S: i j Phi(re im) Pi(re im) of the final state\n")
        for i in ROWS:
            for j in range(nth):
                f.write("S %d %d %.17g %.17g %.17g %.17g\n" % (i, j, phi[i, j].real, phi[i, j].imag,
                                                            pi[i, j].real, pi[i, j].imag))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
