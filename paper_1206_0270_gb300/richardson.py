"""Richardson extrapolation of waveforms over a resolution ladder, and the
spin-weighted spherical-harmonic projection of the extracted field.

The paper ("Mathematical Advances", item 3) improves its second-order
solutions by Richardson extrapolation, and estimates their error by computing
the waveform's Richardson extrapolant two ways and taking the relative
difference (footnote to the "Accuracy" section).  Here:

  * a ladder of runs halves h, dtheta and dt at each level (nr -> 2 nr - 1 so
    the r* nodes nest, nth -> 2 nth, dt -> dt / 2, sampling interval in steps
    doubled so that all levels sample at the same times); the levels run
    together as one teuk_batch;
  * each level's waveform rows Phi(t, r*_ext, theta_j) are projected on
    sY_lm(theta) (the theta grids do not nest, the projection does);
  * R(h, h/2) = (4 f(h/2) - f(h)) / 3 removes the O(h^2) error; with three
    levels the error estimate is |R(h, h/2) - R(h/2, h/4)| / |R(h/2, h/4)|.

This is post-processing of extracted waveforms (host numpy); the evolutions
themselves run in libteuk.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def swsh_theta(s: int, l: int, m: int, theta: np.ndarray) -> np.ndarray:
    """theta-part of the spin-weighted spherical harmonic sY_lm (the full
    function is this times e^{i m phi}), by the explicit finite sum of
    Goldberg et al., J. Math. Phys. 8, 2155 (1967):
      sY_lm = (-1)^m sqrt((l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)) sin^{2l}(theta/2)
              sum_r C(l-s, r) C(l+s, r+s-m) (-1)^{l-r-s} cot^{2r+s-m}(theta/2)."""
    if l < max(abs(m), abs(s)):
        raise ValueError("need l >= max(|m|, |s|)")
    theta = np.asarray(theta, dtype=float)
    f = math.factorial
    pref = (-1) ** m * math.sqrt(f(l + m) * f(l - m) * (2 * l + 1) / (4 * math.pi * f(l + s) * f(l - s)))
    half = theta / 2.0
    sin_h, cos_h = np.sin(half), np.cos(half)
    out = np.zeros_like(theta)
    for r in range(0, l - s + 1):
        k = r + s - m
        if k < 0 or k > l + s:
            continue
        c = math.comb(l - s, r) * math.comb(l + s, k) * (-1) ** (l - r - s)
        # sin^{2l}(t/2) cot^{2r+s-m}(t/2) = sin^{2l-(2r+s-m)} cos^{2r+s-m}
        p = 2 * r + s - m
        out = out + c * sin_h ** (2 * l - p) * cos_h ** p
    return pref * out


def project(phi_rows: np.ndarray, s: int, l: int, m: int) -> np.ndarray:
    """Phi_lm(t) = 2 pi sum_j Phi(t, theta_j) sY_lm(theta_j) sin(theta_j) dtheta
    (sY_lm's theta-part is real; the e^{i m phi} of Eq. 2 integrates against
    e^{-i m phi} to 2 pi), midpoint rule on theta_j = (j + 1/2) pi / nth."""
    phi_rows = np.asarray(phi_rows)
    nth = phi_rows.shape[-1]
    th = (np.arange(nth) + 0.5) * (np.pi / nth)
    w = 2.0 * np.pi * swsh_theta(s, l, m, th) * np.sin(th) * (np.pi / nth)
    return phi_rows @ w


def extrapolate(f_h: np.ndarray, f_h2: np.ndarray) -> np.ndarray:
    """Richardson extrapolant of a second-order quantity from steps h and h/2."""
    return (4.0 * np.asarray(f_h2) - np.asarray(f_h)) / 3.0


def error_estimate(f_h: np.ndarray, f_h2: np.ndarray, f_h4: np.ndarray) -> np.ndarray:
    """Relative difference of the two Richardson extrapolants R(h, h/2) and
    R(h/2, h/4), pointwise in time."""
    r1 = extrapolate(f_h, f_h2)
    r2 = extrapolate(f_h2, f_h4)
    return np.abs(r1 - r2) / np.maximum(np.abs(r2), np.finfo(float).tiny)


def convergence_order(f_h, f_h2, f_h4) -> float:
    """Observed order from three levels: log2(|f_h - f_h2| / |f_h2 - f_h4|)
    (norms over the samples)."""
    a = np.linalg.norm(np.asarray(f_h) - np.asarray(f_h2))
    b = np.linalg.norm(np.asarray(f_h2) - np.asarray(f_h4))
    return float(np.log2(a / b))


@dataclass
class Level:
    nr: int
    nth: int
    dt: float
    every: int
    steps: int


def ladder(nr: int, nth: int, dt: float, every: int, steps: int, levels: int = 3):
    """Resolution ladder from the coarsest level: h, dtheta and dt halve per
    level, the r* nodes nest, all levels sample at the same times."""
    out = []
    for k in range(levels):
        f = 2 ** k
        out.append(Level(nr=f * (nr - 1) + 1, nth=f * nth, dt=dt / f, every=f * every, steps=f * steps))
    return out


def run_ladder(levels, a, s, m, rstar_min, rstar_max, rstar_ext, init=None, source=None, stream=None):
    """Evolve every level on the GPU in one batch; returns [(t, phi_rows)] per
    level.  init(level) -> (phi, pi) host arrays or None for zero data;
    source: dict for Solver.set_source or None."""
    from . import teuk as T
    solvers = []
    B = T.Batch(stream=stream)
    try:
        for lv in levels:
            g = T.Solver(lv.nr, lv.nth, rstar_min, rstar_max, lv.dt, a, s, m)
            if init is not None:
                phi, pi = init(lv)
                g.set_initial(phi, pi)
            if source:
                g.set_source(**source)
            g.set_extraction(rstar_ext, lv.every, capacity=lv.steps // lv.every + 1)
            solvers.append(g)
            B.add(g, lv.steps)
        B.step(max(lv.steps for lv in levels))
        B.sync()
        return [g.extract() for g in solvers]
    finally:
        B.close()                   # release the handles before destroying them
        for g in solvers:
            g.close()
