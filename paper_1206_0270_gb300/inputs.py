"""Seeded synthetic inputs and workload definitions.

This module holds no arithmetic of the solver itself: it only draws initial
data, parameter sets and random fields, so that the CUDA path and the CPU
oracle can be driven with identical inputs.  Grid positions follow the
solver's grid convention (r*_i = r*_min + i h with h = (r*_max - r*_min)/(nr-1),
theta_j = (j + 1/2) pi / nth), which is part of the input recipe.

Arrays are numpy complex128 of shape (nr, nth), theta fastest.
"""
from __future__ import annotations

import numpy as np

# Workloads named by what they are.  Coordinates in units of the black-hole
# mass M.  c_r / c_theta are the Courant factors of the time-step rule
# dt = min(c_r h / max b, c_theta / omega_max) and eps the strength of the
# angular Kreiss-Oliger dissipation; c_theta = 0.8 needs eps = 1 (the bare
# scheme, eps = 0, needs c_theta = 0.1).
STEP_RULE = dict(c_r=0.5, c_theta=0.8, eps=1.0)

WORKLOADS = {
    # Schwarzschild, no source, Gaussian pulse (width 5M) with the lowest
    # spin-weighted angular profile, 2000 steps.
    "schwarzschild_s-2_m2_1024x64": dict(
        a=0.0, s=-2, m=2, nr=1024, nth=64, rstar_min=-100.0, rstar_max=300.0,
        **STEP_RULE, steps=2000,
        pulse=dict(center=50.0, width=5.0), source=None,
        extraction=dict(rstar=100.0, every=10)),
    # Kerr a = 0.9M, circular equatorial orbit r0 = 10M, Gaussian source width
    # 0.05M, zero initial data, 1e5 steps (t = 1170M), waveform at r* = 500M
    # every 10 steps.  The outer boundary at r* = 1000M stays out of causal
    # contact with the observer for the whole run (a wave reflected there
    # would reach r* = 500M only after t = 1490M).
    "kerr_a0.9_s-2_m2_8192x128_r0_10": dict(
        a=0.9, s=-2, m=2, nr=8192, nth=128, rstar_min=-100.0, rstar_max=1000.0,
        **STEP_RULE, steps=100000,
        pulse=None, source=dict(r0=10.0, sigma=0.05, amplitude=1.0, prograde=True),
        extraction=dict(rstar=500.0, every=10)),
    # Large single mode whose state (2 x 537 MB) is far larger than L2.
    "kerr_a0.9_s-2_m2_32768x512_r0_10": dict(
        a=0.9, s=-2, m=2, nr=32768, nth=512, rstar_min=-100.0, rstar_max=1000.0,
        **STEP_RULE, steps=2000,
        pulse=None, source=dict(r0=10.0, sigma=0.05, amplitude=1.0, prograde=True),
        extraction=dict(rstar=500.0, every=10)),
}


# Batched workloads.  One Kerr a = 0.7M orbit at r0 = 8M, modes m = 1..8 with
# theta resolution growing with m, 4096 r* points each, 5e4 steps.
MODE_BATCH = dict(
    a=0.7, s=-2, r0=8.0, sigma=0.05, nr=4096, rstar_min=-100.0, rstar_max=600.0, steps=50000,
    modes=[(1, 32), (2, 32), (3, 64), (4, 64), (5, 128), (6, 128), (7, 256), (8, 256)],
    extraction=dict(rstar=500.0, every=10), **STEP_RULE)


def rstar_grid(nr: int, rstar_min: float, rstar_max: float) -> np.ndarray:
    h = (rstar_max - rstar_min) / (nr - 1)
    return rstar_min + h * np.arange(nr)


def theta_grid(nth: int) -> np.ndarray:
    return (np.arange(nth) + 0.5) * (np.pi / nth)


def angular_profile(theta: np.ndarray, s: int, m: int) -> np.ndarray:
    """sin(theta/2)^|m+s| cos(theta/2)^|m-s|: the lowest spin-weighted
    spherical harmonic's theta dependence (l = max(|m|, |s|)), used as initial
    angular shape.  For s = -2, m = 2 this is ((1 + cos theta)/2)^2."""
    return np.sin(theta / 2) ** abs(m + s) * np.cos(theta / 2) ** abs(m - s)


def gaussian_pulse(nr, nth, rstar_min, rstar_max, s, m, center, width, seed=None):
    """Phi(t=0) = e^{i alpha} exp(-(r* - c)^2 / (2 width^2)) Y(theta).

    With a seed, alpha ~ U[0, 2 pi) and c is jittered by U[-1, 1] M; with
    seed=None the pulse is real and centred exactly at `center`."""
    c, alpha = float(center), 0.0
    if seed is not None:
        rng = np.random.default_rng(seed)
        alpha = rng.uniform(0.0, 2 * np.pi)
        c += rng.uniform(-1.0, 1.0)
    rs = rstar_grid(nr, rstar_min, rstar_max)
    th = theta_grid(nth)
    radial = np.exp(-((rs - c) ** 2) / (2.0 * width * width))
    out = radial[:, None] * angular_profile(th, s, m)[None, :]
    return (out * np.exp(1j * alpha)).astype(np.complex128)


def random_fields(nr, nth, seed, smooth=True):
    """Random complex (Phi, Pi).  With smooth=True the fields are a sum of a
    few random low-order modes in r* and theta (well resolved on the grid);
    otherwise i.i.d. normal values."""
    rng = np.random.default_rng(seed)
    if not smooth:
        z = rng.standard_normal((2, nr, nth)) + 1j * rng.standard_normal((2, nr, nth))
        return z[0].copy(), z[1].copy()
    x = np.linspace(0.0, 1.0, nr)[:, None]
    th = theta_grid(nth)[None, :]
    out = []
    for _ in range(2):
        f = np.zeros((nr, nth), dtype=np.complex128)
        for _k in range(4):
            kr = rng.uniform(1.0, 6.0)
            kt = rng.integers(0, 4)
            amp = rng.standard_normal() + 1j * rng.standard_normal()
            ph = rng.uniform(0, 2 * np.pi)
            f += amp * np.sin(np.pi * kr * x + ph) * np.cos(kt * th)
        out.append(f)
    return out[0], out[1]


def template_bank(n_jobs: int, seed: int = 20120603):
    """Parameter draws of a template bank: a ~ U[0, 0.95], r0 ~ U[6, 20] M,
    m ~ U{1..4}, nr ~ U{2048, 4096, 8192, 16384}, nth ~ U{64, 128, 256},
    steps ~ logU[1e4, 1e5]."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n_jobs):
        jobs.append(dict(
            a=float(rng.uniform(0.0, 0.95)), r0=float(rng.uniform(6.0, 20.0)),
            m=int(rng.integers(1, 5)), s=-2,
            nr=int(rng.choice([2048, 4096, 8192, 16384])), nth=int(rng.choice([64, 128, 256])),
            steps=int(round(10 ** rng.uniform(4.0, 5.0)))))
    return jobs


def small_bank(n_jobs: int = 128, seed: int = 20120605):
    """A bank of small evolutions (the regime in which a single job cannot
    fill the GPU): a ~ U[0, 0.95], r0 ~ U[6, 20] M, m ~ U{1..4}, s = -2,
    nr ~ U{256, 512}, nth ~ U{16, 32}, steps ~ logU[1e4, 4e4]."""
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(n_jobs):
        jobs.append(dict(a=float(rng.uniform(0.0, 0.95)), r0=float(rng.uniform(6.0, 20.0)), m=int(rng.integers(1, 5)),
                         s=-2, nr=int(rng.choice([256, 512])), nth=int(rng.choice([16, 32])),
                         steps=int(round(10 ** rng.uniform(4.0, np.log10(4e4))))))
    return jobs


def serving_requests(n: int, rate: float, seed: int = 20120604, step_range=(1e3, 1e4),
                     grids=((2048, 64), (4096, 64), (4096, 128), (8192, 128), (16384, 256), (32768, 512)),
                     grid_weights=(0.25, 0.25, 0.2, 0.2, 0.08, 0.02), long_tail: int = 0,
                     long_steps=(1e5, 1e6), long_grids=((8192, 128), (16384, 256), (32768, 512)),
                     long_weights=(0.5, 0.3, 0.2)):
    """A Poisson stream of waveform requests: arrival gaps ~ Exp(rate), a ~
    U[0, 0.95], r0 ~ U[6, 20] M, m ~ U{1..4}, s = -2, grid drawn from `grids`
    with `grid_weights`, steps ~ logU[step_range].  With long_tail = k, the
    first k of the n requests (the earliest arrivals, so that they are on the
    GPU while the short ones come in) are long jobs instead: steps ~
    logU[long_steps], grid from `long_grids` with `long_weights` (None: the
    long jobs take the grids in turn)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    w = np.asarray(grid_weights, float)
    w = w / w.sum()
    lw = None if long_weights is None else np.asarray(long_weights, float) / np.sum(long_weights)
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        long_job = k < long_tail
        if long_job:
            nr, nth = long_grids[k % len(long_grids) if lw is None else rng.choice(len(long_grids), p=lw)]
            lo, hi = long_steps
        else:
            nr, nth = grids[rng.choice(len(grids), p=w)]
            lo, hi = step_range
        out.append(dict(arrival=t, a=float(rng.uniform(0.0, 0.95)), r0=float(rng.uniform(6.0, 20.0)),
                        m=int(rng.integers(1, 5)), s=-2, nr=int(nr), nth=int(nth),
                        steps=int(round(10 ** rng.uniform(np.log10(lo), np.log10(hi)))), long=long_job))
    return out
