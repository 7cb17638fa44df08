"""The seeded input generators against the recipes their docstrings state:
parameter ranges, the presence of every listed grid, Poisson arrival gaps and
grid weights, the long-tail layout, determinism under a seed, and the
causality claim of the Kerr workload's outer boundary.  CPU only."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_1206_0270_gb300 import inputs as I  # noqa: E402


def _log_uniform_ok(steps, lo, hi):
    # round(10^U[log lo, log hi]) stays in [lo, hi]; a log-uniform draw puts
    # about half of the mass below the geometric mean
    steps = np.asarray(steps, float)
    assert steps.min() >= lo and steps.max() <= hi
    below = np.mean(steps < math.sqrt(lo * hi))
    assert 0.35 < below < 0.65, below


def test_template_bank_recipe():
    jobs = I.template_bank(256)
    assert len(jobs) == 256
    a = np.array([j["a"] for j in jobs])
    r0 = np.array([j["r0"] for j in jobs])
    assert a.min() >= 0.0 and a.max() <= 0.95
    assert r0.min() >= 6.0 and r0.max() <= 20.0
    assert {j["m"] for j in jobs} == {1, 2, 3, 4}
    assert {j["s"] for j in jobs} == {-2}
    assert {j["nr"] for j in jobs} == {2048, 4096, 8192, 16384}
    assert {j["nth"] for j in jobs} == {64, 128, 256}
    _log_uniform_ok([j["steps"] for j in jobs], 1e4, 1e5)
    assert I.template_bank(256) == jobs                      # seeded
    assert I.template_bank(256, seed=1) != jobs


def test_small_bank_recipe():
    jobs = I.small_bank()
    assert len(jobs) == 128
    assert {j["nr"] for j in jobs} == {256, 512}
    assert {j["nth"] for j in jobs} == {16, 32}
    assert {j["m"] for j in jobs} == {1, 2, 3, 4}
    assert all(0.0 <= j["a"] <= 0.95 and 6.0 <= j["r0"] <= 20.0 for j in jobs)
    _log_uniform_ok([j["steps"] for j in jobs], 1e4, 4e4)
    assert I.small_bank() == jobs


def test_serving_requests_poisson_gaps_and_grid_weights():
    n, rate = 4000, 4.0
    reqs = I.serving_requests(n, rate)
    t = np.array([r["arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # Exp(rate): mean 1/rate and standard deviation 1/rate; the sample mean of
    # n gaps is within 5 standard errors
    assert abs(gaps.mean() - 1 / rate) < 5 / (rate * math.sqrt(n))
    assert abs(gaps.std() - 1 / rate) < 0.1 / rate
    grids = ((2048, 64), (4096, 64), (4096, 128), (8192, 128), (16384, 256), (32768, 512))
    weights = np.array([0.25, 0.25, 0.2, 0.2, 0.08, 0.02])
    counts = np.array([sum((r["nr"], r["nth"]) == g for r in reqs) for g in grids])
    # binomial counts within 5 standard deviations of n w
    assert np.all(np.abs(counts - n * weights) < 5 * np.sqrt(n * weights * (1 - weights)) + 1)
    _log_uniform_ok([r["steps"] for r in reqs], 1e3, 1e4)
    assert not any(r["long"] for r in reqs)
    assert I.serving_requests(n, rate) == reqs


def test_serving_requests_long_tail_layout():
    reqs = I.serving_requests(64, 4.0, long_tail=3, long_steps=(1e5, 1e5),
                              long_grids=((32768, 512), (8192, 128)), long_weights=None)
    assert [r["long"] for r in reqs[:3]] == [True, True, True]
    assert not any(r["long"] for r in reqs[3:])
    # without weights the long jobs take the grids in turn
    assert [(r["nr"], r["nth"]) for r in reqs[:3]] == [(32768, 512), (8192, 128), (32768, 512)]
    assert all(r["steps"] == 100000 for r in reqs[:3])
    assert all(1e3 <= r["steps"] <= 1e4 for r in reqs[3:])
    t = [r["arrival"] for r in reqs]
    assert t == sorted(t)


def test_angular_profile_and_pulse():
    th = I.theta_grid(64)
    assert np.allclose(np.diff(th), np.pi / 64) and th[0] == pytest.approx(np.pi / 128)
    # s = -2, m = 2: ((1 + cos theta)/2)^2, the lowest spin-weighted harmonic's shape
    # (1 + cos theta) cancels next to theta = pi: relative agreement to ~1e-12 there
    assert np.allclose(I.angular_profile(th, -2, 2), ((1 + np.cos(th)) / 2) ** 2, rtol=1e-10, atol=1e-17)
    p = I.gaussian_pulse(1024, 64, -100.0, 300.0, -2, 2, center=50.0, width=5.0)
    assert p.shape == (1024, 64) and p.dtype == np.complex128
    assert np.all(p.imag == 0)
    rs = I.rstar_grid(1024, -100.0, 300.0)
    assert rs[0] == -100.0 and rs[-1] == pytest.approx(300.0, abs=1e-12)
    i_peak = int(np.argmax(np.abs(p[:, 32])))
    assert abs(rs[i_peak] - 50.0) <= (rs[1] - rs[0]) / 2 + 1e-12
    # a seed rotates the phase and jitters the centre by at most 1 M
    q = I.gaussian_pulse(1024, 64, -100.0, 300.0, -2, 2, center=50.0, width=5.0, seed=7)
    ratio = q[np.abs(p) > 1e-3] / np.abs(q[np.abs(p) > 1e-3])
    assert np.allclose(ratio, ratio[0])                       # one global phase
    assert abs(rs[int(np.argmax(np.abs(q[:, 32])))] - 50.0) <= 1.0 + (rs[1] - rs[0])


def test_random_fields_seeded_and_smooth():
    a1, b1 = I.random_fields(512, 32, seed=3)
    a2, b2 = I.random_fields(512, 32, seed=3)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    # at most 6 half-waves over the r* range and cos(k theta), k <= 3: second
    # differences are small against the fields
    d2 = np.abs(a1[2:] - 2 * a1[1:-1] + a1[:-2]).max()
    assert d2 < 1e-3 * np.abs(a1).max()
    z1, _ = I.random_fields(64, 16, seed=3, smooth=False)
    assert abs(z1.real.std() - 1.0) < 0.1


def _tortoise(r, a):
    # r* = r + 2 r+/(r+ - r-) ln((r - r+)/2) - 2 r-/(r+ - r-) ln((r - r-)/2), M = 1
    rp, rm = 1 + math.sqrt(1 - a * a), 1 - math.sqrt(1 - a * a)
    return r + 2 * rp / (rp - rm) * math.log((r - rp) / 2) - 2 * rm / (rp - rm) * math.log((r - rm) / 2)


def test_kerr_workload_outer_boundary_stays_out_of_causal_contact():
    oracle = pytest.importorskip("oracle.oracle")
    w = I.WORKLOADS["kerr_a0.9_s-2_m2_8192x128_r0_10"]
    dt = oracle.stable_dt(w["nr"], w["nth"], w["rstar_min"], w["rstar_max"], w["a"], w["s"], w["m"],
                          w["c_r"], w["c_theta"])
    t_end = w["steps"] * dt
    assert t_end == pytest.approx(1170.0, rel=0.01)
    # signals move in r* at the radial characteristic speed b = (r^2 + a^2) /
    # Sigma_hat, which exceeds 1 by under a^2 / (2 r^2) (less than 0.1 M over
    # the path): from the source out to the boundary and back to the observer
    r_src = _tortoise(w["source"]["r0"], w["a"])
    t_reflect = (w["rstar_max"] - r_src) + (w["rstar_max"] - w["extraction"]["rstar"])
    assert t_reflect == pytest.approx(1490.0, abs=10.0)
    assert t_end < t_reflect


def test_mode_batch_and_workload_table():
    # the mode batch: one a = 0.7, r0 = 8 orbit, m = 1..8 on 4096 r* points with
    # the theta resolution doubling every two modes, 5e4 steps
    mb = I.MODE_BATCH
    assert (mb["a"], mb["r0"], mb["nr"], mb["steps"]) == (0.7, 8.0, 4096, 50000)
    assert [m for m, _ in mb["modes"]] == list(range(1, 9))
    assert [n for _, n in mb["modes"]] == [32, 32, 64, 64, 128, 128, 256, 256]
    # every workload uses the dissipative step rule and keeps its observer
    # inside the grid
    for name, w in I.WORKLOADS.items():
        assert (w["c_r"], w["c_theta"], w["eps"]) == (0.5, 0.8, 1.0), name
        assert w["rstar_min"] < w["extraction"]["rstar"] < w["rstar_max"], name
        assert name.endswith("%dx%d" % (w["nr"], w["nth"])) or "%dx%d_" % (w["nr"], w["nth"]) in name, name
