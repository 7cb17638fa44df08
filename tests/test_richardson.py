"""Richardson extrapolation and the spin-weighted harmonic projection
(post-processing of extracted waveforms): closed forms, orthonormality,
exactness of the extrapolant, and second-order convergence of the oracle
over a resolution ladder."""
import math

import numpy as np
import pytest

from paper_1206_0270_gb300 import inputs, richardson as R


def test_swsh_closed_forms():
    th = np.linspace(0.01, math.pi - 0.01, 57)
    # s = -2, l = m = 2: sqrt(5 / (64 pi)) (1 + cos theta)^2
    np.testing.assert_allclose(R.swsh_theta(-2, 2, 2, th), math.sqrt(5 / (64 * math.pi)) * (1 + np.cos(th)) ** 2,
                               rtol=1e-13, atol=1e-15)
    # s = 0, m = 0: sqrt((2l+1)/(4 pi)) P_l(cos theta)
    for l in range(5):
        Pl = np.polynomial.legendre.Legendre.basis(l)(np.cos(th))
        np.testing.assert_allclose(R.swsh_theta(0, l, 0, th), math.sqrt((2 * l + 1) / (4 * math.pi)) * Pl,
                                   rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("s,m", [(-2, 2), (-2, -1), (2, 3), (0, 1)])
def test_swsh_orthonormal(s, m):
    x, w = np.polynomial.legendre.leggauss(80)          # x = cos theta
    th = np.arccos(x)
    ls = range(max(abs(s), abs(m)), max(abs(s), abs(m)) + 5)
    Y = np.array([R.swsh_theta(s, l, m, th) for l in ls])
    G = 2 * math.pi * (Y * w) @ Y.T
    np.testing.assert_allclose(G, np.eye(len(Y)), atol=1e-12)


def test_projection_of_a_harmonic_row():
    nth = 256
    th = inputs.theta_grid(nth)
    rows = np.array([R.swsh_theta(-2, 3, 2, th), 2j * R.swsh_theta(-2, 2, 2, th)])
    np.testing.assert_allclose(R.project(rows, -2, 3, 2), [1.0, 0.0], atol=1e-4)
    np.testing.assert_allclose(R.project(rows, -2, 2, 2), [0.0, 2j], atol=1e-4)


def test_extrapolant_removes_the_second_order_term():
    a, b, c = 1.25 - 0.5j, 3.0 + 1j, -7.0
    f = lambda h: a + b * h ** 2 + c * h ** 4
    h = 0.1
    assert abs(R.extrapolate(f(h), f(h / 2)) - (a - c * h ** 4 / 4)) < 1e-14
    e = R.error_estimate(f(h), f(h / 2), f(h / 4))
    assert e < 1e-3 and e > 0
    g = lambda h: a + b * h ** 2
    assert R.convergence_order(g(h), g(h / 2), g(h / 4)) == pytest.approx(2.0, abs=1e-9)


def test_ladder_levels_nest_and_share_sample_times():
    lv = R.ladder(101, 8, 0.04, 5, 300, levels=3)
    assert [(l.nr, l.nth) for l in lv] == [(101, 8), (201, 16), (401, 32)]
    for l in lv:
        assert l.steps * l.dt == pytest.approx(300 * 0.04)
        assert l.every * l.dt == pytest.approx(5 * 0.04)


def test_oracle_ladder_converges_at_second_order():
    from oracle import oracle as O
    a, s, m = 0.5, -2, 2
    rmin, rmax = -40.0, 60.0
    base_nr, base_nth = 201, 16
    dt_f = O.stable_dt(4 * (base_nr - 1) + 1, 4 * base_nth, rmin, rmax, a, s, m)
    lv = R.ladder(base_nr, base_nth, 4 * dt_f, every=2, steps=int(12.0 / (4 * dt_f)) // 2 * 2, levels=3)
    series = []
    for l in lv:
        S = O.Solver(l.nr, l.nth, rmin, rmax, l.dt, a, s, m)
        S.set_initial(inputs.gaussian_pulse(l.nr, l.nth, rmin, rmax, s, m, center=15.0, width=4.0), None)
        S.set_extraction(10.0, l.every)
        S.step(l.steps)
        t, rows = S.samples()
        series.append((t, R.project(rows, s, 2, m)))
    for t, _ in series[1:]:
        np.testing.assert_allclose(t, series[0][0], rtol=1e-12)
    f = [x for _, x in series]
    sel = slice(len(f[0]) // 2, None)
    order = R.convergence_order(f[0][sel], f[1][sel], f[2][sel])
    assert 1.6 < order < 2.4, order
    # the extrapolants agree far better than the raw levels
    raw = np.abs(f[1][sel] - f[2][sel]).max()
    ext = np.abs(R.extrapolate(f[0][sel], f[1][sel]) - R.extrapolate(f[1][sel], f[2][sel])).max()
    assert ext < 0.3 * raw


@pytest.mark.gpu
def test_gpu_ladder_matches_oracle_and_extrapolates():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1206_0270_gb300 import build
    build.build()
    a, s, m = 0.7, -2, 2
    rmin, rmax = -40.0, 60.0
    base_nr, base_nth = 201, 16
    dt_f = O.stable_dt(4 * (base_nr - 1) + 1, 4 * base_nth, rmin, rmax, a, s, m)
    lv = R.ladder(base_nr, base_nth, 4 * dt_f, every=2, steps=int(12.0 / (4 * dt_f)) // 2 * 2, levels=3)
    src = dict(r0=6.0, sigma=2.0)
    init = lambda l: (inputs.gaussian_pulse(l.nr, l.nth, rmin, rmax, s, m, center=15.0, width=4.0), None)
    out = R.run_ladder(lv, a, s, m, rmin, rmax, 10.0, init=init, source=src)
    f_gpu, f_ora = [], []
    for l, (t, rows) in zip(lv, out):
        S = O.Solver(l.nr, l.nth, rmin, rmax, l.dt, a, s, m)
        S.set_initial(*init(l))
        S.set_source(**src)
        S.set_extraction(10.0, l.every)
        S.step(l.steps)
        to, ro = S.samples()
        np.testing.assert_array_equal(t, to)
        assert np.abs(rows - ro).max() <= 1e-10 * np.abs(ro).max()
        f_gpu.append(R.project(rows, s, 2, m))
        f_ora.append(R.project(ro, s, 2, m))
    e_gpu = R.error_estimate(*f_gpu)
    e_ora = R.error_estimate(*f_ora)
    sel = slice(len(e_gpu) // 2, None)
    np.testing.assert_allclose(e_gpu[sel], e_ora[sel], rtol=1e-6)
    assert 1.6 < R.convergence_order(*(f[sel] for f in f_gpu)) < 2.4
