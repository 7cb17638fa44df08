"""Kerr quasinormal frequencies by Leaver's continued-fraction method, and a
multi-channel matrix-pencil fit of damped exponentials.  Test helpers only:
they share nothing with the oracle or the CUDA path, and serve as the
independent reference against which the oracle's Kerr evolution is pinned.

Conventions: perturbations go as e^{-i omega t} e^{i m phi} (the m-mode
ansatz of Eq. 2 with Boyer-Lindquist phi), units of the black-hole mass M.

Method: E. W. Leaver, Proc. R. Soc. Lond. A 402, 285 (1985).  The radial
Teukolsky function is expanded about the horizon in a series whose
coefficients obey a three-term recurrence; the quasinormal condition is that
the minimal solution of the recurrence starts the series, which is the
vanishing of a continued fraction.  Leaver works in units 2M = 1; the
conversion is omega_L = 2 M omega, a_L = a / (2 M).  The angular separation
constant A (the eigenvalue of the spin-weighted spheroidal equation,
Teukolsky 1973 Eq. 4.10, with A = (l - s)(l + s + 1) at a omega = 0) is found
in two independent ways: Leaver's angular continued fraction, and a Galerkin
solve in the spin-weighted spherical harmonic basis, here built from Jacobi
polynomials.
"""
import math

import numpy as np
from scipy.special import eval_jacobi


# ---------------------------------------------------------------------------
# Angular problem
# ---------------------------------------------------------------------------

def angular_continued_fraction(A, c, s, m, depth=300):
    """Leaver's angular condition for the spheroidal function
    S = e^{c u} (1 + u)^{k1} (1 - u)^{k2} sum_n a_n (1 + u)^n, u = cos(theta),
    k1 = |m - s| / 2, k2 = |m + s| / 2: alpha_n a_{n+1} + beta_n a_n +
    gamma_n a_{n-1} = 0 has a minimal solution with a_{-1} = 0 exactly when
    beta_0 - alpha_0 gamma_1 / (beta_1 - alpha_1 gamma_2 / (beta_2 - ...))
    vanishes.  Returns that value (zero at an eigenvalue A)."""
    k1, k2 = abs(m - s) / 2, abs(m + s) / 2
    kk = k1 + k2

    def alpha(n):
        return -2.0 * (n + 1) * (n + 2 * k1 + 1)

    def beta(n):
        return (n * (n - 1) + 2 * n * (kk + 1 - 2 * c)
                - (2 * c * (2 * k1 + s + 1) - kk * (kk + 1)) - (c * c + s * (s + 1) + A))

    def gamma(n):
        return 2 * c * (n + kk + s)

    tail = 0j
    for n in range(depth, 0, -1):
        tail = alpha(n - 1) * gamma(n) / (beta(n) - tail)
    return beta(0) - tail


def swsh_basis(s, m, lmax, x):
    """Spin-weighted spherical harmonics sY_lm(theta), l = max(|m|, |s|) ..
    lmax, up to sign, at x = cos(theta): (1 - x)^{|m+s|/2} (1 + x)^{|m-s|/2}
    P_n^{(|m+s|, |m-s|)}(x), n = l - max(|m|, |s|), normalised so that
    2 pi integral_{-1}^{1} Y^2 dx = 1."""
    al, be = abs(m + s), abs(m - s)
    l0 = max(abs(m), abs(s))
    rows = []
    for l in range(l0, lmax + 1):
        n = l - l0
        norm = (2.0 ** (al + be + 1) / (2 * n + al + be + 1)
                * math.gamma(n + al + 1) * math.gamma(n + be + 1)
                / (math.gamma(n + al + be + 1) * math.factorial(n)))
        y = (1 - x) ** (al / 2) * (1 + x) ** (be / 2) * eval_jacobi(n, al, be, x)
        rows.append(y / math.sqrt(2 * math.pi * norm))
    return np.array(rows), list(range(l0, lmax + 1))


def separation_constant(c, s, m, l, method="spectral", lmax=None):
    """A_lm(c) of the Teukolsky angular equation
      (1/sin) d/dtheta(sin dS/dtheta) + (c^2 cos^2 - 2 c s cos
          - (m + s cos)^2 / sin^2 + s + A) S = 0,
    continued from (l - s)(l + s + 1) at c = 0.
    "spectral": in the basis sY_l'm the equation reads
      diag((l' - s)(l' + s + 1)) b - <Y|c^2 cos^2 - 2 c s cos|Y> b = A b;
    "cf": secant iteration on Leaver's angular continued fraction."""
    target = (l - s) * (l + s + 1)
    if method == "spectral":
        lmax = lmax or max(l, abs(m), abs(s)) + 14
        x, w = np.polynomial.legendre.leggauss(4 * lmax + 20)
        Y, ls = swsh_basis(s, m, lmax, x)
        wY = 2 * math.pi * Y * w
        C1, C2 = wY @ (x * Y).T, wY @ (x * x * Y).T
        M = np.diag([(k - s) * (k + s + 1) for k in ls]).astype(complex) - (c * c * C2 - 2 * c * s * C1)
        ev = np.linalg.eigvals(M)
        return complex(ev[np.argmin(abs(ev - target))])
    if method == "cf":
        A0, A1 = complex(target), complex(target) + 1e-3
        f0 = angular_continued_fraction(A0, c, s, m)
        for _ in range(200):
            f1 = angular_continued_fraction(A1, c, s, m)
            if f1 == f0:
                break
            A0, A1, f0 = A1, A1 - f1 * (A1 - A0) / (f1 - f0), f1
            if abs(A1 - A0) <= 1e-14 * max(1.0, abs(A1)):
                break
        return A1
    raise ValueError(method)


# ---------------------------------------------------------------------------
# Radial problem
# ---------------------------------------------------------------------------

def radial_continued_fraction(omega, a, s, m, A, depth=1000):
    """Leaver's radial quasinormal condition (units 2M = 1 inside), for
    e^{-i omega t} e^{i m phi}: with b = sqrt(1 - 4 a_L^2) and
    q = omega_L / 2 - a_L m, the series coefficients obey
    alpha_n a_{n+1} + beta_n a_n + gamma_n a_{n-1} = 0 with
      alpha_n = n^2 + (c0 + 1) n + c0
      beta_n  = -2 n^2 + (c1 + 2) n + c3
      gamma_n = n^2 + (c2 - 3) n + c4 - c2 + 2,
    and omega is quasinormal when the continued fraction vanishes."""
    wl, al = 2.0 * omega, a / 2.0
    b = math.sqrt(1.0 - 4.0 * al * al)
    q = wl / 2 - al * m
    c0 = 1 - s - 1j * wl - 2j / b * q
    c1 = -4 + 2j * wl * (2 + b) + 4j / b * q
    c2 = s + 3 - 3j * wl - 2j / b * q
    c3 = (wl * wl * (4 + 2 * b - al * al) - 2 * al * m * wl - s - 1 + (2 + b) * 1j * wl - A
          + (4 * wl + 2j) / b * q)
    c4 = s + 1 - 2 * wl * wl - (2 * s + 3) * 1j * wl - (4 * wl + 2j) / b * q
    tail = 0j
    for n in range(depth, 0, -1):
        alpha = (n - 1) ** 2 + (c0 + 1) * (n - 1) + c0
        gamma = n * n + (c2 - 3) * n + c4 - c2 + 2
        beta = -2 * n * n + (c1 + 2) * n + c3
        tail = alpha * gamma / (beta - tail)
    return c3 - tail


def kerr_qnm(a, s, m, l, guess, angular="spectral"):
    """Fundamental-branch quasinormal frequency M omega nearest to guess, by
    a secant iteration on the radial continued fraction with A(a omega)."""
    def f(w):
        return radial_continued_fraction(w, a, s, m, separation_constant(a * w, s, m, l, angular))
    w0, w1 = complex(guess), complex(guess) * (1 + 1e-3)
    f0 = f(w0)
    for _ in range(100):
        f1 = f(w1)
        if f1 == f0:
            break
        w0, w1, f0 = w1, w1 - f1 * (w1 - w0) / (f1 - f0), f1
        if abs(w1 - w0) <= 1e-12:
            break
    return w1


# ---------------------------------------------------------------------------
# Damped-exponential fit
# ---------------------------------------------------------------------------

def matrix_pencil(t, Y, K):
    """Fit Y[:, c] = sum_k C_kc e^{-i w_k t} (equally spaced t, frequencies
    shared by all channels c) by the matrix pencil method (Hua & Sarkar,
    IEEE Trans. ASSP 38, 814, 1990): the channels' Hankel matrices are
    stacked, the K leading right singular vectors span the signal space, and
    the shift between their first and last rows has eigenvalues e^{-i w dt}.
    Returns (w, amplitude over channels) sorted by decreasing amplitude."""
    Y = np.asarray(Y, dtype=complex)
    if Y.ndim == 1:
        Y = Y[:, None]
    N = Y.shape[0]
    L = N // 3
    H = np.concatenate([np.array([Y[i:i + L + 1, c] for i in range(N - L)]) for c in range(Y.shape[1])])
    _, _, Vh = np.linalg.svd(H, full_matrices=False)
    V = Vh[:K].T
    z = np.linalg.eigvals(np.linalg.pinv(V[:-1]) @ V[1:])
    w = 1j * np.log(z) / (t[1] - t[0])
    C = np.linalg.lstsq(np.exp(-1j * np.outer(t - t[0], w)), Y, rcond=None)[0]
    amp = np.sqrt((abs(C) ** 2).sum(axis=1))
    order = np.argsort(-amp)
    return w[order], amp[order]
