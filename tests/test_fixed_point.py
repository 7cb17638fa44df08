"""The fixed-point sums of the Pi rows (teuk_fixed_dot): the host build of
the arithmetic the step kernels run, against exact rational arithmetic.

Bound (stated in include/teuk.h): |out - exact| <= n 2^-57 max_k |c_k x_k|
+ 2^-53 |exact| wherever ok; ok is false only for non-finite inputs, results
below 2^-823, or overflow.  The device build is compared with the host build
bit for bit in the GPU test at the end."""
from fractions import Fraction

import numpy as np
import pytest

T = pytest.importorskip("paper_1206_0270_gb300.teuk", reason="libteuk.so not built")


def exact_sum(c, x, flip):
    return sum((-1 if f else 1) * Fraction(float(a)) * Fraction(float(b)) for a, b, f in zip(c, x, flip))


def check_bound(c, x, flip, out, ok):
    n = c.shape[1]
    for i in range(c.shape[0]):
        if not ok[i]:
            continue
        ex = exact_sum(c[i], x[i], flip[i])
        mx = max(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(c[i], x[i]))
        bound = n * Fraction(2) ** -57 * mx + abs(ex) * Fraction(2) ** -53
        assert abs(Fraction(float(out[i])) - ex) <= bound, (i, c[i], x[i], flip[i], out[i], float(ex))


def random_case(rng, count, n, kind):
    c = rng.standard_normal((count, n)) * 10.0 ** rng.integers(-3, 3, (count, n))
    x = rng.standard_normal((count, n)) * 10.0 ** rng.integers(-6, 6, (count, n))
    flip = rng.integers(0, 2, (count, n)).astype(np.uint32)
    if kind == "cancel" and n > 1:
        # last term nearly cancels the others: the sum keeps only a few bits
        sg = np.where(flip == 1, -1.0, 1.0)
        part = np.sum(sg[:, :-1] * c[:, :-1] * x[:, :-1], axis=1)
        x[:, -1] = -part / (sg[:, -1] * c[:, -1]) * (1 + 1e-12 * rng.standard_normal(count))
    elif kind == "zeros":
        x[rng.random((count, n)) < 0.4] = 0.0
        c[rng.random((count, n)) < 0.2] = 0.0
    elif kind == "wide":
        x *= 10.0 ** rng.integers(-250, 250, (count, 1))
        x *= 10.0 ** rng.integers(-30, 30, (count, n))
    return c, x, flip


@pytest.mark.parametrize("n", [1, 2, 6, 7, 9, 10, 16])
@pytest.mark.parametrize("kind", ["plain", "cancel", "zeros", "wide"])
def test_error_bound_against_exact_arithmetic(n, kind):
    rng = np.random.default_rng(1000 * n + len(kind))
    c, x, flip = random_case(rng, 400, n, kind)
    out, ok = T.fixed_dot(c, x, flip)
    assert ok.mean() > 0.9
    check_bound(c, x, flip, out, ok)


def test_subnormal_and_tiny_inputs():
    rng = np.random.default_rng(7)
    c = rng.standard_normal((300, 9))
    x = rng.standard_normal((300, 9))
    x[:100, :3] = 1e-310                      # subnormal fields beside normal ones
    x[100:200] *= 1e-300                      # tiny results: FP64 fallback
    x[200:, 4] = 5e-324
    out, ok = T.fixed_dot(c, x)
    assert ok[:100].all() and not ok[100:200].any()
    check_bound(c, x, np.zeros_like(x, dtype=np.uint32), out, ok)


def test_exact_results_ties_and_zero():
    # exactly representable sums come out exactly
    out, ok = T.fixed_dot(np.array([[3.0, 0.25, -7.0]]), np.array([[5.0, 8.0, 0.5]]))
    assert ok[0] and out[0] == 15.0 + 2.0 - 3.5
    # ties go to even: 1 + 2^-53 -> 1, 1 + 3 2^-53 -> 1 + 2^-51
    out, ok = T.fixed_dot(np.array([[1.0, 2.0 ** -53], [1.0, 3 * 2.0 ** -53]]), np.ones((2, 2)))
    assert ok.all() and out[0] == 1.0 and out[1] == 1.0 + 2.0 ** -51
    # x - x = +0, all-zero sums are +0
    out, ok = T.fixed_dot(np.array([[0.1, 0.1], [0.0, 0.0]]), np.array([[3.0, 3.0], [1.0, -2.0]]),
                          np.array([[0, 1], [0, 0]]))
    assert ok.all() and np.all(out == 0.0) and not np.signbit(out).any()
    # a single product: the truncated low 47 bits of the 106-bit product do
    # not reach the sticky bit, so a window that ends on an exact tie rounds
    # to even where the exact product would round up (within the bound:
    # 2^-57 + half an ulp); otherwise it is the correctly rounded product
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(4000), rng.standard_normal(4000)
    out, ok = T.fixed_dot(a[:, None], b[:, None])
    assert ok.all() and np.mean(out == a * b) > 0.98
    assert np.all(np.abs(out - a * b) <= np.spacing(np.abs(a * b)))


def test_order_and_zero_terms_do_not_change_bits():
    rng = np.random.default_rng(11)
    c, x, flip = random_case(rng, 300, 9, "plain")
    out, ok = T.fixed_dot(c, x, flip)
    perm = rng.permutation(9)
    out_p, ok_p = T.fixed_dot(c[:, perm], x[:, perm], flip[:, perm])
    assert np.array_equal(ok, ok_p) and np.array_equal(out[ok], out_p[ok])
    # interleave zero-coefficient terms with large fields (as the complex path
    # does where the imaginary coefficient parts vanish)
    cz = np.concatenate([c, np.zeros((300, 4))], axis=1)
    xz = np.concatenate([x, 1e200 * rng.standard_normal((300, 4))], axis=1)
    fz = np.concatenate([flip, np.ones((300, 4), np.uint32)], axis=1)
    out_z, ok_z = T.fixed_dot(cz, xz, fz)
    assert np.array_equal(ok, ok_z) and np.array_equal(out[ok], out_z[ok])


def test_doubling_the_fields_doubles_the_sum_exactly():
    rng = np.random.default_rng(5)
    c, x, flip = random_case(rng, 300, 10, "cancel")
    out, ok = T.fixed_dot(c, x, flip)
    out2, ok2 = T.fixed_dot(c, 2.0 * x, flip)
    both = ok & ok2
    assert both.mean() > 0.9 and np.array_equal(out2[both], 2.0 * out[both])


def test_fallback_conditions():
    c = np.ones((4, 3))
    x = np.array([[np.inf, 1.0, 1.0], [np.nan, 1.0, 1.0], [1e308, 1e308, 1e308], [1.0, 2.0, 3.0]])
    c[2] = 10.0                              # 3e309 overflows
    out, ok = T.fixed_dot(c, x)
    assert list(ok) == [False, False, False, True] and out[3] == 6.0
    with pytest.raises(T.TeukError):
        T.fixed_dot(np.ones((2, 17)), np.ones((2, 17)))


def test_bound_and_fallbacks_for_arbitrary_fp64_operands():
    """Property test over arbitrary finite FP64 operands (any exponent,
    subnormals and signed zeros included): wherever the sum reports success
    it meets the bound; it falls back only where the exact sum lies below
    2^-820 or above 2^1020 (the tiny-result and overflow rules)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    finite = st.floats(allow_nan=False, allow_infinity=False, width=64)
    # coefficients as the kernels see them: normal numbers or exact zeros
    coef = st.one_of(st.just(0.0), st.floats(min_value=2.0 ** -60, max_value=2.0 ** 60).map(float),
                     st.floats(min_value=-2.0 ** 60, max_value=-2.0 ** -60).map(float))

    @hyp.settings(max_examples=400, deadline=None, derandomize=True)
    @hyp.given(st.integers(1, 16).flatmap(lambda n: st.tuples(
        st.lists(coef, min_size=n, max_size=n), st.lists(finite, min_size=n, max_size=n),
        st.lists(st.integers(0, 1), min_size=n, max_size=n))))
    def check(case):
        c, x, f = (np.array([v], dtype=t) for v, t in zip(case, (np.float64, np.float64, np.uint32)))
        out, ok = T.fixed_dot(c, x, f)
        ex = exact_sum(c[0], x[0], f[0])
        if ok[0]:
            check_bound(c, x, f, out, ok)
        else:
            assert abs(ex) < Fraction(2) ** -820 or abs(ex) > Fraction(2) ** 1020, (case, float(ex))

    check()


@pytest.mark.gpu
def test_device_build_equals_host_build():
    rng = np.random.default_rng(2026)
    for n in (6, 7, 9, 10, 16):
        for kind in ("plain", "cancel", "zeros", "wide"):
            c, x, flip = random_case(rng, 20000, n, kind)
            oh, kh = T.fixed_dot(c, x, flip, device=False)
            od, kd = T.fixed_dot(c, x, flip, device=True)
            assert np.array_equal(kh, kd)
            assert np.array_equal(oh[kh].view(np.uint64), od[kd].view(np.uint64))


# ---------------------------------------------------------------------------
# The exact sixth difference of the angular dissipation (teuk_fixed_d6)
# ---------------------------------------------------------------------------

D6_WEIGHTS = (-1, 6, -15, 20, -15, 6, -1)


def d6_model(u):
    """The arithmetic stated in include/teuk.h, written out with Python
    integers: prepare, align to the largest exponent (floor), weighted exact
    sum, one rounding to nearest (CPython's int/int division is correctly
    rounded, subnormals included)."""
    prep = []
    for x in u:
        bits = int(np.float64(x).view(np.uint64))
        eraw = (bits >> 52) & 0x7FF
        m = (bits & ((1 << 52) - 1)) | ((1 << 52) if eraw else 0)
        v = m << 4
        prep.append((-v if bits >> 63 else v, max(eraw, 1) if eraw != 0x7FF else 2047))
    F = max(e for _, e in prep)
    if F >= 2047:
        return float("nan")
    D = sum(wt * (v >> (F - e)) for wt, (v, e) in zip(D6_WEIGHTS, prep))
    k = F - 1079
    return D * 2.0 ** k if D == 0 else (Fraction(D) * Fraction(2) ** k).__float__()


def d6_exact(u):
    return sum(wt * Fraction(float(x)) for wt, x in zip(D6_WEIGHTS, u))


def d6_cases(rng, count):
    j = np.arange(7)
    smooth = np.sin(0.3 * (rng.integers(0, 100, (count, 1)) + j)) * 10.0 ** rng.integers(-8, 8, (count, 1))
    noisy = rng.standard_normal((count, 7)) * 10.0 ** rng.integers(-5, 5, (count, 7))
    wide = rng.standard_normal((count, 7)) * 10.0 ** rng.integers(-300, 300, (count, 7))
    zeros = rng.standard_normal((count, 7))
    zeros[rng.random((count, 7)) < 0.5] = 0.0
    return np.concatenate([smooth, noisy, wide, zeros])


def test_d6_equals_its_stated_arithmetic_bit_for_bit():
    u = d6_cases(np.random.default_rng(61), 300)
    out = T.fixed_d6(u)
    ref = np.array([d6_model(r) for r in u])
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))


def test_d6_error_bound_against_exact_arithmetic():
    u = d6_cases(np.random.default_rng(62), 300)
    out = T.fixed_d6(u)
    for r, o in zip(u, out):
        ex = d6_exact(r)
        mx = max(abs(Fraction(float(x))) for x in r)
        bound = Fraction(2) ** -50 * mx + Fraction(2) ** -53 * abs(ex) + Fraction(2) ** -1075
        assert abs(Fraction(float(o)) - ex) <= bound, (r, o, float(ex))


def test_d6_annihilates_low_degree_polynomials_and_scales_exactly():
    # D6 of samples of a polynomial of degree < 6 is exactly zero; of q^6 it is
    # -6! (D6 = -delta^6); integer samples are exact, so no truncation occurs
    q = np.arange(-3, 4, dtype=np.float64)
    rng = np.random.default_rng(63)
    polys = [np.polyval(rng.integers(-50, 50, deg + 1).astype(np.float64), q) for deg in range(6)]
    out = T.fixed_d6(np.array(polys + [q ** 6, np.full(7, 3.25), q ** 6 + 7 * q ** 3]))
    assert np.all(out[:6] == 0.0) and out[6] == -720.0 and out[7] == 0.0 and out[8] == -720.0
    # a power-of-two scale passes through exactly (normal range)
    u = d6_cases(np.random.default_rng(64), 200)[:400]
    u = u[np.all(np.abs(u) < 1e200, axis=1) & np.all((np.abs(u) > 1e-200) | (u == 0), axis=1)]
    assert np.array_equal(T.fixed_d6(4.0 * u), 4.0 * T.fixed_d6(u))


def test_d6_subnormals_and_non_finite():
    tiny = np.array([[5e-324, 0.0, 1e-310, -2e-310, 3e-321, 0.0, 7e-300],
                     [1e-320, 2e-320, 3e-320, 4e-320, 3e-320, 2e-320, 1e-320]])
    out = T.fixed_d6(tiny)
    ref = np.array([d6_model(r) for r in tiny])
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
    assert out[1] == float(d6_exact(tiny[1]))          # exact: all values share one exponent
    bad = np.array([[1.0, 2.0, np.inf, 0.0, 0.0, 0.0, 0.0], [np.nan] + [1.0] * 6])
    assert np.isnan(T.fixed_d6(bad)).all()
    with pytest.raises(ValueError):
        T.fixed_d6(np.ones((3, 6)))


@pytest.mark.gpu
def test_d6_device_build_equals_host_build():
    u = d6_cases(np.random.default_rng(65), 20000)
    oh, od = T.fixed_d6(u, device=False), T.fixed_d6(u, device=True)
    assert np.array_equal(oh.view(np.uint64), od.view(np.uint64))
