"""Pins of the oracle's finite-difference stencils and RK4 integrator.

The stencils are pinned by what fixes them mathematically: 4th-order
centred, upwind-biased and one-sided first derivatives are exact on
polynomials of degree <= 4 (and not on degree 5); the centred second
derivative is exact to degree 5; the mixed derivative (product of two
first-derivative stencils) is exact on x^a y^b, a,b <= 4; the sixth
difference of Kreiss-Oliger dissipation annihilates degree <= 5, gives
720 h^6 on x^6 and -64 on the Nyquist mode.  RK4 is pinned by its
amplification factor 1 + z + z^2/2 + z^3/6 + z^4/24 on y' = lambda y.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import oracle as O

L = O.lib()
H = 0.0137
X0 = 0.31


def _line(fn, n=9):
    xs = X0 + H * (np.arange(n) - n // 2)
    return np.ascontiguousarray([fn(x) for x in xs], dtype=np.float64)


def _centre(a):
    base = a.ctypes.data_as(ctypes.c_void_p).value + 8 * (a.size // 2)
    return ctypes.cast(base, ctypes.POINTER(ctypes.c_double))


@pytest.mark.parametrize("k", range(0, 6))
def test_first_derivative_exactness(k):
    a = _line(lambda x: x ** k)
    exact = k * X0 ** (k - 1) if k else 0.0
    got = L.orc_d1(_centre(a), 1, H)
    if k <= 4:
        assert got == pytest.approx(exact, rel=1e-10, abs=1e-10)
    else:
        assert abs(got - exact) > 1e-9  # 4th order, not 5th


@pytest.mark.parametrize("k", range(0, 7))
def test_second_derivative_exactness(k):
    a = _line(lambda x: x ** k)
    exact = k * (k - 1) * X0 ** (k - 2) if k >= 2 else 0.0
    got = L.orc_d2(_centre(a), 1, H)
    if k <= 5:
        assert got == pytest.approx(exact, rel=1e-8, abs=1e-8)
    else:
        assert abs(got - exact) > 1e-7


@pytest.mark.parametrize("a_pow,b_pow", [(a, b) for a in range(5) for b in range(5)])
def test_mixed_derivative_exactness(a_pow, b_pow):
    hx, hy = 0.021, 0.017
    x0, y0 = 0.4, -0.3
    g = np.empty((5, 5))
    for j in range(5):
        for i in range(5):
            g[j, i] = (x0 + (i - 2) * hx) ** a_pow * (y0 + (j - 2) * hy) ** b_pow
    g = np.ascontiguousarray(g.reshape(-1))
    base = ctypes.cast(g.ctypes.data + 8 * 12, ctypes.POINTER(ctypes.c_double))
    got = L.orc_d11(base, 1, 5, hx, hy)
    exact = (a_pow * x0 ** (a_pow - 1) if a_pow else 0.0) * (b_pow * y0 ** (b_pow - 1) if b_pow else 0.0)
    assert got == pytest.approx(exact, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("forward", [0, 1])
@pytest.mark.parametrize("k", range(0, 6))
def test_upwind_exactness(forward, k):
    a = _line(lambda x: x ** k)
    exact = k * X0 ** (k - 1) if k else 0.0
    got = L.orc_dup(_centre(a), 1, H, forward)
    if k <= 4:
        assert got == pytest.approx(exact, rel=1e-10, abs=1e-10)
    else:
        assert abs(got - exact) > 1e-9


def test_upwind_stencils_are_mirror_images():
    rng = np.random.default_rng(1)
    a = np.ascontiguousarray(rng.normal(size=9))
    b = np.ascontiguousarray(a[::-1])
    f = L.orc_dup(_centre(a), 1, H, 1)
    g = L.orc_dup(_centre(b), 1, H, 0)
    assert f == pytest.approx(-g, rel=1e-14)


@pytest.mark.parametrize("kind", range(5))
@pytest.mark.parametrize("k", range(0, 6))
def test_onesided_exactness(kind, k):
    a = _line(lambda x: x ** k)
    exact = k * X0 ** (k - 1) if k else 0.0
    got = L.orc_d1_onesided(_centre(a), 1, H, kind)
    if k <= 4:
        assert got == pytest.approx(exact, rel=1e-9, abs=1e-9)
    else:
        assert abs(got - exact) > 1e-9


@pytest.mark.parametrize("k", range(0, 7))
def test_ko_sixth_difference(k):
    a = _line(lambda x: x ** k)
    got = L.orc_ko6(_centre(a), 1)
    if k <= 5:
        assert abs(got) < 1e-12
    else:
        assert got == pytest.approx(720.0 * H ** 6, rel=1e-6)


def test_ko_nyquist():
    a = np.ascontiguousarray([(-1.0) ** i for i in range(9)])
    assert L.orc_ko6(_centre(a), 1) == -64.0 * a[4]


def test_rk4_amplification():
    lam = np.array([-3.0, -0.7, 0.0, 0.4, 1.3])
    y = np.ones_like(lam)
    dt = 0.37
    O.rk4_generic(y, dt, lambda v: lam * v)
    z = lam * dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    np.testing.assert_allclose(y, R, rtol=1e-14, atol=1e-15)


def test_rk4_is_fourth_order_on_nonlinear():
    # y' = -y^2, y(0)=1: y(t) = 1/(1+t).  Global error ~ dt^4.
    errs = []
    for n in (10, 20, 40):
        y = np.array([1.0])
        for _ in range(n):
            O.rk4_generic(y, 1.0 / n, lambda v: -v * v)
        errs.append(abs(y[0] - 0.5))
    for e1, e2 in zip(errs, errs[1:]):
        assert math.log2(e1 / e2) == pytest.approx(4.0, abs=0.3)


def test_splitmix_uniform_range_and_reference_value():
    # SplitMix64 reference output: a generator seeded with 0 first returns 0xE220A8397B1DCDAF.
    u = 0xE220A8397B1DCDAF
    expect = 2.0 * ((u >> 11) * 2.0 ** -53) - 1.0
    assert L.orc_splitmix_uniform(0, 0) == expect
    vals = np.array([L.orc_splitmix_uniform(12345, c) for c in range(2000)])
    assert vals.min() >= -1.0 and vals.max() < 1.0
    assert abs(vals.mean()) < 0.05


def _det_state(o, h6):
    y = o.zeros()
    T = o.T
    for s in range(6):
        y[s * T:(s + 1) * T] = h6[s]
    return y


def test_det_enforcement_exact_and_precise():
    """det(gammabar) = det(gammahat) enforcement: det(I + h) = 1 afterwards; the result equals
    (I + h) det^(-1/3) - I evaluated in 50-digit arithmetic; tiny h keeps its relative precision."""
    mpmath = pytest.importorskip("mpmath")
    from oracle.oracle import Oracle
    from paper_2505_00097_gb300 import workloads as W
    o = Oracle(W.sinh_spherical((2, 2, 2)))
    T = o.T
    rng = np.random.default_rng(3)
    for amp in (0.1, 1e-6, 1e-11):
        h6 = rng.uniform(-amp, amp, size=(6, T))
        y = _det_state(o, h6)
        o.enforce_detgb(y)
        mpmath.mp.dps = 50
        for p in range(0, T, max(1, T // 40)):
            H = mpmath.matrix(3, 3)
            for s, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
                H[a, b] = H[b, a] = mpmath.mpf(h6[s, p])
            G = mpmath.eye(3) + H
            f = mpmath.det(G) ** (-mpmath.mpf(1) / 3)
            for s, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
                exact = G[a, b] * f - (1 if a == b else 0)
                got = y[s * T + p]
                assert abs(got - float(exact)) <= 4e-16 * max(abs(float(exact)), amp), (amp, s, got, exact)
            Gn = np.eye(3)
            for s, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
                Gn[a, b] += y[s * T + p]
                Gn[b, a] = Gn[a, b]
            assert abs(np.linalg.det(Gn) - 1.0) < 1e-14
