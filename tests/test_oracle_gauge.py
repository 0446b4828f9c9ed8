"""Pins of the gauge equations (Sec. 2.1: 1+log slicing and the Gamma-driver shift) and of
the lapse terms of the K and Abar equations, on flat conformal data (h = a = 0, W = 1,
Lambdabar = 0) with beta = 0 and a smooth lapse alpha(x), trace K(x) and B^i(x).  There
every curvature and shift term vanishes identically, and the right-hand sides reduce to:
  exact at every point:   d_t alpha = -2 alpha K,   d_t W = alpha K W / 3,   d_t beta^i = B^i,
                          d_t h_ij = 0;
  at 4th order:           d_t Lambdabar^i = -(4/3) alpha D^i K,
                          d_t B^i = (3/4) d_t Lambdabar^i - eta B^i = -alpha D^i K - eta B^i,
                          d_t K = alpha K^2 / 3 - D^2 alpha,
                          d_t Abar_ij = -(D_i D_j alpha)^TF
(flat-space derivatives, frame components).  These fix the factor 2 of the slicing, the
3/4 and eta of the driver, the -4/3 of the K-gradient term and the signs of the lapse
Laplacian and Hessian."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_00097_gb300 import workloads as W
from tests.test_oracle_physics import _frames, _orders, _region, _to_frame_sym, _to_frame_vec

A, B, C, D, E_, F = 0.3, 0.2, 0.25, 0.15, 0.2, 0.1


def _alpha(x):
    """alpha, grad alpha, Hessian of alpha (Cartesian)"""
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    s, c = np.sin(A * X), np.cos(B * Y)
    al = 1.0 + 0.1 * s * c + 0.05 * np.cos(C * Z)
    g = np.stack([0.1 * A * np.cos(A * X) * c, -0.1 * B * s * np.sin(B * Y), -0.05 * C * np.sin(C * Z)], 1)
    H = np.zeros((len(x), 3, 3))
    H[:, 0, 0] = -0.1 * A * A * s * c
    H[:, 1, 1] = -0.1 * B * B * s * c
    H[:, 2, 2] = -0.05 * C * C * np.cos(C * Z)
    H[:, 0, 1] = H[:, 1, 0] = -0.1 * A * B * np.cos(A * X) * np.sin(B * Y)
    return al, g, H


def _trk(x):
    """K and grad K (Cartesian)"""
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    K = 0.2 * np.cos(D * X) + 0.1 * np.sin(E_ * Y + F * Z)
    g = np.stack([-0.2 * D * np.sin(D * X), 0.1 * E_ * np.cos(E_ * Y + F * Z), 0.1 * F * np.cos(E_ * Y + F * Z)], 1)
    return K, g


def _state(o):
    T = o.T
    x = o.cart()
    E = _frames(o)
    y = o.zeros()
    al, _, _ = _alpha(x)
    K, _ = _trk(x)
    y[12 * T:13 * T] = 1.0                      # W
    y[13 * T:14 * T] = K
    y[23 * T:24 * T] = al
    Bc = np.stack([0.02 * np.sin(0.2 * x[:, 2]), -0.03 * np.cos(0.1 * x[:, 0]), 0.01 * np.ones(T)], 1)
    Bf = _to_frame_vec(E, Bc)
    for d in range(3):
        y[(20 + d) * T:(21 + d) * T] = Bf[d]
    return y, x, E, Bf


def test_gauge_terms_exact():
    o = Oracle(W.sinh_spherical((16, 12, 12), ampl=12.0, w=0.3, ko_sigma=0.0))
    y, x, E, Bf = _state(o)
    T = o.T
    r = o.rhs(y)
    m = o.interior_mask()
    al = y[23 * T:24 * T]
    K = y[13 * T:14 * T]
    np.testing.assert_allclose(r[23 * T:24 * T][m], (-2.0 * al * K)[m], rtol=1e-15, atol=0)
    np.testing.assert_allclose(r[12 * T:13 * T][m], (al * K / 3.0)[m], rtol=1e-14, atol=1e-17)
    for d in range(3):   # the oracle unrescales and rescales: a few ulp
        np.testing.assert_allclose(r[(17 + d) * T:(18 + d) * T][m], Bf[d][m], rtol=1e-14, atol=1e-18)
    assert not np.any(r[0:6 * T].reshape(6, T)[:, m])


def test_gauge_and_lapse_terms_converge():
    eta = 2.0
    errs = {k: [] for k in ("lambda", "B", "K", "A")}
    for N in [(16, 16, 16), (32, 32, 32), (64, 64, 64)]:
        o = Oracle(W.sinh_spherical(N, ampl=12.0, w=0.3, ko_sigma=0.0, eta=eta))
        y, x, E, Bf = _state(o)
        T = o.T
        r = o.rhs(y)
        sel = _region(o, 2.0, 6.0)
        al, gal, Hal = _alpha(x)
        K, gK = _trk(x)
        gKf = _to_frame_vec(E, gK)
        lam_ex = -(4.0 / 3.0) * al * gKf
        B_ex = -al * gKf - eta * Bf
        lap = np.trace(Hal, axis1=1, axis2=2)
        K_ex = al * K * K / 3.0 - lap
        HTF = Hal - lap[:, None, None] * np.eye(3)[None] / 3.0
        A_ex = -_to_frame_sym(E, HTF)
        errs["lambda"].append(max(np.abs(r[(14 + d) * T:(15 + d) * T] - lam_ex[d])[sel].max() for d in range(3)))
        errs["B"].append(max(np.abs(r[(20 + d) * T:(21 + d) * T] - B_ex[d])[sel].max() for d in range(3)))
        errs["K"].append(np.abs(r[13 * T:14 * T] - K_ex)[sel].max())
        errs["A"].append(max(np.abs(r[(6 + s) * T:(7 + s) * T] - A_ex[s])[sel].max() for s in range(6)))
    for k, e in errs.items():
        assert e[-1] < 1e-4, (k, e)
        assert _orders(e)[-1] == pytest.approx(4.0, abs=0.6), (k, e)
