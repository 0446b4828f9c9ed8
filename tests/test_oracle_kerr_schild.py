"""Pin of the full nonlinear BSSN right-hand side: a stationary black hole.

Schwarzschild in Kerr-Schild coordinates (M = 1),
    gamma_ij = delta_ij + 2H l_i l_j,  alpha = (1 + 2H)^(-1/2),  beta^i = 2H l^i/(1 + 2H),
    H = M/r, l_i = x_i/r,  K_ij = (D_i beta_j + D_j beta_i)/(2 alpha),
is a time-independent solution of Einstein's equations with this lapse and shift.  Its BSSN
variables (W = det(gamma)^(-1/6), gammabar = W^2 gamma, K = gamma^ij K_ij,
Abar_ij = W^2 (K_ij - gamma_ij K/3), Lambdabar^i = Delta^i) therefore have vanishing
d_t of the conformal metric, Abar, W, K and Lambdabar in the continuum, and the discrete
right-hand sides must converge to zero at 4th order.  K and Abar are nonzero here, so
this fixes the nonlinear terms (-2 alpha Abar_ik Abar^k_j + alpha Abar_ij K in the Abar
equation, 1/3 alpha K^2 + alpha Abar_ij Abar^ij in the K equation) together with every
other term of the geometric equations in a strongly curved, shifted setting.
"""
import numpy as np
import pytest

sp = pytest.importorskip("sympy")

from oracle.oracle import Oracle  # noqa: E402
from paper_2505_00097_gb300 import workloads as W  # noqa: E402
from tests.test_oracle_physics import _frames, _orders, _region, _to_frame_sym, _to_frame_vec  # noqa: E402

X, Y, Z = sp.symbols("X Y Z", real=True)
XS = (X, Y, Z)


def _ks_lambdified():
    r = sp.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    Hf = 1 / r
    l = [X / r, Y / r, Z / r]
    g = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) + 2 * Hf * l[i] * l[j])
    gi = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) - 2 * Hf * l[i] * l[j] / (1 + 2 * Hf))
    alpha = 1 / sp.sqrt(1 + 2 * Hf)
    beta_up = [2 * Hf * l[i] / (1 + 2 * Hf) for i in range(3)]
    beta_dn = [2 * Hf * l[i] for i in range(3)]
    d = lambda f, k: sp.diff(f, XS[k])  # noqa: E731
    Gam = [[[sum(gi[a, m] * (d(g[m, b], c) + d(g[m, c], b) - d(g[b, c], m)) for m in range(3)) / 2
             for c in range(3)] for b in range(3)] for a in range(3)]
    K = sp.Matrix(3, 3, lambda i, j: ((d(beta_dn[j], i) - sum(Gam[m][i][j] * beta_dn[m] for m in range(3)))
                                       + (d(beta_dn[i], j) - sum(Gam[m][j][i] * beta_dn[m] for m in range(3))))
                  / (2 * alpha))
    detg = 1 + 2 * Hf
    Wf = detg ** sp.Rational(-1, 6)
    exprs = {
        "gam": [g[i, j] for i in range(3) for j in range(3)],
        "K": [K[i, j] for i in range(3) for j in range(3)],
        "W": [Wf], "alpha": [alpha], "beta": beta_up,
    }
    return {k: sp.lambdify(XS, v, modules="numpy", cse=True) for k, v in exprs.items()}


def _ev(fn, x, shape):
    vals = fn(x[:, 0], x[:, 1], x[:, 2])
    out = np.empty((len(x),) + shape)
    flat = out.reshape(len(x), -1)
    for c, v in enumerate(vals):
        flat[:, c] = v
    return out


def _ks_state(o, F):
    T = o.T
    x = o.cart()
    E = _frames(o)
    gam = _ev(F["gam"], x, (3, 3))
    Kij = _ev(F["K"], x, (3, 3))
    Wv = _ev(F["W"], x, (1,))[:, 0]
    al = _ev(F["alpha"], x, (1,))[:, 0]
    beta = _ev(F["beta"], x, (3,))
    gb = Wv[:, None, None] ** 2 * gam
    gi = np.linalg.inv(gam)
    trK = np.einsum("pij,pij->p", gi, Kij)
    A = Wv[:, None, None] ** 2 * (Kij - gam * trK[:, None, None] / 3.0)
    y = o.zeros()
    h = _to_frame_sym(E, gb) - np.array([1, 0, 0, 1, 0, 1.0])[:, None]
    a = _to_frame_sym(E, A)
    for s in range(6):
        y[s * T:(s + 1) * T] = h[s]
        y[(6 + s) * T:(7 + s) * T] = a[s]
    y[12 * T:13 * T] = Wv
    y[13 * T:14 * T] = trK
    y[23 * T:24 * T] = al
    v = _to_frame_vec(E, beta)
    for dd in range(3):
        y[(17 + dd) * T:(18 + dd) * T] = v[dd]
    return y, gb, x, E


def test_kerr_schild_is_stationary():
    F = _ks_lambdified()
    # Delta^i needs derivatives of gammabar: differentiate the closed form symbolically as well
    r = sp.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    l = [X / r, Y / r, Z / r]
    Hf = 1 / r
    gam = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) + 2 * Hf * l[i] * l[j])
    Wf = (1 + 2 * Hf) ** sp.Rational(-1, 6)
    gbs = Wf ** 2 * gam
    dgb = sp.lambdify(XS, [sp.diff(gbs[i, j], XS[k]) for i in range(3) for j in range(3) for k in range(3)],
                      modules="numpy", cse=True)
    errs = []
    for N in [(24, 24, 24), (48, 48, 48), (96, 96, 96)]:
        o = Oracle(W.sinh_spherical(N, ampl=12.0, w=0.3, ko_sigma=0.0))
        T = o.T
        y, gb, x, E = _ks_state(o, F)
        dg = _ev(dgb, x, (3, 3, 3))
        gbi = np.linalg.inv(gb)
        Gam = 0.5 * (np.einsum("pil,pjlk->pijk", gbi, dg) + np.einsum("pil,pklj->pijk", gbi, dg)
                     - np.einsum("pil,pjkl->pijk", gbi, dg))
        Delta = np.einsum("pjk,pijk->pi", gbi, Gam)
        lam = _to_frame_vec(E, Delta)
        for dd in range(3):
            y[(14 + dd) * T:(15 + dd) * T] = lam[dd]
        rr = o.rhs(y)
        sel = _region(o, 3.0, 7.0)
        errs.append(max(np.abs(rr[g * T:(g + 1) * T])[sel].max() for g in range(17)))
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=0.6), errs
