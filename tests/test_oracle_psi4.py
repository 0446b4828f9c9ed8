"""Pins of the oracle's Weyl scalar psi4 and its spin-weight -2 decomposition (Sec. 4.1).

* the spin-weighted harmonics equal the textbook closed forms for l = 2 and are
  orthonormal on the sphere (numpy's Gauss-Legendre rule, not the oracle's);
* a linearised plane gravitational wave h_ij = eps e_ij f(t - k.x) travelling along the
  radial direction of a point P gives psi4(P) = f'' eps (e_+ - i e_x), i.e.
  d_t^2 h_+ - i d_t^2 h_x with h_+, h_x relative to the tetrad's theta and phi
  directions (sign and normalisation of the convention), at 4th order;
* Schwarzschild in Kerr-Schild coordinates (shifted, K != 0) is purely electric with
  E_rr = -2M/r^3, E_thth = E_phph = M/r^3 in the tetrad and B = 0, psi4 = 0, at 4th
  order;
* the modes of a field sum_lm a_lm -2Y_lm(theta, phi) g(r) on a sphere recover a_lm g(R)
  at the interpolation's 4th order, exactly for the quadrature.
"""
import math

import numpy as np
import pytest

from oracle import oracle as OL
from oracle.oracle import Oracle
from paper_2505_00097_gb300 import workloads as W
from tests.test_oracle_physics import SYM, _frames, _orders, _region, _to_frame_sym


def test_spin_weighted_harmonics_closed_forms_and_orthonormality():
    for th, ph in [(0.3, 0.1), (1.2, -2.0), (2.5, 2.9)]:
        c, s = math.cos(th), math.sin(th)
        ref = {0: 0.25 * math.sqrt(15 / (2 * math.pi)) * s * s,
               1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c), -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
               2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2, -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2}
        for m, a in ref.items():
            assert OL.sylm(-2, 2, m, th, ph) == pytest.approx(a * complex(math.cos(m * ph), math.sin(m * ph)),
                                                               abs=1e-14)
    x, w = np.polynomial.legendre.leggauss(20)
    phs = -math.pi + 2 * math.pi * (np.arange(40) + 0.5) / 40
    modes = [(l, m) for l in range(2, 6) for m in range(-l, l + 1)]
    Y = np.array([[[OL.sylm(-2, l, m, math.acos(xi), p) for p in phs] for xi in x] for l, m in modes])
    G = np.einsum("aij,bij,i->ab", Y, Y.conj(), w) * (2 * math.pi / 40)
    np.testing.assert_allclose(G, np.eye(len(modes)), atol=1e-13)


def _plane_wave_state(o, P, eps=1e-6, om=1.0, ep=1.0, ex=0.5):
    """linearised TT wave along the radial direction of grid point P; returns state and exact psi4(P)"""
    x = o.cart()
    xp = x[P]
    r = np.linalg.norm(xp)
    th, ph = math.acos(xp[2] / r), math.atan2(xp[1], xp[0])
    k = xp / r
    et = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    ephi = np.array([-math.sin(ph), math.cos(ph), 0.0])
    e = ep * (np.outer(et, et) - np.outer(ephi, ephi)) + ex * (np.outer(et, ephi) + np.outer(ephi, et))
    u = -(x @ k)                      # t - k.x at t = 0
    f, fp = np.sin(om * u + 0.3), om * np.cos(om * u + 0.3)
    gam = np.eye(3)[None] + eps * e[None] * f[:, None, None]
    Kc = -0.5 * eps * e[None] * fp[:, None, None]            # K_ij = -1/2 d_t h_ij
    det = np.linalg.det(gam)
    Wv = det ** (-1.0 / 6.0)
    gb = Wv[:, None, None] ** 2 * gam
    trK = np.einsum("pij,pij->p", np.linalg.inv(gam), Kc)
    A = Wv[:, None, None] ** 2 * (Kc - gam * trK[:, None, None] / 3)
    E = _frames(o)
    T = o.T
    y = o.zeros()
    h = _to_frame_sym(E, gb) - np.array([1, 0, 0, 1, 0, 1.0])[:, None]
    a = _to_frame_sym(E, A)
    for s in range(6):
        y[s * T:(s + 1) * T] = h[s]
        y[(6 + s) * T:(7 + s) * T] = a[s]
    y[12 * T:13 * T] = Wv
    y[13 * T:14 * T] = trK
    y[23 * T:24 * T] = 1.0
    fpp = -om * om * math.sin(om * u[P] + 0.3)
    return y, eps * fpp * complex(ep, -ex)


def test_linear_plane_wave_gives_hdd_plus_minus_i_hdd_cross():
    errs = []
    for N in [(32, 16, 32), (64, 32, 64)]:
        o = Oracle(W.sinh_spherical(N, ampl=12.0, w=0.5, ko_sigma=0.0))
        sel = np.nonzero(_region(o, 3.0, 5.0))[0]
        x = o.cart()
        th = np.arccos(x[sel, 2] / np.linalg.norm(x[sel], axis=1))
        pts = sel[(th > 0.6) & (th < 2.5)]
        e = 0.0
        for P in pts[:: max(1, len(pts) // 3)][:3]:
            y, exact = _plane_wave_state(o, P)
            p4 = o.psi4(y)[0]
            got = complex(p4[0, P], p4[1, P])
            e = max(e, abs(got - exact) / abs(exact))
        errs.append(e)
    assert errs[-1] < 2e-3, errs
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=0.8), errs


def test_schwarzschild_is_purely_electric():
    pytest.importorskip("sympy")
    import sympy as sp

    from tests.test_oracle_kerr_schild import XS, X, Y, Z, _ev, _ks_lambdified, _ks_state
    from tests.test_oracle_physics import _to_frame_vec
    F = _ks_lambdified()
    r = sp.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    l = [X / r, Y / r, Z / r]
    gam = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) + 2 / r * l[i] * l[j])
    gbs = (1 + 2 / r) ** sp.Rational(-1, 3) * gam
    dgb = sp.lambdify(XS, [sp.diff(gbs[i, j], XS[k]) for i in range(3) for j in range(3) for k in range(3)],
                      modules="numpy", cse=True)
    errs = []
    for N in [(24, 24, 24), (48, 48, 48)]:
        o = Oracle(W.sinh_spherical(N, ampl=12.0, w=0.3, ko_sigma=0.0))
        T = o.T
        y, gb, x, E = _ks_state(o, F)
        dg = _ev(dgb, x, (3, 3, 3))
        gbi = np.linalg.inv(gb)
        Gam = 0.5 * (np.einsum("pil,pjlk->pijk", gbi, dg) + np.einsum("pil,pklj->pijk", gbi, dg)
                     - np.einsum("pil,pjkl->pijk", gbi, dg))
        lam = _to_frame_vec(E, np.einsum("pjk,pijk->pi", gbi, Gam))
        for dd in range(3):
            y[(14 + dd) * T:(15 + dd) * T] = lam[dd]
        p4, Et, Bt = o.psi4(y)
        sel = _region(o, 3.0, 7.0)
        rr = np.linalg.norm(x, axis=1)
        exact = [-2 / rr ** 3, 0 * rr, 0 * rr, 1 / rr ** 3, 0 * rr, 1 / rr ** 3]
        e = max(np.abs(Et[s] - exact[s])[sel].max() for s in range(6))
        e = max(e, np.abs(Bt[:, sel]).max(), np.abs(p4[:, sel]).max())
        errs.append(e)
    assert errs[-1] < 1e-4
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=0.8), errs


@pytest.mark.parametrize("coords", ["sph", "cyl"])
def test_modes_of_a_synthetic_field(coords):
    coef = {(2, 0): 1.0 + 0.5j, (2, 1): -0.3j, (3, -2): 0.2, (4, 0): -0.7, (8, 3): 0.1 + 0.1j}
    Rext = 4.0
    errs = []
    for N in ([(32, 16, 32), (64, 32, 64)] if coords == "sph" else [(32, 16, 64), (64, 32, 128)]):
        spec = (W.sinh_spherical(N, ampl=12.0, w=0.5) if coords == "sph"
                else W.sinh_cylindrical(N, rho_max=12.0, z_max=12.0, w=0.5))
        o = Oracle(spec)
        x = o.cart()
        rr = np.linalg.norm(x, axis=1)
        th = np.arccos(np.clip(x[:, 2] / rr, -1, 1))
        ph = np.arctan2(x[:, 1], x[:, 0])
        g = np.exp(-0.1 * rr) * (1 + 0.05 * rr)
        field = np.zeros(o.T, dtype=complex)
        for (l, m), a in coef.items():
            field += a * np.array([OL.sylm(-2, l, m, t, p) for t, p in zip(th, ph)])
        field *= g
        psi = np.array([field.real, field.imag]) * np.tile(o.interior_mask(), (2, 1))
        modes = o.psi4_modes(psi, Rext, ntheta=24, nphi=48, lmax=8)
        gR = math.exp(-0.1 * Rext) * (1 + 0.05 * Rext)
        q = 0
        e = 0.0
        for l in range(2, 9):
            for m in range(-l, l + 1):
                e = max(e, abs(modes[q] - coef.get((l, m), 0.0) * gR))
                q += 1
        errs.append(e)
    # the l = 8 content dominates: ~8 points per angular wavelength on the finer grid
    assert errs[-1] < 1e-3, errs
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=1.0), errs


def test_offset_schwarzschild_invariants_in_any_orthonormal_tetrad():
    """A Schwarzschild hole away from the origin: the tetrad (built from the origin's spherical
    directions) is not aligned with it and is orthonormalised by Gram-Schmidt in a metric with
    off-diagonal terms.  For vacuum type D, E_ab E_ab - B_ab B_ab = 6 M^2 / r^6 and E_ab B_ab = 0
    in every orthonormal tetrad (r: distance to the hole)."""
    sp = pytest.importorskip("sympy")

    from tests.test_oracle_kerr_schild import XS, X, Y, Z, _ev
    from tests.test_oracle_physics import _to_frame_vec
    c = (0.6, -0.4, 0.9)
    r = sp.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    Hf = 1 / r
    l = [(X - c[0]) / r, (Y - c[1]) / r, (Z - c[2]) / r]
    g = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) + 2 * Hf * l[i] * l[j])
    gi = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) - 2 * Hf * l[i] * l[j] / (1 + 2 * Hf))
    alpha = 1 / sp.sqrt(1 + 2 * Hf)
    beta_dn = [2 * Hf * l[i] for i in range(3)]
    d = lambda f, k: sp.diff(f, XS[k])  # noqa: E731
    Gam = [[[sum(gi[a, m] * (d(g[m, b], cc) + d(g[m, cc], b) - d(g[b, cc], m)) for m in range(3)) / 2
             for cc in range(3)] for b in range(3)] for a in range(3)]
    K = sp.Matrix(3, 3, lambda i, j: ((d(beta_dn[j], i) - sum(Gam[m][i][j] * beta_dn[m] for m in range(3)))
                                       + (d(beta_dn[i], j) - sum(Gam[m][j][i] * beta_dn[m] for m in range(3))))
                  / (2 * alpha))
    Wf = (1 + 2 * Hf) ** sp.Rational(-1, 6)
    gbs = Wf ** 2 * g
    lam = lambda e: sp.lambdify(XS, e, modules="numpy", cse=True)  # noqa: E731
    Fg = lam([g[i, j] for i in range(3) for j in range(3)])
    FK = lam([K[i, j] for i in range(3) for j in range(3)])
    FW = lam([Wf])
    Fdgb = lam([sp.diff(gbs[i, j], XS[k]) for i in range(3) for j in range(3) for k in range(3)])
    errs = []
    for N in [(24, 24, 24), (48, 48, 48)]:
        o = Oracle(W.sinh_spherical(N, ampl=12.0, w=0.3, ko_sigma=0.0))
        T = o.T
        x = o.cart()
        E = _frames(o)
        gam = _ev(Fg, x, (3, 3))
        Kij = _ev(FK, x, (3, 3))
        Wv = _ev(FW, x, (1,))[:, 0]
        gb = Wv[:, None, None] ** 2 * gam
        trK = np.einsum("pij,pij->p", np.linalg.inv(gam), Kij)
        A = Wv[:, None, None] ** 2 * (Kij - gam * trK[:, None, None] / 3.0)
        dg = _ev(Fdgb, x, (3, 3, 3))
        gbi = np.linalg.inv(gb)
        G3 = 0.5 * (np.einsum("pil,pjlk->pijk", gbi, dg) + np.einsum("pil,pklj->pijk", gbi, dg)
                    - np.einsum("pil,pjkl->pijk", gbi, dg))
        y = o.zeros()
        h = _to_frame_sym(E, gb) - np.array([1, 0, 0, 1, 0, 1.0])[:, None]
        a = _to_frame_sym(E, A)
        lv = _to_frame_vec(E, np.einsum("pjk,pijk->pi", gbi, G3))
        for s in range(6):
            y[s * T:(s + 1) * T] = h[s]
            y[(6 + s) * T:(7 + s) * T] = a[s]
        for dd in range(3):
            y[(14 + dd) * T:(15 + dd) * T] = lv[dd]
        y[12 * T:13 * T] = Wv
        y[13 * T:14 * T] = trK
        y[23 * T:24 * T] = 1.0
        _, Et, Bt = o.psi4(y)
        wgt = np.array([1, 2, 2, 1, 2, 1.0])[:, None]
        rb = np.linalg.norm(x - np.array(c), axis=1)
        sel = _region(o, 3.0, 7.0) & (rb > 2.5)
        I = (wgt * (Et * Et - Bt * Bt)).sum(0)
        J = (wgt * Et * Bt).sum(0)
        errs.append(max(np.abs(I - 6.0 / rb ** 6)[sel].max(), np.abs(J)[sel].max()))
    assert errs[-1] < 1e-5, errs
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=0.8), errs
