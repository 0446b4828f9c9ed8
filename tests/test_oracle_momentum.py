"""Pins of the oracle's momentum constraint (Eq. Mconstraint).

Each test fixes the oracle against something other than itself:
* Brill-Lindquist data (Abar = K = 0) has M = 0 exactly;
* with gammabar = delta, Abar = 0 and a non-constant K, the constraint reduces
  to M^i = -2/3 psi^-4 d_i K (closed form, reached at 4th order);
* a Bowen-York extrinsic curvature (flat-space transverse-traceless) on any
  conformal factor, Abar^ij = psi^-6 Ahat^ij_BY, K = 0, solves the momentum
  constraint: the D Abar and 6 Abar d phi terms cancel, so M -> 0 at 4th order;
* the same physical data split two ways -- (gammabar = delta, W = psi^-2, Abar)
  and (gammabar = psi^4 delta, W = 1, psi^4 Abar) -- give the same M^i, since
  e^{-4 phi} (Dbar_j Abar^ij + 6 Abar^ij d_j phi) is the physical divergence
  for any conformal split.  In the first split the Delta terms vanish and in
  the second the d phi terms do, so each side checks the other (difference
  -> 0 at 4th order while M itself is of order one);
* Schwarzschild in Kerr-Schild coordinates (h, K and Abar all non-zero) is a
  vacuum solution: M -> 0 at 4th order.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_00097_gb300 import workloads as W
from tests.test_oracle_physics import SYM, _frames, _orders, _psi, _region, _to_frame_sym, _to_frame_vec

NS_SPH = [(24, 16, 8), (48, 32, 16), (96, 64, 32)]
NS_CYL = [(24, 8, 48), (48, 16, 96), (96, 32, 192)]
PUNCT = ((0.8,), ((0.0, 0.0, 0.0),))
P_BY = np.array([0.1, -0.2, 0.3])


def _spec(coords, N):
    if coords == "sph":
        return W.sinh_spherical(N, ampl=12.0, w=0.3, ko_sigma=0.0)
    return W.sinh_cylindrical(N, rho_max=12.0, z_max=12.0, w=0.3, ko_sigma=0.0)


def _by(x):
    """Bowen-York Ahat_ij (Cartesian, flat-space TT) of momentum P_BY at the origin"""
    r = np.sqrt((x * x).sum(1))
    nv = x / r[:, None]
    pn = nv @ P_BY
    A = (P_BY[None, :, None] * nv[:, None, :] + P_BY[None, None, :] * nv[:, :, None]
         - (np.eye(3)[None] - nv[:, :, None] * nv[:, None, :]) * pn[:, None, None])
    return 1.5 * A / r[:, None, None] ** 2


def _state(o, psi, A_cart, K, conformal_in_metric=False):
    """BSSN state with the physical metric psi^4 delta, Abar_ij from A_cart (gammabar = delta split),
    trace K; conformal_in_metric puts psi^4 into gammabar (W = 1) and rescales Abar by psi^4."""
    T = o.T
    E = _frames(o)
    y = o.zeros()
    a = _to_frame_sym(E, A_cart * (psi[:, None, None] ** 4 if conformal_in_metric else 1.0))
    for s, (i, j) in enumerate(SYM):
        if conformal_in_metric and i == j:
            y[s * T:(s + 1) * T] = psi ** 4 - 1.0
        y[(6 + s) * T:(7 + s) * T] = a[s]
    y[12 * T:13 * T] = 1.0 if conformal_in_metric else psi ** -2
    y[13 * T:14 * T] = K
    y[23 * T:24 * T] = 1.0
    return y, E


@pytest.mark.parametrize("coords", ["sph", "cyl"])
def test_brill_lindquist_momentum_is_exactly_zero(coords):
    o = Oracle(_spec(coords, (24, 16, 8) if coords == "sph" else (24, 8, 48)))
    y = o.brill_lindquist(*PUNCT)
    M, mag, l2, linf, cnt = o.momentum(y)
    assert cnt > 0 and np.all(M == 0.0) and linf == 0.0


@pytest.mark.parametrize("coords", ["sph", "cyl"])
def test_gradient_of_K_closed_form(coords):
    errs = []
    for N in (NS_SPH if coords == "sph" else NS_CYL):
        o = Oracle(_spec(coords, N))
        x = o.cart()
        psi, dpsi, _ = _psi(x, *PUNCT)
        c = np.array([0.3, -0.2, 0.5])
        d = x - c
        K = 0.2 * np.exp(-(d * d).sum(1) / 9.0)
        dK = K[:, None] * (-2.0 * d / 9.0)
        y, E = _state(o, psi, np.zeros((o.T, 3, 3)), K)
        M = o.momentum(y)[0]
        exact = _to_frame_vec(E, -(2.0 / 3.0) * psi[:, None] ** -4 * dK)
        sel = _region(o, 2.5, 6.0)
        errs.append(max(np.abs(M[q] - exact[q])[sel].max() for q in range(3)))
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=0.6), errs


@pytest.mark.parametrize("coords", ["sph", "cyl"])
def test_bowen_york_solves_the_momentum_constraint(coords):
    errs, scale = [], []
    for N in (NS_SPH if coords == "sph" else NS_CYL):
        o = Oracle(_spec(coords, N))
        x = o.cart()
        psi = _psi(x, *PUNCT)[0]
        y, E = _state(o, psi, psi[:, None, None] ** -6 * _by(x), np.zeros(o.T))
        M, mag, l2, linf, cnt = o.momentum(y, 2.5, 6.0)
        sel = _region(o, 2.5, 6.0)
        errs.append(mag[sel].max())
        # the two terms that cancel are each of order |P|/r^3 psi^-10 here
        scale.append(np.abs(_to_frame_sym(E, _by(x)))[:, sel].max())
    assert errs[-1] < 1e-3 * scale[-1]
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=0.6), errs


@pytest.mark.parametrize("coords", ["sph", "cyl"])
def test_conformal_split_invariance(coords):
    diffs, sizes = [], []
    for N in (NS_SPH if coords == "sph" else NS_CYL):
        o = Oracle(_spec(coords, N))
        x = o.cart()
        psi = _psi(x, *PUNCT)[0]
        c = np.array([0.4, 0.1, -0.3])
        d = x - c
        g = np.exp(-(d * d).sum(1) / 8.0)
        Xt = 0.05 * g[:, None, None] * (d[:, :, None] * d[:, None, :] - np.eye(3)[None] * (d * d).sum(1)[:, None, None] / 3)
        A = psi[:, None, None] ** -6 * _by(x) + Xt          # traceless, not divergence-free
        K = 0.1 * g
        ya, _ = _state(o, psi, A, K)
        yb, _ = _state(o, psi, A, K, conformal_in_metric=True)
        Ma, maga = o.momentum(ya)[:2]
        Mb, magb = o.momentum(yb)[:2]
        sel = _region(o, 2.5, 6.0)
        diffs.append(max(np.abs(Ma[q] - Mb[q])[sel].max() for q in range(3)))
        sizes.append(maga[sel].max())
    assert sizes[-1] > 1e-3
    assert diffs[-1] < 1e-4 * sizes[-1]
    assert _orders(diffs)[-1] == pytest.approx(4.0, abs=0.6), diffs


def test_kerr_schild_solves_the_momentum_constraint():
    pytest.importorskip("sympy")
    from tests.test_oracle_kerr_schild import _ks_lambdified, _ks_state
    F = _ks_lambdified()
    errs = []
    for N in [(24, 24, 24), (48, 48, 48), (96, 96, 96)]:
        o = Oracle(W.sinh_spherical(N, ampl=12.0, w=0.3, ko_sigma=0.0))
        y = _ks_state(o, F)[0]
        mag = o.momentum(y)[1]
        errs.append(mag[_region(o, 3.0, 7.0)].max())
    assert _orders(errs)[-1] == pytest.approx(4.0, abs=0.6), errs
