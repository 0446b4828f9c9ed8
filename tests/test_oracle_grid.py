"""Pins of the oracle's grid, reference metric, CFL step and boundary maps.

* dt: the paper's single-node test (Sec. 4.2.1) runs 7.5 M in 8428 steps on
  a 72x12x24 spherical grid at CFL 0.5 (Sec. 4.1): tests/golden/dt_pin.txt.
* reference metric: the Riemann tensor of gammahat built from the oracle's
  Gammahat and d Gammahat must vanish (flat space in curvilinear
  coordinates); d gammahat agrees with a numerical derivative of gammahat;
  Gammahat of plain spherical coordinates equals the textbook symbols.
* maps: the inverse-coordinate map equals a brute-force nearest Cartesian
  search on tiny grids; parity signs of each ghost class; idempotence.
* the worked example of Sec. 2.2 (tests/golden/worked_example_vector.txt).
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_00097_gb300 import workloads as W


def _golden(name):
    out = {}
    with open(f"tests/golden/{name}") as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(None, 1)
            out[k] = v.strip()
    return out


def test_dt_pin_8428_iterations():
    g = _golden("dt_pin.txt")
    N = tuple(int(v) for v in g["N"].split())
    o = Oracle(W.spherical(N, r_max=float(g["r_max"]), cfl=float(g["cfl"])))
    dt = o.dt()
    assert math.floor(float(g["t_final"]) / dt) == int(g["iterations"])


SPECS = [
    W.sinh_spherical((8, 6, 4)),
    W.spherical((8, 6, 4)),
    W.sinh_cylindrical((8, 4, 10), rho_max=5.0, z_max=4.0, w=0.3),
]


def _riemann(G, dG):
    # R^a_bcd = d_c G^a_db - d_d G^a_cb + G^a_ce G^e_db - G^a_de G^e_cb
    R = (np.einsum("adbc->abcd", dG) - np.einsum("acbd->abcd", dG)
         + np.einsum("ace,edb->abcd", G, G) - np.einsum("ade,ecb->abcd", G, G))
    return R


@pytest.mark.parametrize("spec", SPECS, ids=["sinhsph", "sph", "sinhcyl"])
def test_refmetric_flat_and_consistent(spec):
    o = Oracle(spec)
    rng = np.random.default_rng(7)
    for _ in range(6):
        if spec["coords"] == W.SINH_CYLINDRICAL:
            xx = np.array([rng.uniform(0.1, 0.9), rng.uniform(-3, 3), rng.uniform(-0.9, 0.9)])
        else:
            xx = np.array([rng.uniform(0.1, 0.9), rng.uniform(0.2, 2.9), rng.uniform(-3, 3)])
        S, g, dg, ddg, G, dG = o.refmetric(xx)
        scale = max(1.0, np.abs(dG).max(), np.abs(G).max() ** 2)
        assert np.abs(_riemann(G, dG)).max() < 1e-11 * scale
        np.testing.assert_allclose(np.diag(g), S ** 2, rtol=1e-14)
        # derivatives of gammahat and Gammahat vs 4th-order numerical derivatives
        h = 1e-4
        for k in range(3):
            e = np.zeros(3); e[k] = h
            gp = [o.refmetric(xx + s * e) for s in (-2, -1, 1, 2)]
            num_dg = (gp[0][1] - 8 * gp[1][1] + 8 * gp[2][1] - gp[3][1]) / (12 * h)
            num_dG = (gp[0][4] - 8 * gp[1][4] + 8 * gp[2][4] - gp[3][4]) / (12 * h)
            num_ddg = (gp[0][2] - 8 * gp[1][2] + 8 * gp[2][2] - gp[3][2]) / (12 * h)
            np.testing.assert_allclose(dg[..., k], num_dg, rtol=1e-7, atol=1e-7 * np.abs(dg).max())
            np.testing.assert_allclose(dG[..., k], num_dG, rtol=1e-7, atol=1e-7 * max(1, np.abs(dG).max()))
            np.testing.assert_allclose(ddg[..., k], num_ddg, rtol=1e-6, atol=1e-6 * max(1, np.abs(ddg).max()))


def test_refmetric_textbook_spherical():
    A = 2.5
    o = Oracle(W.spherical((4, 4, 4), r_max=A))
    xx = np.array([0.37, 1.1, 0.4])
    r, th = A * xx[0], xx[1]
    S, g, dg, ddg, G, dG = o.refmetric(xx)
    np.testing.assert_allclose(S, [A, r, r * math.sin(th)], rtol=1e-15)
    expect = np.zeros((3, 3, 3))
    expect[0, 1, 1] = -r / A
    expect[0, 2, 2] = -r * math.sin(th) ** 2 / A
    expect[1, 0, 1] = expect[1, 1, 0] = A / r
    expect[1, 2, 2] = -math.sin(th) * math.cos(th)
    expect[2, 0, 2] = expect[2, 2, 0] = A / r
    expect[2, 1, 2] = expect[2, 2, 1] = math.cos(th) / math.sin(th)
    np.testing.assert_allclose(G, expect, atol=1e-14)


TINY = [
    W.sinh_spherical((6, 4, 2)),
    W.sinh_spherical((5, 3, 4)),
    W.spherical((4, 5, 6)),
    W.sinh_cylindrical((6, 2, 5), rho_max=3.0, z_max=3.0),
    W.sinh_cylindrical((4, 6, 4), rho_max=3.0, z_max=2.0, w=0.4),
    # one or two cells per axis: ghost layers deeper than the grid wrap several times
    W.sinh_spherical((1, 2, 2)),
    W.sinh_spherical((3, 1, 4)),
    W.sinh_cylindrical((1, 2, 1), rho_max=3.0, z_max=3.0),
]


@pytest.mark.parametrize("spec", TINY, ids=[f"tiny{i}" for i in range(len(TINY))])
def test_map_equals_bruteforce(spec):
    o = Oracle(spec)
    rc1, s1, p1, c1 = o.build_map()
    rc2, s2, p2, c2 = o.build_map(brute=True)
    assert rc1 == 0 and rc2 == 0
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(c1, c2)


def _class_counts(o, cls):
    return np.bincount(cls, minlength=3)


@pytest.mark.parametrize("spec", [W.sinh_spherical((64, 16, 2)), W.sinh_cylindrical((16, 2, 32))],
                         ids=["c1", "cyl"])
def test_map_invariants(spec):
    o = Oracle(spec)
    rc, src, par, cls = o.build_map()
    assert rc == 0
    N, NG = spec["N"], 3
    n = [v + 2 * NG for v in N]
    T = n[0] * n[1] * n[2]
    interior = int(np.prod(N))
    cnt = _class_counts(o, cls)
    assert cnt[0] == interior
    # sources are canonical (interior or pure outer), never inner ghosts
    assert np.all(cls[src] != 2)
    assert np.all(src[cls != 2] == np.nonzero(cls != 2)[0])
    assert set(np.unique(par)) <= {-1, 1}
    # applying the inner boundary conditions twice changes nothing
    y = W.random_state(tuple(n), seed=3)
    o.inner_bc(y)
    y2 = y.copy()
    o.inner_bc(y2)
    assert np.array_equal(y, y2)
    # expected parity classes (rescaled-basis vectors): see Sec. 2.2 worked example
    i0, i1, i2 = np.unravel_index(np.arange(T), (n[2], n[1], n[0]))[::-1]
    if spec["coords"] == W.SINH_SPHERICAL:
        sel = (i0 < NG) & (i1 >= NG) & (i1 < NG + N[1]) & (i2 >= NG) & (i2 < NG + N[2])   # r < 0 only
        assert np.all(par[sel, 1:4] == [-1, 1, -1])
        sel = (i0 >= NG) & (i0 < NG + N[0]) & (i1 < NG) & (i2 >= NG) & (i2 < NG + N[2])   # theta < 0 only
        assert np.all(par[sel, 1:4] == [1, -1, -1])
        sel = (i0 >= NG) & (i0 < NG + N[0]) & (i1 >= NG) & (i1 < NG + N[1]) & (i2 < NG)   # phi periodic only
        assert np.all(par[sel, 1:4] == [1, 1, 1])
    else:
        sel = (i0 < NG) & (i1 >= NG) & (i1 < NG + N[1])                                   # rho < 0
        assert np.all(par[sel, 1:4] == [-1, -1, 1])
        sel = (i0 >= NG) & (i1 < NG)                                                       # phi periodic
        assert np.all(par[sel, 1:4] == [1, 1, 1])
    # DD parity is the product of the two vector parities
    for s, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        assert np.array_equal(par[:, 4 + s], par[:, 1 + a] * par[:, 1 + b])


def _frame_components_of_constant_vector(o, V):
    """Rescaled (orthonormal-frame) components of a constant Cartesian vector at every point,
    with the analytically continued frame of each point (spherical-like grids)."""
    n0, n1, n2 = o.n
    x1 = o.xx(1); x2 = o.xx(2)
    th = x1[None, :, None] * np.ones((n2, n1, n0))
    ph = x2[:, None, None] * np.ones((n2, n1, n0))
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    e0 = np.stack([st * cp, st * sp, ct])
    e1 = np.stack([ct * cp, ct * sp, -st])
    e2 = np.stack([-sp, cp, np.zeros_like(sp)])
    return [np.tensordot(V, e, axes=1).reshape(-1) for e in (e0, e1, e2)], (e0, e1, e2)


@pytest.mark.parametrize("spec", [W.sinh_spherical((16, 8, 6)), W.spherical((12, 6, 8), r_max=3.0)],
                         ids=["sinhsph", "sph"])
def test_worked_example_rescaled_vector(spec):
    """Sec. 2.2: V=(1,0,0) has rescaled components (sin th cos ph, cos th cos ph, -sin ph) that are
    regular everywhere; after the inner boundary conditions every ghost holds exactly these values
    (evaluated at its own, analytically continued, coordinates), and the same for any constant
    vector and any constant symmetric tensor."""
    g = _golden("worked_example_vector.txt")
    assert g["rescaled_components"].replace(" ", "") == "sin(th)*cos(ph);cos(th)*cos(ph);-sin(ph)"
    o = Oracle(spec)
    rc, src, par, cls = o.build_map()
    assert rc == 0
    T = o.T
    canon = cls != 2
    for V in (np.array([1.0, 0.0, 0.0]), np.array([0.3, -0.8, 0.45])):
        comps, (e0, e1, e2) = _frame_components_of_constant_vector(o, V)
        if V[0] == 1.0 and V[1] == 0.0:
            th = np.repeat(o.xx(1)[None, :, None], o.n[2], 0).repeat(o.n[0], 2).reshape(-1)
            ph = np.repeat(o.xx(2)[:, None, None], o.n[1], 1).repeat(o.n[0], 2).reshape(-1)
            np.testing.assert_allclose(comps[0], np.sin(th) * np.cos(ph), atol=1e-15)
            np.testing.assert_allclose(comps[1], np.cos(th) * np.cos(ph), atol=1e-15)
            np.testing.assert_allclose(comps[2], -np.sin(ph), atol=1e-15)
        y = np.zeros(24 * T)
        for gf0 in (14, 17, 20):  # lambdaU, vetU, betU are vectors
            for d in range(3):
                y[(gf0 + d) * T:(gf0 + d + 1) * T] = np.where(canon, comps[d], 12345.0)
        # a constant symmetric tensor in hDD and aDD
        Tc = np.array([[0.2, -0.1, 0.05], [-0.1, 0.4, 0.3], [0.05, 0.3, -0.6]])
        E = [e0.reshape(3, -1), e1.reshape(3, -1), e2.reshape(3, -1)]
        for s, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
            tab = np.einsum("ip,ij,jp->p", E[a], Tc, E[b])
            for gf0 in (0, 6):
                y[(gf0 + s) * T:(gf0 + s + 1) * T] = np.where(canon, tab, 12345.0)
        o.inner_bc(y)
        for d in range(3):
            for gf0 in (14, 17, 20):
                np.testing.assert_allclose(y[(gf0 + d) * T:(gf0 + d + 1) * T], comps[d], atol=1e-14)
        for s, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
            tab = np.einsum("ip,ij,jp->p", E[a], Tc, E[b])
            np.testing.assert_allclose(y[s * T:(s + 1) * T], tab, atol=1e-14)


def test_worked_example_coordinate_components():
    """Coordinate-basis components = rescaled / S_i (Sec. 2.2): with the oracle's scale factors,
    (sin th cos ph, cos th cos ph, -sin ph) / S gives the printed (.., cos th cos ph / r, -sin ph/(r sin th))."""
    A = 3.0
    o = Oracle(W.spherical((4, 4, 4), r_max=A))
    for xx in ([0.2, 0.7, 0.3], [0.9, 2.5, -2.0]):
        S = o.refmetric(np.array(xx))[0]
        r, th, ph = A * xx[0], xx[1], xx[2]
        resc = np.array([math.sin(th) * math.cos(ph), math.cos(th) * math.cos(ph), -math.sin(ph)])
        coord = resc / S
        # with r measured in the logical coordinate (dr = A dxx0), component 0 carries 1/A
        np.testing.assert_allclose(coord * np.array([A, 1, 1]),
                                   [math.sin(th) * math.cos(ph), math.cos(th) * math.cos(ph) / r,
                                    -math.sin(ph) / (r * math.sin(th))], rtol=1e-14)
