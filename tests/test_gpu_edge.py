"""Degenerate grids and calls through the C ABI, against the oracle.

* Grids with one to three cells along an axis, where the ghost layers are deeper than
  the grid and the parity map wraps several times (Sec. 3): the right-hand side with
  both boundary conditions (1e-12 per tensor) and a few steps of the integrator
  (1e-10), at both orders, on the two-point-azimuth and the general kernels.
* A step count of zero leaves the state untouched, bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle  # noqa: E402
from paper_2505_00097_gb300 import binding as B  # noqa: E402
from paper_2505_00097_gb300 import build as BUILD  # noqa: E402
from paper_2505_00097_gb300 import workloads as W  # noqa: E402
from tests._common import assert_close  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
KO8 = [0.3] * 17 + [0.99] * 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BUILD.build()
    B.lib()


TINY = [
    W.sinh_spherical((1, 2, 2)),                                          # two-point azimuth
    W.sinh_spherical((3, 1, 4)),                                          # general, one theta cell
    W.spherical((2, 3, 2)),
    W.sinh_cylindrical((1, 2, 1), rho_max=3.0, z_max=3.0),                # one cell in rho and z
    W.sinh_cylindrical((2, 4, 3), rho_max=3.0, z_max=3.0),                # general
    dict(W.sinh_spherical((3, 3, 4)), NG=5, ko_sigma=KO8),
    dict(W.sinh_spherical((1, 2, 2)), NG=5, ko_sigma=KO8),
    dict(W.sinh_cylindrical((1, 2, 1), rho_max=3.0, z_max=3.0), NG=5, ko_sigma=KO8),
]
IDS = ["sph122", "sph314", "plain232", "cyl121", "cyl243", "sph334-o8", "sph122-o8", "cyl121-o8"]


@pytest.mark.parametrize("spec", TINY, ids=IDS)
def test_rhs_and_boundaries_on_tiny_grids(spec):
    o = Oracle(spec)
    g = B.Grid(spec)
    y = W.random_state(o.n, seed=21, smooth=True)
    o.inner_bc(y)
    ref = o.full_rhs(y)
    yd = torch.from_numpy(y).to(DEV)
    out = torch.zeros_like(yd)
    g.rhs(yd, out)
    g.apply_bcs(yd, out)
    torch.cuda.synchronize()
    assert_close(out.cpu().numpy(), ref, o.T, 1e-12, what="tiny-grid rhs with boundaries")


@pytest.mark.parametrize("spec", TINY, ids=IDS)
def test_steps_on_tiny_grids(spec):
    o = Oracle(spec)
    masses, pos = (0.6, 0.4), ((0.0, 0.0, 0.45), (0.0, 0.0, -0.55))
    y = o.brill_lindquist(masses, pos, 1e-8, seed=4)
    g = B.Grid(spec)
    g.set_state(y, True)
    dt = o.dt()
    if spec["NG"] == 5:
        o.ssprk3(y, dt, 5)
        g.ssprk3_step(dt, 5)
    else:
        o.rk4(y, dt, 5)
        g.rk4_step(dt, 5)
    got = np.empty_like(y)
    g.get_state(got, True)
    assert np.all(np.isfinite(got))
    assert_close(got, y, o.T, 1e-10, what="tiny-grid steps")


def test_zero_steps_leave_the_state_untouched():
    spec = W.sinh_cylindrical((16, 2, 24), rho_max=20.0, z_max=20.0)
    g = B.Grid(spec)
    g.set_brill_lindquist((1.0,), ((0.0, 0.0, 0.0),), 1e-8, 3)
    a = np.empty(24 * g.T)
    g.get_state(a, True)
    g.rk4_step(g.dt_cfl, 0)
    g.ssprk3_step(g.dt_cfl, 0)
    b = np.empty_like(a)
    g.get_state(b, True)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_det_enforcement_isolated_by_a_vanishing_step():
    """det(gammabar) = det(gammahat) enforcement (after every substage) on its own: with
    dt = 1e-300 every stage input equals y bit for bit, so one RK4 step returns the enforced
    state.  h is random with det(1 + h) - 1 from 1e-8 to 5e-3, covering both evaluations of
    (1 + x)^(-1/3) - 1 in the kernel; the result agrees with the oracle's expm1/log1p form to
    round-off and has det(1 + h) = 1 to round-off."""
    spec = W.sinh_cylindrical((16, 2, 24), rho_max=20.0, z_max=20.0)
    o = Oracle(spec)
    T = o.T
    rng = np.random.default_rng(77)
    y = o.zeros()
    eps = 10.0 ** rng.uniform(-8.0, -2.3, size=T)
    for s in range(6):
        y[s * T:(s + 1) * T] = eps * rng.uniform(-1.0, 1.0, size=T)
    y[12 * T:13 * T] = 1.0
    y[23 * T:24 * T] = 1.0
    o.inner_bc(y)
    g = B.Grid(spec)
    g.set_state(y, True)
    g.rk4_step(1e-300, 1)
    got = np.empty_like(y)
    g.get_state(got, True)
    ref = y.copy()
    o.enforce_detgb(ref)
    m = o.interior_mask()
    h = got[:6 * T].reshape(6, T)[:, m]
    href = ref[:6 * T].reshape(6, T)[:, m]

    def det(hh):
        h00, h01, h02, h11, h12, h22 = hh
        return ((1 + h00) * ((1 + h11) * (1 + h22) - h12 * h12) - h01 * (h01 * (1 + h22) - h12 * h02)
                + h02 * (h01 * h12 - (1 + h11) * h02))

    x = np.abs(det(y[:6 * T].reshape(6, T)[:, m]) - 1.0)
    assert x.min() < 1e-6 and x.max() > 2.0 ** -10 and (x > 2.0 ** -10).sum() > 10   # both branches ran
    assert np.abs(h - href).max() <= 4e-16 * np.abs(href).max()
    assert np.abs(det(h) - 1.0).max() <= 1e-15


@pytest.mark.parametrize("bad", [float("nan"), float("inf")], ids=["nan", "inf"])
def test_a_non_finite_value_spreads_and_is_reported(bad):
    """A single non-finite h_ij value at one interior point reaches W and alpha through the
    stencils within a few steps (also through the exponent-field scalings of the point code),
    and nr_check_finite reports NR_ENONFINITE; a finite state passes."""
    spec = W.sinh_cylindrical((16, 2, 24), rho_max=20.0, z_max=20.0)
    g = B.Grid(spec)
    g.set_brill_lindquist((1.0,), ((0.0, 0.0, 0.0),), 0.0, 0)
    g.check_finite()
    y = np.empty(24 * g.T)
    g.get_state(y, True)
    n0, n1 = g.n[0], g.n[1]
    idx = 3 + 5 + n0 * (3 + n1 * (3 + 10))   # an interior point
    y[0 * g.T + idx] = bad
    g.set_state(y, True)
    g.rk4_step(g.dt_cfl, 3)
    with pytest.raises(B.NrError) as ei:
        g.check_finite()
    assert ei.value.code == 5
