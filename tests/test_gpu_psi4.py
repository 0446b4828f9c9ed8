"""Waveform extraction of Sec. 4.1 on the GPU, through the C ABI, against the oracle.

* the Weyl scalar psi4 at every interior point: 1e-12 relative to the field's
  maximum, on noise and smooth random states, at 4th and 8th order, on grids with
  a two-point azimuth and on general ones; inner ghosts hold the value of the
  point they map to, outer ghosts are zero;
* the spin-weight -2 modes C_lm on a sphere: 1e-10 relative to the largest mode
  (the GPU takes -2Y_lm from Wigner's small-d matrix, the oracle from Goldberg's
  closed form, so the two agree to rounding only);
* spheres that reach the outer boundary and l_max above 16 are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle  # noqa: E402
from paper_2505_00097_gb300 import binding as B  # noqa: E402
from paper_2505_00097_gb300 import build as BUILD  # noqa: E402
from paper_2505_00097_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
KO8 = [0.3] * 17 + [0.99] * 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BUILD.build()
    B.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


SPECS = [
    W.sinh_spherical((64, 16, 2)),
    W.sinh_spherical((37, 11, 10)),
    W.sinh_cylindrical((33, 2, 70), rho_max=20.0, z_max=20.0),
    W.sinh_cylindrical((20, 6, 19), rho_max=5.0, z_max=5.0, w=0.4),
    dict(W.sinh_spherical((37, 11, 10)), NG=5, ko_sigma=KO8),
    dict(W.sinh_cylindrical((33, 2, 70), rho_max=20.0, z_max=20.0), NG=5, ko_sigma=KO8),
]
IDS = ["sph2", "sph3d", "cyl2", "cyl3d", "sph3d-o8", "cyl2-o8"]


def _psi4_both(spec, seed, smooth):
    o = Oracle(spec)
    g = B.Grid(spec)
    y = W.random_state(o.n, seed=seed, smooth=smooth)
    o.inner_bc(y)
    ref = o.psi4(y)[0]
    out = torch.full((2 * o.T,), float("nan"), dtype=torch.float64, device=DEV)
    g.psi4(out, _dev(y))
    torch.cuda.synchronize()
    return o, g, y, ref, out.cpu().numpy().reshape(2, o.T)


@pytest.mark.parametrize("smooth", [False, True], ids=["noise", "smooth"])
@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_psi4_field_parity(spec, smooth):
    o, g, y, ref, got = _psi4_both(spec, 41 + int(smooth), smooth)
    m = o.interior_mask()
    scale = np.abs(ref[:, m]).max()
    assert scale > 0.0 and np.all(np.isfinite(got))
    assert np.abs(got[:, m] - ref[:, m]).max() <= 1e-12 * scale
    src, par, cls = B.build_maps(spec["coords"], spec["N"], spec.get("NG", 3))
    gh = np.nonzero(cls == 2)[0]
    assert np.array_equal(got[:, gh], got[:, src[gh]])
    assert np.all(got[:, cls == 1] == 0.0)


def _radius(o, spec):
    if spec["coords"] == W.SINH_CYLINDRICAL:
        return 0.5 * min(spec["ampl"][0], spec["ampl"][2])
    r = np.sqrt((o.cart() ** 2).sum(1))[o.interior_mask()]
    return 0.5 * r.max()


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_psi4_modes_parity(spec):
    o = Oracle(spec)
    g = B.Grid(spec)
    y = W.random_state(o.n, seed=8, smooth=True)
    o.inner_bc(y)
    R = _radius(o, spec)
    ref = o.psi4_modes(o.psi4(y)[0], R, 20, 40, 6)
    got = g.psi4_modes(R, 20, 40, 6, _dev(y))
    assert got.shape == ref.shape == (sum(2 * l + 1 for l in range(2, 7)),)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_grid_state_is_the_default_input():
    spec = SPECS[1]
    o = Oracle(spec)
    g = B.Grid(spec)
    y = W.random_state(o.n, seed=3, smooth=True)
    o.inner_bc(y)
    g.set_state(y, True)
    a = torch.zeros(2 * o.T, dtype=torch.float64, device=DEV)
    b = torch.zeros_like(a)
    g.psi4(a)
    g.psi4(b, _dev(y))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    R = _radius(o, spec)
    assert np.array_equal(g.psi4_modes(R, 8, 16, 4), g.psi4_modes(R, 8, 16, 4, _dev(y)))


def test_bad_spheres_and_orders_are_refused():
    spec = SPECS[3]
    g = B.Grid(spec)
    with pytest.raises(B.NrError, match="outer boundary"):
        g.psi4_modes(0.99 * spec["ampl"][2], 8, 16, 4)
    with pytest.raises(B.NrError):
        g.psi4_modes(1.0, 8, 16, 17)
    with pytest.raises(B.NrError):
        g.psi4_modes(-1.0, 8, 16, 4)
    # 285 modes x 8e6 nodes: refused before any table is built
    with pytest.raises(B.NrError, match="2\\^26"):
        g.psi4_modes(1.0, 2000, 4000, 16)
