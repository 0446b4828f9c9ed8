"""Compact state transfer through the C ABI (nr_get_state_compact / nr_set_state_compact).

Inner ghost points hold parity copies of canonical points (Sec. 3), so the state at
the interior and pure outer points determines the whole padded array:
* the compact array equals the full state at the canonical points, in flat order,
  bit for bit (host and device variants);
* uploading it into a fresh grid reproduces the full state bit for bit, and both
  grids then evolve identically;
* for arbitrary ghost values, the upload leaves the oracle's inner boundary
  condition applied to the same canonical values.
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BUILD.build()
    B.lib()


SPECS = [
    W.sinh_cylindrical((48, 2, 96), rho_max=20.0, z_max=20.0),
    W.sinh_spherical((37, 11, 10)),
    dict(W.sinh_cylindrical((33, 2, 70), rho_max=20.0, z_max=20.0), NG=5, ko_sigma=[0.3] * 17 + [0.99] * 7),
]
IDS = ["cyl2", "sph3d", "cyl2-o8"]


def _canon(spec):
    cls = B.build_maps(spec["coords"], spec["N"], spec.get("NG", 3))[2]
    return np.nonzero(cls != 2)[0]


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_compact_round_trip_is_bit_exact(spec):
    masses, pos = (0.6, 0.4), ((0.0, 0.0, 0.45), (0.0, 0.0, -0.55))
    g = B.Grid(spec)
    g.set_brill_lindquist(masses, pos, 1e-8, 5)
    g.rk4_step(g.dt_cfl, 2)
    T = g.T
    canon = _canon(spec)
    nc = g.info.n_state_points
    assert nc == canon.size == g.interior + g.info.n_outer
    full = np.empty(24 * T)
    g.get_state(full, True)
    comp = np.empty(24 * nc)
    g.get_state_compact(comp, True)
    assert np.array_equal(comp.reshape(24, nc), full.reshape(24, T)[:, canon])
    dcomp = torch.empty(24 * nc, dtype=torch.float64, device=DEV)
    g.get_state_compact(dcomp, False)
    torch.cuda.synchronize()
    assert np.array_equal(dcomp.cpu().numpy(), comp)

    for from_host, src in ((True, comp), (False, dcomp)):
        g2 = B.Grid(spec)
        g2.set_state_compact(src, from_host)
        back = np.empty(24 * T)
        g2.get_state(back, True)
        assert np.array_equal(back.view(np.uint64), full.view(np.uint64))
        dt = g.dt_cfl
        ga = B.Grid(spec)
        ga.set_state(full, True)
        ga.rk4_step(dt, 3)
        g2.rk4_step(dt, 3)
        a = np.empty(24 * T)
        b = np.empty(24 * T)
        ga.get_state(a, True)
        g2.get_state(b, True)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_upload_rebuilds_inner_ghosts_as_the_oracle(spec):
    o = Oracle(spec)
    y = W.random_state(o.n, seed=12, smooth=False)
    canon = _canon(spec)
    comp = np.ascontiguousarray(y.reshape(24, o.T)[:, canon]).reshape(-1)
    o.inner_bc(y)
    g = B.Grid(spec)
    g.set_state_compact(comp, True)
    got = np.empty(24 * o.T)
    g.get_state(got, True)
    assert np.array_equal(got, y)


def test_compact_state_is_the_canonical_fraction_of_the_headon_grid():
    spec = W.config_headon()
    g = B.Grid(spec)
    info = g.info
    assert info.n_state_points == info.interior + info.n_outer
    # 256 x 2 x 512 interior points with three ghost layers: a quarter of the padded array
    assert 0.24 < info.n_state_points / info.T < 0.26


def test_stale_azimuthal_ghosts_are_refreshed_before_use():
    """With a two-point azimuth the integrators leave the azimuthal ghost copies of the state
    stale; the constraints and psi4 of the grid-owned state, called right after the steps, must
    see the refreshed copies -- the same values as the explicit full state."""
    spec = W.sinh_cylindrical((48, 2, 96), rho_max=20.0, z_max=20.0)
    g = B.Grid(spec)
    assert g.info.n_inner > g.info.n_inner_stencil
    g.set_brill_lindquist((0.6, 0.4), ((0.0, 0.0, 0.45), (0.0, 0.0, -0.55)), 1e-8, 5)
    g.rk4_step(g.dt_cfl, 5)
    T = g.T
    H_own = torch.zeros(T, dtype=torch.float64, device=DEV)
    n_own = g.hamiltonian(None, H_own)
    M_own = torch.zeros(3 * T, dtype=torch.float64, device=DEV)
    m_own = g.momentum(None, M_own)
    p_own = torch.zeros(2 * T, dtype=torch.float64, device=DEV)
    g.psi4(p_own)
    y = torch.empty(24 * T, dtype=torch.float64, device=DEV)
    g.get_state(y, False)
    H = torch.zeros_like(H_own)
    M = torch.zeros_like(M_own)
    p = torch.zeros_like(p_own)
    assert g.hamiltonian(y, H) == n_own
    assert g.momentum(y, M) == m_own
    g.psi4(p, y)
    torch.cuda.synchronize()
    assert torch.equal(H, H_own) and torch.equal(M, M_own) and torch.equal(p, p_own)
    # the refreshed ghosts are exact parity copies
    src, par, cls = B.build_maps(spec["coords"], spec["N"], 3)
    yh = y.cpu().numpy().reshape(24, T)
    gh = np.nonzero(cls == 2)[0]
    types = [4, 5, 6, 7, 8, 9, 4, 5, 6, 7, 8, 9, 0, 0, 1, 2, 3, 1, 2, 3, 1, 2, 3, 0]
    for gf in range(24):
        assert np.array_equal(yh[gf, gh], par[gh, types[gf]] * yh[gf, src[gh]])


@pytest.mark.parametrize("integrator", ["rk4", "ssprk3"])
@pytest.mark.parametrize("spec", [SPECS[0], SPECS[2], SPECS[1]], ids=["cyl2", "cyl2-o8", "sph3d"])
def test_step_io_equals_the_separate_calls(spec, integrator):
    """nr_step_io (upload, steps, read-back by the last stage into pinned host memory; or the
    gather-and-copy path for pageable memory) gives bit for bit what nr_set_state_compact, the
    steps and nr_get_state_compact give."""
    masses, pos = (0.6, 0.4), ((0.0, 0.0, 0.45), (0.0, 0.0, -0.55))
    g0 = B.Grid(spec)
    g0.set_brill_lindquist(masses, pos, 1e-8, 5)
    nc = g0.info.n_state_points
    c0 = np.empty(24 * nc)
    g0.get_state_compact(c0, True)
    dt = g0.dt_cfl
    step = g0.ssprk3_step if integrator == "ssprk3" else g0.rk4_step
    g0.set_state_compact(c0, True)
    step(dt, 3)
    ref = np.empty(24 * nc)
    g0.get_state_compact(ref, True)
    full_ref = np.empty(24 * g0.T)
    g0.get_state(full_ref, True)
    pinned_in = torch.from_numpy(c0).pin_memory()
    for out in (torch.zeros(24 * nc, dtype=torch.float64).pin_memory(), np.zeros(24 * nc)):
        g = B.Grid(spec)
        g.step_io(dt, 3, pinned_in, out, integrator)
        got = out.numpy() if isinstance(out, torch.Tensor) else out
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
        full = np.empty(24 * g.T)
        g.get_state(full, True)
        assert np.array_equal(full.view(np.uint64), full_ref.view(np.uint64))
        g.close()


_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x):
    """first output of SplitMix64 (Steele, Lea & Flood 2014) for states x (uint64, wrapping)"""
    z = x + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _host_digest(state, canon, T):
    """the digest nr_state_digest documents, over the canonical points, in numpy"""
    total = np.uint64(0)
    idx = canon.astype(np.uint64)
    with np.errstate(over="ignore"):
        for g in range(24):
            bits = state[g * T + canon].view(np.uint64)
            key = _splitmix64((np.uint64(g) << np.uint64(40)) | idx)
            total = total + np.sum(_splitmix64(bits ^ key), dtype=np.uint64)
    return int(total & _M64)


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_state_digest_is_the_documented_sum(spec):
    """nr_state_digest equals the documented sum computed on the host from the fetched state, for
    the grid-owned state and for a caller-owned copy; changing one canonical value changes it and
    changing an inner ghost does not."""
    g = B.Grid(spec)
    g.set_brill_lindquist((0.6, 0.4), ((0.0, 0.0, 0.45), (0.0, 0.0, -0.55)), 1e-8, 5)
    g.rk4_step(g.dt_cfl, 2)
    T = g.T
    canon = _canon(spec)
    full = np.empty(24 * T)
    g.get_state(full, True)
    d = g.digest()
    assert d == _host_digest(full, canon, T)
    y = torch.from_numpy(full).to(DEV)
    assert g.digest(y) == d
    y2 = full.copy()
    t = canon[canon.size // 2]
    y2[13 * T + t] = np.nextafter(y2[13 * T + t], np.inf)
    assert g.digest(torch.from_numpy(y2).to(DEV)) != d
    ghost = np.setdiff1d(np.arange(T), canon)[0]
    y3 = full.copy()
    y3[5 * T + ghost] += 1.0
    assert g.digest(torch.from_numpy(y3).to(DEV)) == d
    g.close()
