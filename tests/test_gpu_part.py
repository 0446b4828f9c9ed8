"""One grid cut into partitions (nr_part_*, the chare decomposition of Sec. 3) against the whole
grid on the same GPU: after every substage each partition computes the points it owns, fills
its inner boundary points (from its own points or by messages from other partitions) and
exchanges halos face by face.  Every point runs the single-grid arithmetic on the same values,
so the partitioned evolution must be bitwise that of nr_rk4_step / nr_ssprk3_step -- the
paper's check that the Charm++ and OpenMP codes agree."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle  # noqa: E402
from paper_2505_00097_gb300 import binding as B  # noqa: E402
from paper_2505_00097_gb300 import build as BUILD  # noqa: E402
from paper_2505_00097_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

KO8 = [0.3] * 17 + [0.99] * 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BUILD.build()
    B.lib()


CASES = [
    ("cyl-two-point", W.sinh_cylindrical((48, 2, 96), rho_max=20.0, z_max=20.0), (2, 1, 3),
     (0.5, 0.5), ((0, 0, 0.5), (0, 0, -0.5)), 0.0, "rk4", 100),
    ("sph-general", W.sinh_spherical((24, 12, 8)), (2, 2, 2), (1.0,), ((0.0, 0.0, 0.0),), 1e-10, "rk4", 100),
    ("spherical-ragged", W.spherical((19, 10, 12)), (3, 2, 3), (0.8,), ((0.05, 0.0, 0.1),), 1e-9, "rk4", 60),
    ("cyl-general", W.sinh_cylindrical((20, 8, 30), rho_max=20.0, z_max=20.0), (2, 2, 3),
     (0.6, 0.4), ((0.2, 0, 0.4), (0, 0, -0.6)), 1e-10, "rk4", 60),
    ("cyl-order8-ssprk3", dict(W.sinh_cylindrical((40, 2, 64), rho_max=20.0, z_max=20.0), NG=5, ko_sigma=KO8, cfl=0.35),
     (2, 1, 3), (0.5, 0.5), ((0, 0, 0.5), (0, 0, -0.5)), 0.0, "ssprk3", 60),
    ("sph-general-order8", dict(W.sinh_spherical((20, 12, 10)), NG=5, ko_sigma=KO8, cfl=0.35), (2, 2, 2),
     (1.0,), ((0.0, 0.0, 0.0),), 1e-10, "ssprk3", 30),
]


@pytest.mark.parametrize("name,spec,parts,masses,pos,amp,integ,steps", CASES, ids=[c[0] for c in CASES])
def test_partitioned_evolution_is_bitwise_the_whole_grid(name, spec, parts, masses, pos, amp, integ, steps):
    g = B.Grid(spec)
    g.set_brill_lindquist(masses, pos, amp, 21)
    pg = B.PartGrid(spec, parts)
    assert pg.nparts == int(np.prod(parts)) and pg.dt_cfl == g.dt_cfl
    pg.set_brill_lindquist(masses, pos, amp, 21)
    T = g.T
    a = np.empty(24 * T)
    b = np.empty(24 * T)
    g.get_state(a, True)
    pg.get_state(b, True)
    assert np.array_equal(a, b), "initial data"
    dt = g.dt_cfl
    (g.ssprk3_step if integ == "ssprk3" else g.rk4_step)(dt, steps)
    (pg.ssprk3_step if integ == "ssprk3" else pg.rk4_step)(dt, steps)
    g.get_state(a, True)
    pg.get_state(b, True)
    assert np.all(np.isfinite(a))
    assert np.array_equal(a, b), f"{name}: partitioned state differs after {steps} steps"
    assert pg.digest() == g.digest()
    # the constraint norms from the partitions' points: the whole grid's up to summation order
    l2, linf = pg.hamiltonian()
    l2g, linfg = g.hamiltonian()
    assert linf == linfg and l2 == pytest.approx(l2g, rel=1e-13)
    pg.close()
    g.close()


def test_partitioned_from_a_whole_state_on_the_device():
    """A seeded random state (inner ghosts made parity copies by the oracle) uploaded from a device
    array, advanced 10 RK4 steps, read back to a device array: bitwise the whole grid's."""
    spec = W.sinh_spherical((18, 10, 8))
    o = Oracle(spec)
    y = W.random_state(o.n, seed=91, smooth=True)
    o.inner_bc(y)
    g = B.Grid(spec)
    pg = B.PartGrid(spec, (2, 2, 2))
    yd = torch.from_numpy(y).to("cuda:0")
    g.set_state(yd, False)
    pg.set_state(yd, False)
    g.rk4_step(g.dt_cfl, 10)
    pg.rk4_step(g.dt_cfl, 10)
    a = torch.empty_like(yd)
    b = torch.full_like(yd, float("nan"))
    g.get_state(a, False)
    pg.get_state(b, False)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    pg.close()
    g.close()


def test_head_on_grid_in_four_slabs():
    """The head-on workload's grid (256x2x512) in 4 slabs along z, 20 RK4 steps: bitwise nr_rk4_step."""
    spec = W.config_headon()
    g = B.Grid(spec)
    g.set_brill_lindquist(spec["masses"], spec["positions"])
    pg = B.PartGrid(spec, (1, 1, 4))
    pg.set_brill_lindquist(spec["masses"], spec["positions"])
    g.rk4_step(g.dt_cfl, 20)
    pg.rk4_step(g.dt_cfl, 20)
    assert pg.digest() == g.digest()
    assert pg.messages[0] == 0 and pg.messages[3] == 6
    pg.close()
    g.close()
