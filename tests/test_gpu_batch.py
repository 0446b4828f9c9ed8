"""Batched mode: many uneven grids advanced by one launch per substage over all their tiles.

Each grid's state after n batched steps must be bitwise the state after n
single-grid steps (nr_rk4_step, nr_ssprk3_step) from the same initial data -- for
every tile shape the autotuner can pick, in any batch composition and at both
finite-difference orders -- and therefore within the oracle tolerance of the
single-grid path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_00097_gb300 import binding as B  # noqa: E402
from paper_2505_00097_gb300 import build as BUILD  # noqa: E402
from paper_2505_00097_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TILES = [(32, 4), (64, 2), (128, 1), (16, 8), (32, 2), (64, 1), (32, 1)]
KO8 = [0.3] * 17 + [0.99] * 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BUILD.build()
    B.lib()


def _cyl_runs():
    runs = []
    for k, (nr, m1, d) in enumerate([(12, 0.5, 1.0), (20, 0.7, 0.6), (33, 0.4, 1.5), (16, 0.8, 2.0)]):
        s = W.sinh_cylindrical((nr, 2, 2 * nr + k), rho_max=30.0, z_max=30.0)
        s.update(masses=(m1, 1 - m1), positions=((0, 0, d * (1 - m1)), (0, 0, -d * m1)))
        runs.append(s)
    return runs


def _sph_runs(three_d=False):
    runs = []
    shapes = [(13, 6, 4), (11, 8, 6), (9, 5, 8)] if three_d else [(20, 8, 2), (13, 6, 2), (30, 10, 2)]
    for k, N in enumerate(shapes):
        s = W.sinh_spherical(N)
        s.update(masses=(1.0,), positions=((0, 0, 0.01 * k),), perturb=1e-8 * (k + 1))
        runs.append(s)
    return runs


def _cyl3d_runs():
    runs = []
    for k, (nr, nphi) in enumerate([(12, 4), (17, 6), (9, 8)]):
        s = W.sinh_cylindrical((nr, nphi, 2 * nr + k), rho_max=30.0, z_max=30.0)
        s.update(masses=(0.6, 0.4), positions=((0.1, 0, 0.4), (0, 0.05, -0.6)))
        runs.append(s)
    return runs


def _o8(runs):
    return [dict(s, NG=5, ko_sigma=KO8) for s in runs]


def _states(runs, nsteps, batched, tile=None, autotune=False, ssp=False):
    grids = [B.Grid(s) for s in runs]
    for g, s in zip(grids, runs):
        g.set_brill_lindquist(s["masses"], s["positions"], s.get("perturb", 0.0), 7)
    dts = [g.dt_cfl for g in grids]
    chosen = None
    if batched:
        b = B.Batch(grids)
        if tile:
            b.set_tile(*tile)
        if autotune:
            chosen = b.autotune(dts)
        (b.ssprk3_step if ssp else b.rk4_step)(dts, nsteps)
    else:
        for g, dt in zip(grids, dts):
            (g.ssprk3_step if ssp else g.rk4_step)(dt, nsteps)
    out = []
    for g in grids:
        st = np.empty(24 * g.T)
        g.get_state(st, True)
        out.append(st)
    if batched:
        b.close()
    for g in grids:
        g.close()
    return out, chosen


@pytest.mark.parametrize("tile", TILES, ids=[f"{a}x{b}" for a, b in TILES])
def test_batched_cylindrical_bitwise_equals_single_grid(tile):
    runs = _cyl_runs()
    ref, _ = _states(runs, 6, batched=False)
    got, _ = _states(runs, 6, batched=True, tile=tile)
    for a, b in zip(got, ref):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("tile", [(32, 4), (16, 8), (32, 1)], ids=["32x4", "16x8", "32x1"])
@pytest.mark.parametrize("three_d", [False, True], ids=["nphi2", "3d"])
def test_batched_spherical_bitwise_equals_single_grid(tile, three_d):
    runs = _sph_runs(three_d)
    ref, _ = _states(runs, 5, batched=False)
    got, _ = _states(runs, 5, batched=True, tile=tile)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("tile", [(32, 4), (64, 1)], ids=["32x4", "64x1"])
def test_batched_cylindrical_3d_bitwise_equals_single_grid(tile):
    runs = _cyl3d_runs()
    ref, _ = _states(runs, 4, batched=False)
    got, _ = _states(runs, 4, batched=True, tile=tile)
    for a, b in zip(got, ref):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("ssp", [False, True], ids=["rk4", "ssprk3"])
@pytest.mark.parametrize("tile", [(32, 4), (128, 1), (16, 8)], ids=["32x4", "128x1", "16x8"])
def test_batched_8th_order_bitwise_equals_single_grid(tile, ssp):
    runs = _o8(_cyl_runs())
    ref, _ = _states(runs, 5, batched=False, ssp=ssp)
    got, _ = _states(runs, 5, batched=True, tile=tile, ssp=ssp)
    for a, b in zip(got, ref):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("three_d", [False, True], ids=["nphi2", "3d"])
def test_batched_8th_order_spherical_ssprk3(three_d):
    runs = _o8(_sph_runs(three_d))
    ref, _ = _states(runs, 4, batched=False, ssp=True)
    got, _ = _states(runs, 4, batched=True, tile=(32, 4), ssp=True)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_one_batch_switches_integrators():
    """RK4, then SSPRK3, then RK4 again on one batch: the table and the graph follow the
    integrator, and each grid ends bitwise where the same sequence of single-grid steps ends."""
    runs = _cyl_runs()
    out = []
    for batched in (False, True):
        grids = [B.Grid(s) for s in runs]
        for g, s in zip(grids, runs):
            g.set_brill_lindquist(s["masses"], s["positions"], 0.0, 0)
        dts = [g.dt_cfl for g in grids]
        if batched:
            b = B.Batch(grids)
            b.rk4_step(dts, 2)
            b.ssprk3_step(dts, 2)
            b.rk4_step(dts, 1)
            b.close()
        else:
            for g, dt in zip(grids, dts):
                g.rk4_step(dt, 2)
                g.ssprk3_step(dt, 2)
                g.rk4_step(dt, 1)
        st = []
        for g in grids:
            a = np.empty(24 * g.T)
            g.get_state(a, True)
            st.append(a)
            g.close()
        out.append(st)
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_batch_membership_does_not_change_results():
    runs = _cyl_runs()
    alone, _ = _states(runs[1:2], 4, batched=True)
    mixed, _ = _states(runs, 4, batched=True)
    assert np.array_equal(alone[0], mixed[1])


def test_autotune_picks_a_compiled_shape_and_keeps_results():
    runs = _cyl_runs()
    ref, _ = _states(runs, 3, batched=False)
    got, chosen = _states(runs, 3, batched=True, autotune=True)
    assert tuple(chosen[:2]) in TILES and chosen[2] > 0
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_mixed_orders_and_streams_rejected():
    g4 = B.Grid(W.sinh_cylindrical((8, 2, 16), rho_max=10.0, z_max=10.0))
    g8 = B.Grid(dict(W.sinh_cylindrical((8, 2, 16), rho_max=10.0, z_max=10.0), NG=5, ko_sigma=KO8))
    with pytest.raises(B.NrError, match="8th-order"):
        B.Batch([g4, g8])
    s = torch.cuda.Stream()
    g5 = B.Grid(W.sinh_cylindrical((10, 2, 16), rho_max=10.0, z_max=10.0), stream=s.cuda_stream)
    with pytest.raises(B.NrError, match="stream"):
        B.Batch([g4, g5])


def test_mixed_families_rejected():
    g1 = B.Grid(W.sinh_cylindrical((8, 2, 16), rho_max=10.0, z_max=10.0))
    g2 = B.Grid(W.sinh_spherical((8, 4, 2)))
    with pytest.raises(B.NrError):
        B.Batch([g1, g2])
    with pytest.raises(B.NrError):
        B.Batch([g1, g1])
    g3 = B.Grid(W.sinh_cylindrical((8, 4, 16), rho_max=10.0, z_max=10.0))   # four-point azimuth
    with pytest.raises(B.NrError, match="azimuth"):
        B.Batch([g1, g3])
