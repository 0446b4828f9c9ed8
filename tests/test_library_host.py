"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point declared in include/nr.h, and its host logic -- closed-form boundary
maps and the CFL step -- agrees bit-exactly with the oracle's independent
inverse-coordinate maps."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_00097_gb300 import binding as B
from paper_2505_00097_gb300 import build as BUILD
from paper_2505_00097_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    BUILD.build()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nr_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = B.lib()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(B.EXPORTS) == declared


def test_params_default():
    p = B.NrParams()
    assert B.lib().nr_params_default(0, ctypes.byref(p)) == 0
    assert p.NG == 3 and p.eta == 2.0 and p.cfl == 0.5 and p.enforce_detgb == 1
    assert list(p.ko_sigma) == [0.3] * 24
    assert p.f_inf[12] == 1.0 and p.f_inf[23] == 1.0 and sum(p.f_inf) == 2.0


def test_invalid_arguments_are_reported():
    Nx = (ctypes.c_int * 3)(64, 16, 3)   # odd N_phi cannot map r<0 ghosts
    src = np.zeros(70 * 22 * 9, dtype=np.int32); cls = src.copy(); par = np.zeros(10 * src.size, dtype=np.int8)
    rc = B.lib().nr_build_maps(0, Nx, 3, src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               par.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                               cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert rc == 6 and b"even" in B.lib().nr_last_error()
    Nx = (ctypes.c_int * 3)(64, 16, 2)
    assert B.lib().nr_build_maps(0, Nx, 2, src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 par.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                 cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))) == 1


MAP_SPECS = [
    W.sinh_spherical((64, 16, 2)), W.sinh_spherical((6, 4, 2)), W.sinh_spherical((5, 3, 4)), W.spherical((4, 5, 6)),
    W.sinh_spherical((12, 8, 10)), W.sinh_cylindrical((16, 2, 32)), W.sinh_cylindrical((6, 2, 5)),
    W.sinh_cylindrical((4, 6, 4), w=0.4), W.sinh_cylindrical((7, 8, 3)),
    # five ghost layers (8th-order scheme)
    dict(W.sinh_spherical((12, 8, 2)), NG=5), dict(W.sinh_spherical((7, 5, 6)), NG=5),
    dict(W.sinh_cylindrical((9, 2, 11)), NG=5), dict(W.sinh_cylindrical((6, 6, 4), w=0.4), NG=5),
    # fewer theta cells than ghost layers: the deepest theta ghosts need repeated reflections
    W.sinh_spherical((1, 2, 2)), W.sinh_spherical((3, 1, 4)), W.spherical((2, 3, 2)),
    dict(W.sinh_spherical((3, 3, 4)), NG=5), dict(W.sinh_spherical((1, 1, 2)), NG=5),
    W.sinh_cylindrical((1, 2, 1)), dict(W.sinh_cylindrical((1, 4, 1)), NG=5),
]


@pytest.mark.parametrize("spec", MAP_SPECS,
                         ids=[f"{s['coords']}-{'x'.join(map(str, s['N']))}-ng{s['NG']}" for s in MAP_SPECS])
def test_maps_bit_exact_vs_oracle(spec):
    o = Oracle(spec)
    rc, s1, p1, c1 = o.build_map()
    assert rc == 0
    s2, p2, c2 = B.build_maps(spec["coords"], spec["N"], spec["NG"])
    np.testing.assert_array_equal(c2, c1)
    np.testing.assert_array_equal(s2, s1)
    np.testing.assert_array_equal(p2, p1)


@pytest.mark.parametrize("spec", [W.config_single_puncture(), W.config_headon(), W.spherical((72, 12, 24)),
                                  W.sinh_spherical((24, 12, 8))], ids=["c1", "c2", "sph", "sph3d"])
def test_dt_cfl_vs_oracle(spec):
    assert B.dt_cfl(spec) == pytest.approx(Oracle(spec).dt(), rel=1e-15)


def test_server_queue_and_policy_arguments_on_the_host():
    srv = B.Server(2 ** 30, 4)
    with pytest.raises(B.NrError):
        srv.set_policy("lifo")
    assert B.lib().nr_server_set_policy(srv.h, 1, -1) == 1
    srv.set_policy("srpt", 10 ** 6)
    spec = W.sinh_cylindrical((12, 2, 24), rho_max=30.0, z_max=30.0)
    spec.update(masses=(1.0,), positions=((0, 0, 0),))
    rid = srv.submit(spec, 0.5)
    info = srv.poll(rid)
    assert info["status"] == 0 and info["steps_done"] == 0   # queued: no device work until advance
    bad = dict(spec, N=(12, 2, 0))
    with pytest.raises(B.NrError):
        srv.submit(bad, 0.5)
    srv.close()


def test_dissipation_strengths_must_split_metric_and_gauge():
    ok = W.sinh_cylindrical((8, 2, 16), rho_max=10.0, z_max=10.0, ko_sigma=[0.3] * 17 + [0.99] * 7)
    dt = B.dt_cfl(ok)
    assert dt > 0.0
    bad = dict(ok, ko_sigma=[0.3] * 16 + [0.5] + [0.99] * 7)
    with pytest.raises(B.NrError, match="ko_sigma"):
        B.dt_cfl(bad)
    with pytest.raises(B.NrError, match="ko_sigma"):
        B.Grid(bad)


def test_ghost_layers_select_the_scheme():
    for NG, ok in ((3, True), (5, True), (4, False), (2, False)):
        spec = dict(W.sinh_cylindrical((8, 2, 16), rho_max=10.0, z_max=10.0), NG=NG)
        if ok:
            assert B.dt_cfl(spec) > 0.0
        else:
            with pytest.raises(B.NrError, match="NG"):
                B.dt_cfl(spec)
    # the integrator field: RK4 or SSPRK3, anything else is refused (grid set-up and server)
    spec = W.sinh_cylindrical((8, 2, 16), rho_max=10.0, z_max=10.0)
    p = B.make_params(spec)
    Nx = (ctypes.c_int * 3)(8, 2, 16)
    dt = ctypes.c_double()
    for integ, ok in ((0, True), (1, True), (2, False), (-1, False)):
        p.integrator = integ
        rc = B.lib().nr_dt_cfl(int(spec["coords"]), Nx, ctypes.byref(p), ctypes.byref(dt))
        assert (rc == 0) == ok
        if not ok:
            assert b"integrator" in B.lib().nr_last_error()
    srv = B.Server(2 ** 30, 2)
    spec = dict(spec, NG=5, masses=(1.0,), positions=((0, 0, 0),), integrator="ssprk3")
    assert srv.submit(spec, 1.0) >= 0
    srv.close()


# the C example of the user guide: create a grid, set Brill-Lindquist data, step, read H
C_EXAMPLE = r"""
#include <stdio.h>
#include "nr.h"

int main(void)
{
    nr_params p;
    nr_grid* g = NULL;
    const int N[3] = {256, 2, 512};
    const double mass[2] = {0.5, 0.5}, xyz[6] = {0.0, 0.0, 0.5, 0.0, 0.0, -0.5};
    nr_grid_info info;
    double l2 = 0.0, linf = 0.0;
    if (nr_params_default(NR_SINH_CYLINDRICAL, &p) != NR_OK) return 1;
    if (nr_grid_create(NR_SINH_CYLINDRICAL, N, &p, &g) != NR_OK) {
        fprintf(stderr, "%s\n", nr_last_error());
        return 1;
    }
    nr_query(g, &info);
    nr_set_brill_lindquist(g, 2, mass, xyz, 0.0, 0);
    nr_rk4_step(g, info.dt_cfl, 100);
    nr_hamiltonian(g, NULL, NULL, &l2, &linf);
    printf("t = %g  |H|_2 = %g\n", 100 * info.dt_cfl, l2);
    nr_grid_destroy(g);
    return 0;
}
"""


def test_header_is_plain_c_and_the_example_links(tmp_path):
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = tmp_path / "example.c"
    src.write_text(C_EXAMPLE)
    inc = os.path.join(ROOT, "include")
    lib = B.library_path()
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src),
                        "-o", str(tmp_path / "example"), lib, "-Wl,-rpath," + os.path.dirname(lib)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_null_handles_are_refused_by_every_entry_point():
    """Every entry point that takes a grid, batch or server handle returns NR_EINVAL (and a
    message) for a NULL handle instead of touching memory; destroy calls accept NULL."""
    L = B.lib()
    d = ctypes.c_double()
    i = ctypes.c_int()
    i64 = ctypes.c_int64()
    calls = {
        "nr_query": (None, None),
        "nr_set_brill_lindquist": (None, 0, None, None, 0.0, 0),
        "nr_rhs": (None, None, None),
        "nr_apply_bcs": (None, None, None),
        "nr_apply_inner_bcs": (None, None),
        "nr_rk4_step": (None, 0.1, 1),
        "nr_ssprk3_step": (None, 0.1, 1),
        "nr_hamiltonian": (None, None, None, ctypes.byref(d), ctypes.byref(d)),
        "nr_momentum": (None, None, None, ctypes.byref(d), ctypes.byref(d)),
        "nr_psi4": (None, None, None),
        "nr_psi4_modes": (None, None, 1.0, 8, 16, 4, None),
        "nr_get_state": (None, None, 1),
        "nr_set_state": (None, None, 1),
        "nr_get_state_compact": (None, None, 1),
        "nr_set_state_compact": (None, None, 1),
        "nr_step_io": (None, 0, 0.1, 1, None, None),
        "nr_sync": (None,),
        "nr_check_finite": (None,),
        "nr_batch_set_tile": (None, 32, 4),
        "nr_batch_autotune": (None, None, None, None, None),
        "nr_batch_rk4_step": (None, None, 1),
        "nr_batch_ssprk3_step": (None, None, 1),
        "nr_server_set_tile": (None, 32, 4),
        "nr_server_set_policy": (None, 0, 0),
        "nr_server_submit": (None, 0, None, None, 0, None, None, 1.0, 0, ctypes.byref(i64)),
        "nr_server_advance": (None, 1, ctypes.byref(i), ctypes.byref(i)),
        "nr_server_poll": (None, 0, ctypes.byref(i), ctypes.byref(i64), ctypes.byref(i64), ctypes.byref(d),
                           ctypes.byref(d)),
        "nr_server_fetch_state": (None, 0, None, 0),
    }
    for name, args in calls.items():
        fn = getattr(L, name)
        assert fn(*args) == 1, name
        assert L.nr_last_error(), name
    L.nr_grid_destroy(None)
    L.nr_batch_destroy(None)
    L.nr_server_destroy(None)
