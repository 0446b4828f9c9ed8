"""The kernels' per-point arithmetic (csrc/bssn_point.cuh), compiled for the host with g++
and evaluated at every interior point, against the oracle on the same seeded states.

This checks, without a GPU, that the kernels' formulation of the BSSN equations (Sec. 2:
the frame components, the rotation-generator form of the flat connection, the
regroupings of the Ricci tensor and the Lie derivatives, the merged advection +
dissipation stencil, the two-point-azimuth specialisations and the stored first
differences) computes the oracle's discrete right-hand side and constraints.  The GPU
parity tests check the compiled kernels themselves; both use the same tolerances:
  * right-hand side: 1e-12 of the largest component of each tensor;
  * Hamiltonian constraint: 1e-12 of its largest value;
  * momentum constraint: 1e-12 of its largest component.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_00097_gb300 import workloads as W
from tests._common import assert_close

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host_point", "host_point.cpp")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    so = str(tmp_path_factory.mktemp("host_point") / "host_point.so")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-Wall", "-Wno-unknown-pragmas",
                        SRC, "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.host_point.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp, dp, ctypes.c_double, dp, dp,
                             ctypes.c_int, ctypes.c_int]
    L.host_point.restype = None
    return L


def _run(L, spec, y, which, out_len):
    dp = ctypes.POINTER(ctypes.c_double)
    N = (ctypes.c_int * 3)(*spec["N"])
    A = (ctypes.c_double * 3)(*spec["ampl"])
    w = (ctypes.c_double * 3)(*spec["sinhw"])
    ko = spec.get("ko_sigma", 0.3)
    sig = (ctypes.c_double * 24)(*(list(ko) if isinstance(ko, (list, tuple)) else [ko] * 24))
    out = np.zeros(out_len)
    L.host_point(int(spec["coords"]), N, A, w, sig, float(spec.get("eta", 2.0)), y.ctypes.data_as(dp),
                 out.ctypes.data_as(dp), which, int(spec.get("NG", 3)))
    return out


GRIDS4 = [
    ("sinhsph_general", W.sinh_spherical((10, 8, 6))),
    ("sinhcyl_general", W.sinh_cylindrical((10, 4, 12), rho_max=5.0, z_max=5.0)),
    ("spherical_general", W.spherical((8, 6, 8))),
    ("sinhsph_two_point_phi", W.sinh_spherical((12, 8, 2))),
    ("sinhcyl_two_point_phi", W.sinh_cylindrical((12, 2, 14), rho_max=5.0, z_max=5.0)),
]


def _order8(spec):
    s = dict(spec)
    s.update(NG=5, ko_sigma=[0.3] * 17 + [0.99] * 7)
    return s


GRIDS8 = [
    ("sinhsph_general_ord8", _order8(W.sinh_spherical((12, 10, 6)))),
    ("sinhcyl_two_point_phi_ord8", _order8(W.sinh_cylindrical((14, 2, 16), rho_max=5.0, z_max=5.0))),
]


def _state(o, seed, smooth):
    y = W.random_state(o.n, seed=seed, smooth=smooth)
    o.inner_bc(y)
    return y


@pytest.mark.parametrize("name,spec", GRIDS4 + GRIDS8, ids=[g[0] for g in GRIDS4 + GRIDS8])
@pytest.mark.parametrize("smooth", [True, False], ids=["smooth", "noise"])
def test_rhs_matches_oracle(lib, name, spec, smooth):
    o = Oracle(spec)
    y = _state(o, 11, smooth)
    ref = o.rhs(y)
    m = o.interior_mask()
    got = _run(lib, spec, y, 0, y.size)
    assert_close(got, ref, o.T, 1e-12, mask=m, what=f"{name} rhs")
    # the same with the mixed derivatives from stored first differences: the same expression
    got_s = _run(lib, spec, y, 3, y.size)
    assert_close(got_s, ref, o.T, 1e-12, mask=m, what=f"{name} rhs, stored differences")
    assert np.array_equal(got_s[np.tile(m, 24)], got[np.tile(m, 24)])


@pytest.mark.parametrize("name,spec", GRIDS4 + GRIDS8[:1], ids=[g[0] for g in GRIDS4 + GRIDS8[:1]])
def test_constraints_match_oracle(lib, name, spec):
    o = Oracle(spec)
    y = _state(o, 12, True)
    m = o.interior_mask()
    H_ref = o.hamiltonian(y)[0]
    H = _run(lib, spec, y, 1, o.T)
    assert np.abs(H[m] - H_ref[m]).max() <= 1e-12 * np.abs(H_ref[m]).max()
    M_ref = o.momentum(y)[0]
    M = _run(lib, spec, y, 2, 3 * o.T).reshape(3, o.T)
    scale = np.abs(M_ref[:, m]).max()
    assert np.abs(M[:, m] - M_ref[:, m]).max() <= 1e-12 * scale


def test_planted_mistake_is_caught(lib):
    """The comparison is sharp enough to see a small change in one term: the oracle's
    right-hand side of K, scaled by (1 + 1e-9), no longer passes the same bound."""
    spec = W.sinh_cylindrical((12, 2, 14), rho_max=5.0, z_max=5.0)
    o = Oracle(spec)
    y = _state(o, 13, True)
    ref = o.rhs(y)
    got = _run(lib, spec, y, 0, y.size)
    m = o.interior_mask()
    assert_close(got, ref, o.T, 1e-12, mask=m, what="unchanged")
    g = W.GF_NAMES.index("trK")
    ref[g * o.T:(g + 1) * o.T] *= 1.0 + 1e-9
    with pytest.raises(AssertionError):
        assert_close(got, ref, o.T, 1e-12, mask=m, what="planted")


def _sc2_inputs():
    """Every exponent field with a few mantissas, both signs, zeros, the subnormal range,
    the edges of the normal range, infinities and NaNs, plus random bit patterns."""
    bits = []
    for e in range(0x800):
        for m in (0, 1, 0x8000000000000, 0xFFFFFFFFFFFFF, 0x123456789ABCD, 0x8000000000001, 0x7FFFFFFFFFFFF):
            for s in (0, 1):
                bits.append((s << 63) | (e << 52) | m)
    # subnormals whose scaling by 2^-1 rounds (ties to even and not) or renormalises
    for m in (2, 3, 5, 6, 7, 0x10, 0x11, 0x13, 0xFFFFF, 0x80000000, 0x4000000000000, 0xFFFFFFFFFFFFE):
        bits += [m, (1 << 63) | m]
    rng = np.random.default_rng(7)
    bits += [int(v) for v in rng.integers(0, 2 ** 63, size=20000, dtype=np.int64)]
    bits += [int(v) | (1 << 63) for v in rng.integers(0, 2 ** 63, size=20000, dtype=np.int64)]
    return np.array(bits, dtype=np.uint64).view(np.float64)


@pytest.mark.parametrize("K", [-1, 1, 2, 5, 9])
def test_power_of_two_scaling_is_the_ieee_product(lib, K):
    """sc2<K>, the point code's integer-pipe scaling by 2^K, gives the bits of the IEEE product
    x * 2^K for every input: normal numbers, zeros of both signs, subnormal inputs and results
    (rounded to nearest even), overflow to infinity, infinities and NaNs (quiet, payload kept)."""
    x = _sc2_inputs()
    out = np.empty_like(x)
    L = lib
    L.host_sc2.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.c_long]
    L.host_sc2.restype = ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    assert L.host_sc2(K, x.ctypes.data_as(dp), out.ctypes.data_as(dp), x.size) == 0
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        ref = x * np.float64(2.0) ** K
    bad = np.nonzero(out.view(np.uint64) != ref.view(np.uint64))[0]
    assert bad.size == 0, [(hex(int(x.view(np.uint64)[i])), hex(int(out.view(np.uint64)[i])),
                            hex(int(ref.view(np.uint64)[i]))) for i in bad[:8]]
