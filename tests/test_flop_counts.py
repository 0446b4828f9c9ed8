"""FP64 operation counts behind the roofline, reproduced on the CPU.

Two counting builds, each compiling its source unchanged with `double` replaced by a
number type that counts the FP64 operations issued on it:

* the oracle's (oracle/nr_oracle_count.cpp): one right-hand-side evaluation of the
  plain coordinate-basis discretisation (Sec. 2.1 equations, upwinded advection,
  Kreiss-Oliger dissipation), i.e. the work the method does when evaluated plainly.
  Its per-point count is bench.F_METHOD, reported as roofline.frac_method;
* the kernels' point code (tests/host_point/count_point.cpp): the census of what
  k_rhs and its k_d1 pre-pass issue per interior point in the source.  bench.F_ALG
  holds the counts of the compiled kernels (DADD + DMUL + 2 DFMA from ncu), which
  differ from the source by the compiler's common-subexpression elimination and its
  expansion of the one division; bench.KERNEL_CENSUS holds the census those counts
  were taken with, so a change of the point code's arithmetic fails here until both
  are brought up to date.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import bench
from oracle.oracle import Oracle
from paper_2505_00097_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
KO8 = [0.3] * 17 + [0.99] * 7

# a small grid of each workload's family (coordinates, azimuth kind, order)
FAMILY = {
    "headon": lambda N: W.sinh_cylindrical(N),
    "headon8": lambda N: dict(W.sinh_cylindrical(N), NG=5, ko_sigma=KO8),
    "large3d": lambda N: W.sinh_spherical(N),
    "large3d8": lambda N: dict(W.sinh_spherical(N), NG=5, ko_sigma=KO8),
}
SMALL = {"headon": [(16, 2, 32), (24, 2, 40)], "headon8": [(16, 2, 32), (20, 2, 36)],
         "large3d": [(12, 10, 8), (16, 12, 10)], "large3d8": [(12, 10, 10), (16, 12, 10)]}


def _compile(src, name, tmp, extra=()):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    so = str(tmp / name)
    r = subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-fno-fast-math", "-ffp-contract=off",
                        "-Wno-unused-function", *extra, src, "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return ctypes.CDLL(so)


@pytest.fixture(scope="module")
def ocount(tmp_path_factory):
    L = _compile(os.path.join(ROOT, "oracle", "nr_oracle_count.cpp"), "ocount.so",
                 tmp_path_factory.mktemp("ocount"), ("-fvisibility=hidden",))
    L.orc_count_rhs.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]
    return L


@pytest.fixture(scope="module")
def kcount(tmp_path_factory):
    L = _compile(os.path.join(HERE, "host_point", "count_point.cpp"), "kcount.so", tmp_path_factory.mktemp("kc"))
    dp = ctypes.POINTER(ctypes.c_double)
    L.census_rhs.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
    L.census_diag.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp, ctypes.c_int, dp,
                              ctypes.POINTER(ctypes.c_longlong)]
    return L


def _oracle_count(L, spec, seed=3):
    o = Oracle(spec)
    y = W.random_state(o.n, seed=seed)
    o.inner_bc(y)
    rhs = np.zeros_like(y)
    out = (ctypes.c_longlong * 6)()
    L.orc_count_rhs(ctypes.byref(o.p), y.ctypes.data, rhs.ctypes.data, out)
    return np.array(list(out), dtype=np.int64), math.prod(spec["N"]), o, y, rhs


@pytest.mark.parametrize("wl", sorted(FAMILY))
def test_oracle_counting_build(ocount, wl):
    """The counting build computes the oracle's right-hand side bit for bit, its counts do not
    depend on the data, and its per-point count (from two grid sizes, which removes the per-call
    set-up of the stencil weights) is bench.F_METHOD."""
    (c1, n1, o, y, rhs), (c2, n2, *_) = [_oracle_count(ocount, FAMILY[wl](N)) for N in SMALL[wl]]
    m = np.tile(o.interior_mask(), 24)
    assert np.array_equal(rhs[m], o.rhs(y)[m])
    c1b = _oracle_count(ocount, FAMILY[wl](SMALL[wl][0]), seed=11)[0]
    assert np.array_equal(c1, c1b)
    per = (c2 - c1) / (n2 - n1)
    assert np.all(per == np.round(per))
    add, mul, div = per[:3]
    assert add + mul + div == bench.F_METHOD[wl]
    assert per[3] == 0 and per[4] > 0       # no square root; the reference metric from library calls


def _census(L, spec, seed=5):
    o = Oracle(spec)
    y = W.random_state(o.n, seed=seed, smooth=True)
    o.inner_bc(y)
    rhs = np.zeros_like(y)
    out = (ctypes.c_longlong * 12)()
    ko = spec["ko_sigma"]
    km, kg = (ko[0], ko[17]) if isinstance(ko, (list, tuple)) else (ko, ko)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = L.census_rhs(spec["coords"], (ctypes.c_int * 3)(*spec["N"]), (ctypes.c_double * 3)(*spec["ampl"]),
                      (ctypes.c_double * 3)(*spec["sinhw"]), km, kg, 2.0, spec["NG"], y.ctypes.data_as(dp),
                      rhs.ctypes.data_as(dp), out)
    assert rc == 0
    v = list(out)
    return v, o, y, rhs


def _stored_differences_per_point(spec):
    """stored first differences of the k_d1 pre-pass per interior point at the workload's size"""
    N0, N1, N2 = spec["N"]
    E = spec["NG"] - 1
    cyl = spec["coords"] == W.SINH_CYLINDRICAL
    ax = 1 if (cyl and N1 == 2) else 2 if (not cyl and N2 == 2) else -1
    E1, E2 = (0 if ax == 1 else E), (0 if ax == 2 else E)
    n = N0 * (N1 + 2 * E1) * (N2 + 2 * E2) + (N0 * N1 * (N2 + 2 * E2) if ax < 0 else 0)
    return 11 * n / (N0 * N1 * N2)


@pytest.mark.parametrize("wl", sorted(FAMILY))
def test_kernel_census_matches_the_benchmark_constants(kcount, wl):
    """The census of the point code equals bench.KERNEL_CENSUS (the code whose compiled counts
    bench.F_ALG holds), its right-hand side agrees with the oracle's, and F_ALG is within 3 % of
    the census (the compiler's common subexpressions and division expansion)."""
    v, o, y, rhs = _census(kcount, FAMILY[wl](SMALL[wl][0]))
    add, mul, fma, div = v[:4]
    nint = v[10]
    assert v[4] == 0                             # no square root in the right-hand side
    assert div == nint                            # one division per point
    flops = (add + mul + 2 * fma + div) / nint
    assert flops == bench.KERNEL_CENSUS[wl]
    d_add, d_mul, d_fma, d_div = v[5:9]
    assert d_div == 0
    diffs = _stored_differences_per_point(FAMILY[wl](SMALL[wl][0]))
    per_diff = (d_add + d_mul + 2 * d_fma) / (diffs * nint)
    assert per_diff == (4.0 if FAMILY[wl]((8, 2, 8))["NG"] == 3 else 11.0)
    m = np.tile(o.interior_mask(), 24)
    ref = o.rhs(y)
    assert np.abs(rhs[m] - ref[m]).max() <= 1e-12 * np.abs(ref[m]).max()
    spec = bench.workload(wl)
    total = flops + per_diff * _stored_differences_per_point(spec)
    assert abs(bench.F_ALG[wl] / total - 1.0) <= 0.03, (bench.F_ALG[wl], total)
    # the FP64 instruction mix of the source: FLOPs over twice the instructions is the fraction of the
    # FLOP peak a fully busy FP64 pipe reaches (a DADD or DMUL is one FLOP in an FMA's slot)
    instr = (add + mul + fma) / nint + (d_add + d_mul + d_fma) / (diffs * nint) * _stored_differences_per_point(spec)
    assert abs(bench.MIX_CEILING[wl] - total / (2 * instr)) < 5e-4


def test_constraint_census_matches_the_benchmark_constants(kcount):
    """The Hamiltonian and momentum constraints' point code: its census equals bench.DIAG_CENSUS, and the
    compiled kernels' counts in bench.DIAG_FLOPS are within 0.5 % (Hamiltonian) and 5 % (momentum: the
    square root's expansion) of it."""
    spec = W.sinh_cylindrical((16, 2, 32))
    o = Oracle(spec)
    y = W.random_state(o.n, seed=5, smooth=True)
    o.inner_bc(y)
    out = (ctypes.c_longlong * 10)()
    dp = ctypes.POINTER(ctypes.c_double)
    assert kcount.census_diag(spec["coords"], (ctypes.c_int * 3)(*spec["N"]), (ctypes.c_double * 3)(*spec["ampl"]),
                              (ctypes.c_double * 3)(*spec["sinhw"]), 3, y.ctypes.data_as(dp), out) == 0
    v = list(out)
    n = v[9]
    ham = (v[0] + v[1] + 2 * v[2] + v[3]) / n
    mom = (v[4] + v[5] + 2 * v[6] + v[7]) / n
    assert v[3] == n and v[7] == n and v[8] == n      # one division each, one square root for |M|
    assert ham == bench.DIAG_CENSUS["headon"]["hamiltonian"] and mom == bench.DIAG_CENSUS["headon"]["momentum"]
    assert abs(bench.DIAG_FLOPS["headon"]["hamiltonian"] / ham - 1.0) <= 0.005
    assert abs(bench.DIAG_FLOPS["headon"]["momentum"] / mom - 1.0) <= 0.05
