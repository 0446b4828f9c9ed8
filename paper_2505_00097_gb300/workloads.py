"""Workload definitions and seeded synthetic inputs.

Plain data and random-number plumbing only: this module holds none of the
BSSN arithmetic.  It is the one module shared by the CUDA-path tests, the
oracle tests and bench.py.  Every workload is synthetic; the grids and
physics numbers follow arXiv 2505.00097 (Sec. 4.1 sinh-cylindrical head-on
grids with rho_max = z_max = 300, w = 0.2; Sec. 4.2.1 4th-order FD with three
ghost layers and RK4) and the Brill-Lindquist puncture data the workloads are
defined with.
"""
from __future__ import annotations

import math

import numpy as np

MASTER_SEED = 2505000097

SINH_SPHERICAL, SINH_CYLINDRICAL, SPHERICAL = 0, 1, 2
NGF = 24
GF_NAMES = (
    "hDD00", "hDD01", "hDD02", "hDD11", "hDD12", "hDD22",
    "aDD00", "aDD01", "aDD02", "aDD11", "aDD12", "aDD22",
    "cf", "trK", "lambdaU0", "lambdaU1", "lambdaU2",
    "vetU0", "vetU1", "vetU2", "betU0", "betU1", "betU2", "alpha",
)
# gridfunction groups that are components of one tensor (for error norms)
GF_GROUPS = (tuple(range(0, 6)), tuple(range(6, 12)), (12,), (13,), (14, 15, 16),
             (17, 18, 19), (20, 21, 22), (23,))


def base_spec(coords: int, N, ampl=(10.0, 10.0, 10.0), sinhw=(0.2, 0.2, 0.2), **kw) -> dict:
    spec = dict(coords=int(coords), N=tuple(int(v) for v in N), NG=3, ampl=tuple(float(a) for a in ampl),
                sinhw=tuple(float(w) for w in sinhw), ko_sigma=0.3, eta=2.0, cfl=0.5, wavespeed=1.0,
                enforce_detgb=1)
    spec.update(kw)
    return spec


def sinh_spherical(N, ampl=10.0, w=0.2, **kw) -> dict:
    return base_spec(SINH_SPHERICAL, N, ampl=(ampl, 1.0, 1.0), sinhw=(w, w, w), **kw)


def sinh_cylindrical(N, rho_max=300.0, z_max=300.0, w=0.2, **kw) -> dict:
    return base_spec(SINH_CYLINDRICAL, N, ampl=(rho_max, 1.0, z_max), sinhw=(w, w, w), **kw)


def spherical(N, r_max=7.5, **kw) -> dict:
    return base_spec(SPHERICAL, N, ampl=(r_max, 1.0, 1.0), **kw)


# ---------------------------------------------------------------- configs

def config_single_puncture() -> dict:
    """Single BL puncture M=1 at the origin, SinhSpherical AMPL=10 w=0.2, 64x16x2, 20 RK4 steps."""
    s = sinh_spherical((64, 16, 2))
    s.update(name="single_puncture_sinhsph_64x16x2", masses=(1.0,), positions=((0.0, 0.0, 0.0),),
             perturb_amp=0.0, seed=0, steps=20, h_every=0, psi4_radius=5.0)
    return s


def config_headon() -> dict:
    """Head-on BL binary m=0.5+0.5 at z=+-0.5, SinhCylindrical rho,z in 300, 256x2x512, 2000 RK4 steps."""
    s = sinh_cylindrical((256, 2, 512))
    s.update(name="headon_sinhcyl_256x2x512", masses=(0.5, 0.5), positions=((0.0, 0.0, 0.5), (0.0, 0.0, -0.5)),
             perturb_amp=0.0, seed=0, steps=2000, h_every=100, psi4_radius=100.0)
    return s


def config_headon8() -> dict:
    """The head-on configuration with the production scheme of Sec. 4.1: 8th-order finite differences
    (NG = 5), SSPRK3, Kreiss-Oliger 0.3 on the metric and 0.99 on the gauge gridfunctions.  CFL 0.35:
    on this grid SSPRK3 at CFL 0.5 goes unstable near the rho axis (measured at both orders; RK4,
    whose stability interval on the imaginary axis is wider, is stable at 0.5)."""
    s = config_headon()
    s.update(name="headon8_sinhcyl_256x2x512", NG=5, ko_sigma=[0.3] * 17 + [0.99] * 7, integrator="ssprk3",
             cfl=0.35)
    return s


def config_large3d() -> dict:
    """Single BL puncture + 1e-10 SplitMix64 perturbation of hDD, SinhSpherical 384x192x384, 200 RK4 steps."""
    s = sinh_spherical((384, 192, 384))
    s.update(name="vacuum3d_sinhsph_384x192x384", masses=(1.0,), positions=((0.0, 0.0, 0.0),),
             perturb_amp=1e-10, seed=MASTER_SEED + 3, steps=200, h_every=0, psi4_radius=5.0)
    return s


def config_large3d8() -> dict:
    """The large 3D configuration with the production scheme of Sec. 4.1: 8th-order finite differences
    (NG = 5), SSPRK3 at CFL 0.35 (as the head-on production workload), Kreiss-Oliger 0.3 on the metric and
    0.99 on the gauge gridfunctions; the general (three-dimensional) 8th-order kernel."""
    s = config_large3d()
    s.update(name="vacuum3d8_sinhsph_384x192x384", NG=5, ko_sigma=[0.3] * 17 + [0.99] * 7, integrator="ssprk3",
             cfl=0.35)
    return s


def config_batch(n_runs: int = 64, steps: int = 500, seed: int = MASTER_SEED + 4) -> list[dict]:
    """64 head-on runs: q~U[1,4], d~U[0.5,2], N_rho in {64,96,128,192,256}, N_z=2 N_rho, N_phi=2."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(n_runs):
        q = float(rng.uniform(1.0, 4.0))
        d = float(rng.uniform(0.5, 2.0))
        nrho = int(rng.choice([64, 96, 128, 192, 256]))
        m1, m2 = q / (1.0 + q), 1.0 / (1.0 + q)
        s = sinh_cylindrical((nrho, 2, 2 * nrho))
        s.update(name=f"batch_run{r}", masses=(m1, m2), positions=((0.0, 0.0, d * m2), (0.0, 0.0, -d * m1)),
                 perturb_amp=0.0, seed=0, steps=steps, h_every=0)
        runs.append(s)
    return runs


def config_served(n_requests: int = 64, rate_per_min: float = 20.0, seed: int = MASTER_SEED + 5,
                  t_final: float = 50.0) -> list[dict]:
    """Poisson stream of single-puncture / head-on requests, 1e5..4e6 points, SinhCylindrical grids."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += float(rng.exponential(60.0 / rate_per_min))
        pts = float(math.exp(rng.uniform(math.log(1e5), math.log(4e6))))
        nrho = max(8, int(round(math.sqrt(pts / 4.0))))
        s = sinh_cylindrical((nrho, 2, 2 * nrho))
        if rng.uniform() < 0.5:
            m = float(rng.uniform(0.5, 1.5))
            s.update(masses=(m,), positions=((0.0, 0.0, 0.0),))
        else:
            q = float(rng.uniform(1.0, 4.0)); d = float(rng.uniform(0.5, 2.0))
            m1, m2 = q / (1.0 + q), 1.0 / (1.0 + q)
            s.update(masses=(m1, m2), positions=((0.0, 0.0, d * m2), (0.0, 0.0, -d * m1)))
        s.update(name=f"req{r}", arrival_s=t, t_final=t_final, perturb_amp=0.0, seed=0, h_every=0)
        reqs.append(s)
    return reqs


# ---------------------------------------------------------- random states

_RANGES = {  # (lo, hi) per gridfunction: a generic, well-posed BSSN state
    "hDD": (-0.05, 0.05), "aDD": (-0.1, 0.1), "cf": (0.3, 1.0), "trK": (-0.1, 0.1),
    "lambdaU": (-0.1, 0.1), "vetU": (-0.1, 0.1), "betU": (-0.1, 0.1), "alpha": (0.3, 1.0),
}


def _range_of(name: str):
    for k, v in _RANGES.items():
        if name.startswith(k):
            return v
    raise KeyError(name)


def random_state(n: tuple, seed: int, smooth: bool = False) -> np.ndarray:
    """A (24*T,) FP64 state on a padded grid of shape n=(n0,n1,n2).

    smooth=False: independent uniform values at every point (exercises every
    stencil coefficient).  smooth=True: a few random low-frequency modes of the
    logical indices, within the same ranges.
    """
    rng = np.random.default_rng(seed)
    n0, n1, n2 = n
    T = n0 * n1 * n2
    out = np.empty((NGF, T))
    if smooth:
        i2, i1, i0 = np.meshgrid(np.arange(n2) / n2, np.arange(n1) / n1, np.arange(n0) / n0, indexing="ij")
    for g, name in enumerate(GF_NAMES):
        lo, hi = _range_of(name)
        if not smooth:
            out[g] = rng.uniform(lo, hi, size=T)
        else:
            mid, amp = 0.5 * (lo + hi), 0.5 * (hi - lo)
            f = np.zeros((n2, n1, n0))
            for _ in range(3):
                k = rng.integers(0, 3, size=3)
                ph = rng.uniform(0, 2 * np.pi)
                f += np.cos(2 * np.pi * (k[0] * i0 + k[1] * i1 + k[2] * i2) + ph)
            out[g] = (mid + amp * f / 3.0).reshape(-1)
    return out.reshape(-1)
