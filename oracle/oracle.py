"""ctypes binding of the CPU reference oracle (nr_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by bench.py's CPU-baseline / reference arm.  The product path never imports
this module.  The oracle follows arXiv 2505.00097 Sec. 2 (BSSN equations,
tensor rescaling), Sec. 3 (grid, stencils, boundary classes) and the RK4
integrator of Sec. 4.2.1; see the header comment of nr_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nr_oracle.c")
_HDR = os.path.join(_HERE, "nr_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

SINH_SPHERICAL, SINH_CYLINDRICAL, SPHERICAL = 0, 1, 2
NGF = 24


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("coords", ctypes.c_int),
        ("N", ctypes.c_int * 3),
        ("NG", ctypes.c_int),
        ("enforce_detgb", ctypes.c_int),
        ("ampl", ctypes.c_double * 3),
        ("sinhw", ctypes.c_double * 3),
        ("ko_sigma", ctypes.c_double * 24),
        ("eta", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("wavespeed", ctypes.c_double * 24),
        ("f_inf", ctypes.c_double * 24),
        ("nthreads", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain FP64, no fast-math, no contraction)."""
    with _lock:
        os.makedirs(_OUT_DIR, exist_ok=True)
        up_to_date = (
            os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        )
        if force or not up_to_date:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fno-fast-math", "-ffp-contract=off",
                   "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OrcParams)
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        L.orc_sizes.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
        L.orc_sizes.restype = ctypes.c_long
        L.orc_xx.argtypes = [P, ctypes.c_int, ctypes.c_int]
        L.orc_xx.restype = ctypes.c_double
        L.orc_cart.argtypes = [P, ctypes.c_long, dp]
        L.orc_cart_all.argtypes = [P, dp]
        L.orc_refmetric.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
        for name in ("orc_build_map", "orc_build_map_bruteforce"):
            getattr(L, name).argtypes = [P, i32p, i8p, i32p]
            getattr(L, name).restype = ctypes.c_int
        L.orc_dt.argtypes = [P]
        L.orc_dt.restype = ctypes.c_double
        L.orc_brill_lindquist.argtypes = [P, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_uint64, dp]
        L.orc_brill_lindquist.restype = ctypes.c_int
        L.orc_rhs.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_int]
        L.orc_outer_bc.argtypes = [P, dp, dp]
        L.orc_inner_bc.argtypes = [P, dp]
        L.orc_inner_bc.restype = ctypes.c_int
        L.orc_full_rhs.argtypes = [P, dp, dp]
        L.orc_full_rhs.restype = ctypes.c_int
        L.orc_enforce_detgb.argtypes = [P, dp]
        L.orc_rk4_step.argtypes = [P, dp, ctypes.c_double, ctypes.c_int]
        L.orc_rk4_step.restype = ctypes.c_int
        L.orc_hamiltonian.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp,
                                      ctypes.POINTER(ctypes.c_long)]
        L.orc_momentum.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp,
                                   ctypes.POINTER(ctypes.c_long)]
        L.orc_psi4.argtypes = [P, dp, dp, dp, dp]
        L.orc_sylm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_psi4_modes.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.orc_psi4_modes.restype = ctypes.c_int
        L.orc_rk4_generic.argtypes = [ctypes.c_long, dp, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_ssprk3_generic.argtypes = [ctypes.c_long, dp, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_ssprk3_step.argtypes = [P, dp, ctypes.c_double, ctypes.c_int]
        L.orc_ssprk3_step.restype = ctypes.c_int
        L.orc_fd_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.orc_fd_weights.restype = ctypes.c_int
        for name in ("orc_d1", "orc_d2", "orc_ko6"):
            getattr(L, name).restype = ctypes.c_double
        L.orc_d1.argtypes = [dp, ctypes.c_long, ctypes.c_double]
        L.orc_d2.argtypes = [dp, ctypes.c_long, ctypes.c_double]
        L.orc_d11.argtypes = [dp, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double]
        L.orc_d11.restype = ctypes.c_double
        L.orc_dup.argtypes = [dp, ctypes.c_long, ctypes.c_double, ctypes.c_int]
        L.orc_dup.restype = ctypes.c_double
        L.orc_ko6.argtypes = [dp, ctypes.c_long]
        L.orc_d1_onesided.argtypes = [dp, ctypes.c_long, ctypes.c_double, ctypes.c_int]
        L.orc_d1_onesided.restype = ctypes.c_double
        L.orc_splitmix_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_splitmix_uniform.restype = ctypes.c_double
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One grid of the oracle.  `spec` is a plain dict of grid/physics numbers."""

    def __init__(self, spec: dict):
        self.spec = dict(spec)
        p = OrcParams()
        p.coords = int(spec["coords"])
        for d in range(3):
            p.N[d] = int(spec["N"][d])
            p.ampl[d] = float(spec["ampl"][d])
            p.sinhw[d] = float(spec["sinhw"][d])
        p.NG = int(spec.get("NG", 3))
        p.enforce_detgb = int(spec.get("enforce_detgb", 1))
        ko = spec.get("ko_sigma", 0.3)
        ko = [float(ko)] * NGF if np.isscalar(ko) else [float(v) for v in ko]
        ws = spec.get("wavespeed", 1.0)
        ws = [float(ws)] * NGF if np.isscalar(ws) else [float(v) for v in ws]
        for g in range(NGF):
            p.ko_sigma[g] = ko[g]
            p.wavespeed[g] = ws[g]
            p.f_inf[g] = 0.0
        finf = spec.get("f_inf")
        if finf is None:
            p.f_inf[12] = 1.0   # W
            p.f_inf[23] = 1.0   # alpha
        else:
            for g in range(NGF):
                p.f_inf[g] = float(finf[g])
        p.eta = float(spec.get("eta", 2.0))
        p.cfl = float(spec.get("cfl", 0.5))
        p.nthreads = int(spec.get("nthreads", 0))
        self.p = p
        self.L = lib()
        n = (ctypes.c_int * 3)()
        self.T = int(self.L.orc_sizes(ctypes.byref(p), n))
        self.n = tuple(int(v) for v in n)
        self.NG = p.NG

    # ---- geometry
    @property
    def shape(self):
        """(24, n2, n1, n0) view shape of a gridfunction set."""
        return (NGF, self.n[2], self.n[1], self.n[0])

    def xx(self, d: int) -> np.ndarray:
        return np.array([self.L.orc_xx(ctypes.byref(self.p), d, i) for i in range(self.n[d])])

    def cart(self) -> np.ndarray:
        out = np.empty((self.T, 3))
        self.L.orc_cart_all(ctypes.byref(self.p), _dp(out.reshape(-1)))
        return out

    def refmetric(self, xx):
        xx = np.ascontiguousarray(xx, dtype=np.float64)
        S = np.zeros(3)
        g = np.zeros((3, 3)); dg = np.zeros((3, 3, 3)); ddg = np.zeros((3, 3, 3, 3))
        G = np.zeros((3, 3, 3)); dG = np.zeros((3, 3, 3, 3))
        self.L.orc_refmetric(ctypes.byref(self.p), _dp(xx), _dp(S), _dp(g), _dp(dg), _dp(ddg), _dp(G), _dp(dG))
        return S, g, dg, ddg, G, dG

    def build_map(self, brute: bool = False):
        src = np.zeros(self.T, dtype=np.int32)
        par = np.zeros(self.T * 10, dtype=np.int8)
        cls = np.zeros(self.T, dtype=np.int32)
        fn = self.L.orc_build_map_bruteforce if brute else self.L.orc_build_map
        rc = fn(ctypes.byref(self.p), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                par.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return rc, src, par.reshape(self.T, 10), cls

    def dt(self) -> float:
        return float(self.L.orc_dt(ctypes.byref(self.p)))

    # ---- data
    def zeros(self) -> np.ndarray:
        return np.zeros(NGF * self.T)

    def brill_lindquist(self, masses, positions, perturb_amp=0.0, seed=0) -> np.ndarray:
        m = np.ascontiguousarray(masses, dtype=np.float64)
        x = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1)
        y = self.zeros()
        rc = self.L.orc_brill_lindquist(ctypes.byref(self.p), len(m), _dp(m), _dp(x), float(perturb_amp),
                                        ctypes.c_uint64(int(seed)), _dp(y))
        if rc:
            raise ValueError(f"orc_brill_lindquist failed ({rc})")
        return y

    def rhs(self, y: np.ndarray, k_lo: int = 0, k_hi: int | None = None) -> np.ndarray:
        out = np.zeros_like(y)
        self.L.orc_rhs(ctypes.byref(self.p), _dp(y), _dp(out), int(k_lo), int(self.p.N[2] if k_hi is None else k_hi))
        return out

    def outer_bc(self, y: np.ndarray, rhs: np.ndarray) -> None:
        self.L.orc_outer_bc(ctypes.byref(self.p), _dp(y), _dp(rhs))

    def inner_bc(self, y: np.ndarray) -> None:
        if self.L.orc_inner_bc(ctypes.byref(self.p), _dp(y)):
            raise ValueError("inner boundary map failed")

    def full_rhs(self, y: np.ndarray) -> np.ndarray:
        out = np.zeros_like(y)
        self.L.orc_full_rhs(ctypes.byref(self.p), _dp(y), _dp(out))
        return out

    def enforce_detgb(self, y: np.ndarray) -> None:
        self.L.orc_enforce_detgb(ctypes.byref(self.p), _dp(y))

    def rk4(self, y: np.ndarray, dt: float, nsteps: int) -> None:
        if self.L.orc_rk4_step(ctypes.byref(self.p), _dp(y), float(dt), int(nsteps)):
            raise ValueError("inner boundary map failed")

    def ssprk3(self, y: np.ndarray, dt: float, nsteps: int) -> None:
        if self.L.orc_ssprk3_step(ctypes.byref(self.p), _dp(y), float(dt), int(nsteps)):
            raise ValueError("inner boundary map failed")

    def hamiltonian(self, y: np.ndarray, rmin: float = 0.0, rmax: float = 1e300):
        H = np.zeros(self.T)
        l2 = ctypes.c_double(); linf = ctypes.c_double(); cnt = ctypes.c_long()
        self.L.orc_hamiltonian(ctypes.byref(self.p), _dp(y), _dp(H), float(rmin), float(rmax),
                               ctypes.byref(l2), ctypes.byref(linf), ctypes.byref(cnt))
        return H, l2.value, linf.value, cnt.value

    def momentum(self, y: np.ndarray, rmin: float = 0.0, rmax: float = 1e300):
        """Eq. Mconstraint: rescaled S_i M^i (3, T), |M| (T), and the L2 / Linf norms of |M| over the band."""
        M = np.zeros(3 * self.T)
        mag = np.zeros(self.T)
        l2 = ctypes.c_double(); linf = ctypes.c_double(); cnt = ctypes.c_long()
        self.L.orc_momentum(ctypes.byref(self.p), _dp(y), _dp(M), _dp(mag), float(rmin), float(rmax),
                            ctypes.byref(l2), ctypes.byref(linf), ctypes.byref(cnt))
        return M.reshape(3, self.T), mag, l2.value, linf.value, cnt.value

    def psi4(self, y: np.ndarray):
        """Weyl scalar psi4 (2, T) and E, B in the tetrad (6, T each) at interior points."""
        out = np.zeros(2 * self.T)
        E = np.zeros(6 * self.T)
        Bm = np.zeros(6 * self.T)
        self.L.orc_psi4(ctypes.byref(self.p), _dp(y), _dp(out), _dp(E), _dp(Bm))
        return out.reshape(2, self.T), E.reshape(6, self.T), Bm.reshape(6, self.T)

    def psi4_modes(self, psi4: np.ndarray, Rext: float, ntheta: int = 24, nphi: int = 48, lmax: int = 8):
        """Complex modes C_lm, l = 2..lmax, m = -l..l, of a psi4 field (2, T) on the sphere Rext."""
        nm = sum(2 * l + 1 for l in range(2, lmax + 1))
        out = np.zeros(2 * nm)
        f = np.ascontiguousarray(psi4, dtype=np.float64).reshape(-1)
        if self.L.orc_psi4_modes(ctypes.byref(self.p), _dp(f), float(Rext), int(ntheta), int(nphi), int(lmax), _dp(out)):
            raise ValueError("sphere outside the grid or map failed")
        return out[0::2] + 1j * out[1::2]

    def interior_mask(self) -> np.ndarray:
        NG = self.NG
        m = np.zeros(self.n[::-1], dtype=bool)
        m[NG:self.n[2] - NG, NG:self.n[1] - NG, NG:self.n[0] - NG] = True
        return m.reshape(-1)


RHS_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))


def rk4_generic(y: np.ndarray, dt: float, f) -> None:
    """Run one classic RK4 step of the oracle's integrator on y' = f(y)."""
    n = y.size

    def cb(_ctx, yp, kp):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        kk = np.ctypeslib.as_array(kp, shape=(n,))
        kk[:] = f(yy.copy())

    fn = RHS_FN(cb)
    lib().orc_rk4_generic(n, _dp(y), float(dt), ctypes.cast(fn, ctypes.c_void_p), None)


def ssprk3_generic(y: np.ndarray, dt: float, f) -> None:
    """Run one SSPRK3 step of the oracle's integrator on y' = f(y)."""
    n = y.size

    def cb(_ctx, yp, kp):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        kk = np.ctypeslib.as_array(kp, shape=(n,))
        kk[:] = f(yy.copy())

    fn = RHS_FN(cb)
    lib().orc_ssprk3_generic(n, _dp(y), float(dt), ctypes.cast(fn, ctypes.c_void_p), None)


def fd_weights(NG: int, which: int, a: int = 0) -> np.ndarray:
    """Weights of the oracle's order-2(NG-1) stencils (see orc_fd_weights)."""
    w = np.zeros(32)
    n = lib().orc_fd_weights(int(NG), int(which), int(a), _dp(w))
    if n == 0:
        raise ValueError("no such stencil")
    return w[:n].copy()


def sylm(s: int, l: int, m: int, th: float, ph: float) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_sylm(int(s), int(l), int(m), float(th), float(ph), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def threads_used(spec: dict) -> int:
    n = int(spec.get("nthreads", 0))
    return n if n > 0 else (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
