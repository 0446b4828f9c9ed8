"""Thin ctypes binding of libnrgpu (include/nr.h).

Argument marshalling only: every step of the evolution runs in the library's
CUDA kernels.  Device buffers handed to the library are torch CUDA tensors
(torch provides device memory and streams, nothing else).  If the compiled
library is missing this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NGF = 24
NR_OK = 0
STATUS = {0: "NR_OK", 1: "NR_EINVAL", 2: "NR_ENOMEM", 3: "NR_ECUDA", 4: "NR_ETIMEOUT", 5: "NR_ENONFINITE",
          6: "NR_EMAP"}
COORDS = {"sinh_spherical": 0, "sinh_cylindrical": 1, "spherical": 2}
INTEGRATORS = {"rk4": 0, "ssprk3": 1}

# every entry point declared in include/nr.h
EXPORTS = (
    "nr_params_default", "nr_grid_create", "nr_grid_destroy", "nr_query", "nr_set_brill_lindquist", "nr_rhs",
    "nr_apply_bcs", "nr_apply_inner_bcs", "nr_rk4_step", "nr_ssprk3_step", "nr_hamiltonian", "nr_momentum",
    "nr_psi4", "nr_psi4_modes", "nr_get_state", "nr_get_state_compact", "nr_set_state_compact", "nr_step_io",
    "nr_set_state",
    "nr_sync", "nr_check_finite", "nr_build_maps", "nr_dt_cfl", "nr_fp64_peak", "nr_hamiltonian_noalloc",
    "nr_batch_create", "nr_batch_destroy", "nr_batch_set_tile", "nr_batch_autotune", "nr_batch_rk4_step", "nr_batch_ssprk3_step",
    "nr_server_create", "nr_server_destroy", "nr_server_set_tile", "nr_server_set_policy", "nr_server_submit",
    "nr_server_advance",
    "nr_server_poll", "nr_server_fetch_state", "nr_server_set_guard", "nr_server_request_error",
    "nr_server_fetch_digest", "nr_server_set_starvation_cap", "nr_server_stats",
    "nr_server_set_prefetch", "nr_state_digest",
    "nr_part_create", "nr_part_destroy", "nr_part_query", "nr_part_set_brill_lindquist", "nr_part_set_state",
    "nr_part_get_state", "nr_part_rk4_step", "nr_part_ssprk3_step", "nr_part_digest", "nr_part_hamiltonian", "nr_part_sync",
    "nr_part_plan_info", "nr_part_plan_boxes", "nr_part_plan_records", "nr_last_error",
)


class NrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class NrParams(ctypes.Structure):
    _fields_ = [
        ("ampl", ctypes.c_double * 3),
        ("sinhw", ctypes.c_double * 3),
        ("ko_sigma", ctypes.c_double * 24),
        ("eta", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("wavespeed", ctypes.c_double * 24),
        ("f_inf", ctypes.c_double * 24),
        ("h_rmin", ctypes.c_double),
        ("h_rmax", ctypes.c_double),
        ("NG", ctypes.c_int),
        ("enforce_detgb", ctypes.c_int),
        ("device", ctypes.c_int),
        ("integrator", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


class NrGridInfo(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int * 3),
        ("n", ctypes.c_int * 3),
        ("T", ctypes.c_int64),
        ("interior", ctypes.c_int64),
        ("n_outer", ctypes.c_int64),
        ("n_inner", ctypes.c_int64),
        ("dt_cfl", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t),
        ("n_inner_stencil", ctypes.c_int64),
        ("launches_per_step", ctypes.c_int),
        ("launches_per_ssprk3_step", ctypes.c_int),
        ("n_state_points", ctypes.c_int64),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libnrgpu.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libnrgpu.so is missing ({path}); run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    P = ctypes.POINTER(NrParams)
    L.nr_params_default.argtypes = [ctypes.c_int, P]
    L.nr_grid_create.argtypes = [ctypes.c_int, ip, P, ctypes.POINTER(vp)]
    L.nr_grid_destroy.argtypes = [vp]
    L.nr_grid_destroy.restype = None
    L.nr_query.argtypes = [vp, ctypes.POINTER(NrGridInfo)]
    L.nr_set_brill_lindquist.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_uint64]
    L.nr_rhs.argtypes = [vp, vp, vp]
    L.nr_apply_bcs.argtypes = [vp, vp, vp]
    L.nr_apply_inner_bcs.argtypes = [vp, vp]
    L.nr_rk4_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.nr_ssprk3_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.nr_hamiltonian.argtypes = [vp, vp, vp, dp, dp]
    L.nr_momentum.argtypes = [vp, vp, vp, dp, dp]
    L.nr_psi4.argtypes = [vp, vp, vp]
    L.nr_psi4_modes.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
    L.nr_get_state.argtypes = [vp, vp, ctypes.c_int]
    L.nr_set_state.argtypes = [vp, vp, ctypes.c_int]
    L.nr_get_state_compact.argtypes = [vp, vp, ctypes.c_int]
    L.nr_set_state_compact.argtypes = [vp, vp, ctypes.c_int]
    L.nr_step_io.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, vp]
    L.nr_sync.argtypes = [vp]
    L.nr_check_finite.argtypes = [vp]
    L.nr_build_maps.argtypes = [ctypes.c_int, ip, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int32)]
    L.nr_dt_cfl.argtypes = [ctypes.c_int, ip, P, dp]
    L.nr_fp64_peak.argtypes = [ctypes.c_int, dp]
    L.nr_hamiltonian_noalloc.argtypes = [ctypes.c_int, ip, P, vp, vp, dp, dp]
    L.nr_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
    L.nr_batch_destroy.argtypes = [vp]
    L.nr_batch_destroy.restype = None
    L.nr_batch_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.nr_batch_autotune.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp]
    L.nr_batch_rk4_step.argtypes = [vp, dp, ctypes.c_int]
    L.nr_batch_ssprk3_step.argtypes = [vp, dp, ctypes.c_int]
    L.nr_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.nr_server_destroy.argtypes = [vp]
    L.nr_server_destroy.restype = None
    L.nr_server_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.nr_server_set_policy.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
    L.nr_server_submit.argtypes = [vp, ctypes.c_int, ip, P, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int64)]
    L.nr_server_advance.argtypes = [vp, ctypes.c_int, ip, ip]
    L.nr_server_poll.argtypes = [vp, ctypes.c_int64, ip, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64), dp, dp]
    L.nr_server_fetch_state.argtypes = [vp, ctypes.c_int64, dp, ctypes.c_size_t]
    L.nr_server_set_guard.argtypes = [vp, ctypes.c_int]
    L.nr_server_set_starvation_cap.argtypes = [vp, ctypes.c_double]
    L.nr_server_stats.argtypes = [vp, dp]
    L.nr_server_set_prefetch.argtypes = [vp, ctypes.c_int]
    L.nr_server_request_error.argtypes = [vp, ctypes.c_int64, ip]
    L.nr_server_fetch_digest.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
    L.nr_state_digest.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.nr_part_create.argtypes = [ctypes.c_int, ip, P, ip, ctypes.POINTER(vp)]
    L.nr_part_destroy.argtypes = [vp]
    L.nr_part_destroy.restype = None
    L.nr_part_query.argtypes = [vp, i64p, i64p, dp, ctypes.POINTER(ctypes.c_size_t)]
    L.nr_part_set_brill_lindquist.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_uint64]
    L.nr_part_set_state.argtypes = [vp, vp, ctypes.c_int]
    L.nr_part_get_state.argtypes = [vp, vp, ctypes.c_int]
    L.nr_part_rk4_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.nr_part_ssprk3_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.nr_part_digest.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    L.nr_part_hamiltonian.argtypes = [vp, dp, dp]
    L.nr_part_sync.argtypes = [vp]
    L.nr_part_plan_info.argtypes = [ctypes.c_int, ip, ctypes.c_int, ip, i64p, i64p]
    L.nr_part_plan_boxes.argtypes = [ctypes.c_int, ip, ctypes.c_int, ip, i32p]
    L.nr_part_plan_records.argtypes = [ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_int, i32p, ctypes.c_int64]
    L.nr_last_error.argtypes = []
    L.nr_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int) -> None:
    if rc != NR_OK:
        raise NrError(rc, lib().nr_last_error().decode())


def _ptr(t) -> int:
    """device pointer of a contiguous float64 torch tensor (or an int address)"""
    if isinstance(t, int):
        return t
    assert t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous()
    return t.data_ptr()


def make_params(spec: dict, stream=None, device: int = 0) -> NrParams:
    """nr_params from a workload dict (see workloads.py)."""
    p = NrParams()
    _check(lib().nr_params_default(int(spec["coords"]), ctypes.byref(p)))
    for d in range(3):
        p.ampl[d] = float(spec["ampl"][d])
        p.sinhw[d] = float(spec["sinhw"][d])
    ko = spec.get("ko_sigma", 0.3)
    ko = [float(ko)] * NGF if np.isscalar(ko) else [float(v) for v in ko]
    ws = spec.get("wavespeed", 1.0)
    ws = [float(ws)] * NGF if np.isscalar(ws) else [float(v) for v in ws]
    for g in range(NGF):
        p.ko_sigma[g] = ko[g]
        p.wavespeed[g] = ws[g]
    if spec.get("f_inf") is not None:
        for g in range(NGF):
            p.f_inf[g] = float(spec["f_inf"][g])
    p.eta = float(spec.get("eta", 2.0))
    p.cfl = float(spec.get("cfl", 0.5))
    p.h_rmin = float(spec.get("h_rmin", 0.0))
    p.h_rmax = float(spec.get("h_rmax", 1e300))
    p.NG = int(spec.get("NG", 3))
    p.enforce_detgb = int(spec.get("enforce_detgb", 1))
    p.integrator = INTEGRATORS[spec.get("integrator", "rk4")]
    p.device = int(device)
    p.stream = stream
    return p


def build_maps(coords: int, N, NG: int = 3):
    """Host-only closed-form boundary maps: (src, parity[T,10], cls)."""
    n = [int(v) + 2 * NG for v in N]
    T = n[0] * n[1] * n[2]
    src = np.zeros(T, dtype=np.int32)
    par = np.zeros(10 * T, dtype=np.int8)
    cls = np.zeros(T, dtype=np.int32)
    Nx = (ctypes.c_int * 3)(*[int(v) for v in N])
    _check(lib().nr_build_maps(int(coords), Nx, NG, src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               par.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                               cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return src, par.reshape(T, 10), cls


def dt_cfl(spec: dict) -> float:
    p = make_params(spec)
    Nx = (ctypes.c_int * 3)(*[int(v) for v in spec["N"]])
    out = ctypes.c_double()
    _check(lib().nr_dt_cfl(int(spec["coords"]), Nx, ctypes.byref(p), ctypes.byref(out)))
    return out.value


def fp64_peak(device: int = 0) -> float:
    """measured FP64 FMA throughput of the device in FLOP/s"""
    out = ctypes.c_double()
    _check(lib().nr_fp64_peak(int(device), ctypes.byref(out)))
    return out.value


def hamiltonian_noalloc(spec: dict, y, H=None, stream=None, device: int = 0):
    """nr_hamiltonian_noalloc: Hamiltonian constraint of a caller-owned state without any allocation;
    returns (l2, linf)."""
    p = make_params(spec, stream=stream, device=device)
    Nx = (ctypes.c_int * 3)(*[int(v) for v in spec["N"]])
    l2, linf = ctypes.c_double(), ctypes.c_double()
    _check(lib().nr_hamiltonian_noalloc(int(spec["coords"]), Nx, ctypes.byref(p), _ptr(y),
                                        None if H is None else _ptr(H), ctypes.byref(l2), ctypes.byref(linf)))
    return l2.value, linf.value


class Grid:
    """One nr_grid (library-owned state on the GPU)."""

    def __init__(self, spec: dict, stream=None, device: int = 0):
        self.spec = dict(spec)
        self.params = make_params(spec, stream=stream, device=device)
        h = ctypes.c_void_p()
        Nx = (ctypes.c_int * 3)(*[int(v) for v in spec["N"]])
        _check(lib().nr_grid_create(int(spec["coords"]), Nx, ctypes.byref(self.params), ctypes.byref(h)))
        self.h = h
        info = NrGridInfo()
        _check(lib().nr_query(self.h, ctypes.byref(info)))
        self.info = info
        self.T = int(info.T)
        self.n = tuple(int(v) for v in info.n)
        self.N = tuple(int(v) for v in info.N)
        self.interior = int(info.interior)
        self.dt_cfl = float(info.dt_cfl)

    def close(self) -> None:
        if self.h:
            lib().nr_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_brill_lindquist(self, masses, positions, perturb_amp: float = 0.0, seed: int = 0) -> None:
        m = np.ascontiguousarray(masses, dtype=np.float64)
        x = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1)
        _check(lib().nr_set_brill_lindquist(self.h, len(m), m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(perturb_amp),
                                            ctypes.c_uint64(int(seed))))

    def rhs(self, y, out) -> None:
        _check(lib().nr_rhs(self.h, _ptr(y), _ptr(out)))

    def apply_bcs(self, y, rhs) -> None:
        _check(lib().nr_apply_bcs(self.h, _ptr(y), _ptr(rhs)))

    def apply_inner_bcs(self, gfs) -> None:
        _check(lib().nr_apply_inner_bcs(self.h, _ptr(gfs)))

    def rk4_step(self, dt: float, nsteps: int = 1) -> None:
        _check(lib().nr_rk4_step(self.h, float(dt), int(nsteps)))

    def ssprk3_step(self, dt: float, nsteps: int = 1) -> None:
        _check(lib().nr_ssprk3_step(self.h, float(dt), int(nsteps)))

    def hamiltonian(self, y=None, H=None, norms: bool = True):
        """(l2, linf) of H; norms=False skips the norms' device-to-host read (no synchronisation)."""
        l2, linf = ctypes.c_double(), ctypes.c_double()
        _check(lib().nr_hamiltonian(self.h, None if y is None else _ptr(y), None if H is None else _ptr(H),
                                    ctypes.byref(l2) if norms else None, ctypes.byref(linf) if norms else None))
        return (l2.value, linf.value) if norms else None

    def psi4(self, out, y=None) -> None:
        """psi4 (2*T doubles on the device: re, im) of y (default: the grid-owned state)."""
        _check(lib().nr_psi4(self.h, None if y is None else _ptr(y), _ptr(out)))

    def psi4_modes(self, Rext: float, ntheta: int = 24, nphi: int = 48, lmax: int = 8, y=None) -> np.ndarray:
        """Complex C_lm, l = 2..lmax, m = -l..l."""
        nm = sum(2 * l + 1 for l in range(2, lmax + 1))
        out = np.zeros(2 * nm)
        _check(lib().nr_psi4_modes(self.h, None if y is None else _ptr(y), float(Rext), int(ntheta), int(nphi),
                                   int(lmax), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out[0::2] + 1j * out[1::2]

    def momentum(self, y=None, M=None, norms: bool = True):
        """(l2, linf) of |M|; norms=False skips the norms' device-to-host read (no synchronisation)."""
        l2, linf = ctypes.c_double(), ctypes.c_double()
        _check(lib().nr_momentum(self.h, None if y is None else _ptr(y), None if M is None else _ptr(M),
                                 ctypes.byref(l2) if norms else None, ctypes.byref(linf) if norms else None))
        return (l2.value, linf.value) if norms else None

    def get_state(self, dst, to_host: bool) -> None:
        addr = dst.ctypes.data if isinstance(dst, np.ndarray) else (dst.data_ptr() if not isinstance(dst, int) else dst)
        _check(lib().nr_get_state(self.h, addr, int(bool(to_host))))

    def set_state(self, src, from_host: bool) -> None:
        addr = src.ctypes.data if isinstance(src, np.ndarray) else (src.data_ptr() if not isinstance(src, int) else src)
        _check(lib().nr_set_state(self.h, addr, int(bool(from_host))))

    def get_state_compact(self, dst, to_host: bool) -> None:
        """24 x info.n_state_points doubles: the state at the interior and pure outer points."""
        addr = dst.ctypes.data if isinstance(dst, np.ndarray) else (dst.data_ptr() if not isinstance(dst, int) else dst)
        _check(lib().nr_get_state_compact(self.h, addr, int(bool(to_host))))

    def set_state_compact(self, src, from_host: bool) -> None:
        addr = src.ctypes.data if isinstance(src, np.ndarray) else (src.data_ptr() if not isinstance(src, int) else src)
        _check(lib().nr_set_state_compact(self.h, addr, int(bool(from_host))))

    def step_io(self, dt: float, nsteps: int = 1, host_in=None, host_out=None, integrator: str = "rk4") -> None:
        """nr_step_io: compact state in from host_in, nsteps steps, compact state out to host_out
        (numpy arrays, pinned torch CPU tensors or raw addresses; None skips)."""
        def addr(a):
            if a is None or isinstance(a, int):
                return a
            return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()
        _check(lib().nr_step_io(self.h, INTEGRATORS[integrator], float(dt), int(nsteps), addr(host_in),
                                addr(host_out)))

    def sync(self) -> None:
        _check(lib().nr_sync(self.h))

    def digest(self, y=None) -> int:
        """nr_state_digest of y (default: the grid-owned state)."""
        out = ctypes.c_uint64()
        _check(lib().nr_state_digest(self.h, None if y is None else _ptr(y), ctypes.byref(out)))
        return out.value

    def check_finite(self) -> None:
        _check(lib().nr_check_finite(self.h))


class Batch:
    """nr_batch over a list of Grid objects (which must outlive it)."""

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g.h.value for g in self.grids])
        h = ctypes.c_void_p()
        _check(lib().nr_batch_create(arr, len(self.grids), ctypes.byref(h)))
        self.h = h

    def close(self) -> None:
        if self.h:
            lib().nr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dts(self, dts):
        a = np.ascontiguousarray(dts, dtype=np.float64)
        assert a.size == len(self.grids)
        return a

    def set_tile(self, tx: int, ty: int) -> None:
        _check(lib().nr_batch_set_tile(self.h, int(tx), int(ty)))

    def autotune(self, dts):
        a = self._dts(dts)
        tx, ty, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().nr_batch_autotune(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(tx),
                                       ctypes.byref(ty), ctypes.byref(ms)))
        return tx.value, ty.value, ms.value

    def rk4_step(self, dts, nsteps: int = 1) -> None:
        a = self._dts(dts)
        _check(lib().nr_batch_rk4_step(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nsteps)))

    def ssprk3_step(self, dts, nsteps: int = 1) -> None:
        a = self._dts(dts)
        _check(lib().nr_batch_ssprk3_step(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nsteps)))


SERVE_FIFO, SERVE_SRPT = 0, 1


class Server:
    """nr_server: continuous batching of evolution requests on one device."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, device: int = 0, stream=None):
        h = ctypes.c_void_p()
        _check(lib().nr_server_create(int(hbm_budget_bytes), int(max_slots), int(device), stream, ctypes.byref(h)))
        self.h = h
        self.device = device

    def close(self) -> None:
        if self.h:
            lib().nr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile(self, tx: int, ty: int) -> None:
        _check(lib().nr_server_set_tile(self.h, int(tx), int(ty)))

    def set_policy(self, policy: str, max_batch_points: int = 0) -> None:
        """policy "fifo" or "srpt"; max_batch_points caps the interior points advanced together (0: no cap)."""
        code = {"fifo": SERVE_FIFO, "srpt": SERVE_SRPT}.get(policy, -1)
        _check(lib().nr_server_set_policy(self.h, code, int(max_batch_points)))

    def set_guard(self, every_steps: int) -> None:
        """non-finite check of the advanced requests every every_steps steps (0: off)"""
        _check(lib().nr_server_set_guard(self.h, int(every_steps)))

    def set_starvation_cap(self, seconds: float) -> None:
        """SRPT: requests submitted more than `seconds` ago go first (0: off)"""
        _check(lib().nr_server_set_starvation_cap(self.h, float(seconds)))

    def set_prefetch(self, depth: int) -> None:
        """host-side set-ups of the next `depth` queued requests computed ahead (0: at admission)"""
        _check(lib().nr_server_set_prefetch(self.h, int(depth)))

    def stats(self) -> dict:
        v = (ctypes.c_double * 9)()
        _check(lib().nr_server_stats(self.h, v))
        keys = ("chunks", "rebuilds", "admitted", "retired", "admit_s", "retire_s", "rebuild_s", "fence_s",
                "enqueue_s")
        return dict(zip(keys, list(v)))

    def request_error(self, rid: int) -> int:
        code = ctypes.c_int()
        _check(lib().nr_server_request_error(self.h, int(rid), ctypes.byref(code)))
        return code.value

    def fetch_digest(self, rid: int) -> int:
        out = ctypes.c_uint64()
        _check(lib().nr_server_fetch_digest(self.h, int(rid), ctypes.byref(out)))
        return out.value

    def submit(self, spec: dict, t_final: float, keep_state: bool = False, keep_digest: bool = False) -> int:
        p = make_params(spec, device=self.device)
        Nx = (ctypes.c_int * 3)(*[int(v) for v in spec["N"]])
        m = np.ascontiguousarray(spec["masses"], dtype=np.float64)
        x = np.ascontiguousarray(spec["positions"], dtype=np.float64).reshape(-1)
        rid = ctypes.c_int64()
        _check(lib().nr_server_submit(self.h, int(spec["coords"]), Nx, ctypes.byref(p), len(m),
                                      m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(t_final),
                                      int(bool(keep_state)) | (2 if keep_digest else 0), ctypes.byref(rid)))
        return rid.value

    def advance(self, nsteps: int):
        nr, nq = ctypes.c_int(), ctypes.c_int()
        _check(lib().nr_server_advance(self.h, int(nsteps), ctypes.byref(nr), ctypes.byref(nq)))
        return nr.value, nq.value

    def poll(self, rid: int) -> dict:
        st, sd, stt = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        l2, linf = ctypes.c_double(), ctypes.c_double()
        _check(lib().nr_server_poll(self.h, int(rid), ctypes.byref(st), ctypes.byref(sd), ctypes.byref(stt),
                                    ctypes.byref(l2), ctypes.byref(linf)))
        return {"status": st.value, "steps_done": sd.value, "steps_total": stt.value, "l2": l2.value,
                "linf": linf.value}

    def fetch_state(self, rid: int, size: int) -> np.ndarray:
        out = np.empty(size)
        _check(lib().nr_server_fetch_state(self.h, int(rid), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           size))
        return out


def part_plan(coords: int, N, NG: int, parts):
    """Host-only plan of a grid cut into partitions: (boxes [nparts, 15], records per phase [n, 5])."""
    Nx = (ctypes.c_int * 3)(*[int(v) for v in N])
    Px = (ctypes.c_int * 3)(*[int(v) for v in parts])
    npart = ctypes.c_int64()
    counts = (ctypes.c_int64 * 4)()
    _check(lib().nr_part_plan_info(int(coords), Nx, int(NG), Px, ctypes.byref(npart), counts))
    boxes = np.zeros((npart.value, 15), dtype=np.int32)
    _check(lib().nr_part_plan_boxes(int(coords), Nx, int(NG), Px, boxes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    recs = []
    for ph in range(4):
        r = np.zeros((max(1, counts[ph]), 5), dtype=np.int32)
        _check(lib().nr_part_plan_records(int(coords), Nx, int(NG), Px, ph, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          int(counts[ph])))
        recs.append(r[:counts[ph]])
    return boxes, recs


class PartGrid:
    """nr_part: one grid cut into partitions (library-owned states on one GPU)."""

    def __init__(self, spec: dict, parts, stream=None, device: int = 0):
        self.spec = dict(spec)
        self.params = make_params(spec, stream=stream, device=device)
        h = ctypes.c_void_p()
        Nx = (ctypes.c_int * 3)(*[int(v) for v in spec["N"]])
        Px = (ctypes.c_int * 3)(*[int(v) for v in parts])
        _check(lib().nr_part_create(int(spec["coords"]), Nx, ctypes.byref(self.params), Px, ctypes.byref(h)))
        self.h = h
        NG = int(spec.get("NG", 3))
        self.n = tuple(int(v) + 2 * NG for v in spec["N"])
        self.T = self.n[0] * self.n[1] * self.n[2]
        npart, dt, nbytes = ctypes.c_int64(), ctypes.c_double(), ctypes.c_size_t()
        msgs = (ctypes.c_int64 * 4)()
        _check(lib().nr_part_query(self.h, ctypes.byref(npart), msgs, ctypes.byref(dt), ctypes.byref(nbytes)))
        self.nparts, self.messages, self.dt_cfl, self.device_bytes = npart.value, list(msgs), dt.value, nbytes.value

    def close(self) -> None:
        if self.h:
            lib().nr_part_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_brill_lindquist(self, masses, positions, perturb_amp: float = 0.0, seed: int = 0) -> None:
        m = np.ascontiguousarray(masses, dtype=np.float64)
        x = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1)
        _check(lib().nr_part_set_brill_lindquist(self.h, len(m), m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(perturb_amp),
                                                 ctypes.c_uint64(int(seed))))

    def set_state(self, src, from_host: bool) -> None:
        addr = src.ctypes.data if isinstance(src, np.ndarray) else (src.data_ptr() if not isinstance(src, int) else src)
        _check(lib().nr_part_set_state(self.h, addr, int(bool(from_host))))

    def get_state(self, dst, to_host: bool) -> None:
        addr = dst.ctypes.data if isinstance(dst, np.ndarray) else (dst.data_ptr() if not isinstance(dst, int) else dst)
        _check(lib().nr_part_get_state(self.h, addr, int(bool(to_host))))

    def rk4_step(self, dt: float, nsteps: int = 1) -> None:
        _check(lib().nr_part_rk4_step(self.h, float(dt), int(nsteps)))

    def ssprk3_step(self, dt: float, nsteps: int = 1) -> None:
        _check(lib().nr_part_ssprk3_step(self.h, float(dt), int(nsteps)))

    def digest(self) -> int:
        out = ctypes.c_uint64()
        _check(lib().nr_part_digest(self.h, ctypes.byref(out)))
        return out.value

    def hamiltonian(self):
        """(l2, linf) of the Hamiltonian constraint over the radius band of the spec"""
        l2, linf = ctypes.c_double(), ctypes.c_double()
        _check(lib().nr_part_hamiltonian(self.h, ctypes.byref(l2), ctypes.byref(linf)))
        return l2.value, linf.value

    def sync(self) -> None:
        _check(lib().nr_part_sync(self.h))
