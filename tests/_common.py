"""Shared helpers of the test suite (comparison norms, library build)."""
import numpy as np

from paper_2505_00097_gb300 import workloads as W


def group_errors(got: np.ndarray, ref: np.ndarray, T: int, mask: np.ndarray | None = None):
    """Per gridfunction: max |got - ref| over the masked points divided by the largest |ref|
    of the tensor the gridfunction is a component of (components of one tensor mix under the
    frame changes that separate the two evaluations, so their rounding scales with the whole
    tensor).  A tensor that is identically zero in ref must be exactly zero in got."""
    errs = {}
    for grp in W.GF_GROUPS:
        sl = [slice(g * T, (g + 1) * T) for g in grp]
        r = [ref[s] if mask is None else ref[s][mask] for s in sl]
        q = [got[s] if mask is None else got[s][mask] for s in sl]
        scale = max(float(np.abs(x).max()) if x.size else 0.0 for x in r)
        for g, rr, qq in zip(grp, r, q):
            d = float(np.abs(qq - rr).max()) if rr.size else 0.0
            errs[W.GF_NAMES[g]] = d / scale if scale > 0 else (0.0 if d == 0.0 else np.inf)
    return errs


def assert_close(got, ref, T, tol, mask=None, what=""):
    errs = group_errors(got, ref, T, mask)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what}: relative errors above {tol}: {bad}"
    return max(errs.values())


def axisymmetry_zero_gfs(coords: int):
    """Gridfunctions that vanish exactly under axisymmetry (a two-point azimuth with
    azimuth-independent data): the azimuthal component of each vector and the components of
    each symmetric tensor with exactly one azimuthal index.  The azimuthal axis is 1 for the
    cylindrical-like family, 2 for the spherical-like ones."""
    ax = 1 if coords == W.SINH_CYLINDRICAL else 2
    sym = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    one = [s for s, (i, j) in enumerate(sym) if (i == ax) != (j == ax)]
    return sorted([s for s in one] + [6 + s for s in one] + [14 + ax, 17 + ax, 20 + ax])


def assert_axisymmetry_zeros(got, ref, T, coords, what=""):
    """The components that vanish by axisymmetry are exactly 0.0 in the kernels' result (the
    discrete scheme keeps them zero: no azimuthal differences, no azimuthal frame mixing) and
    within rounding of zero in the oracle's, whose coordinate-basis frames mix them with the
    others at the level of cos(pi/2) ~ 6e-17."""
    for g in axisymmetry_zero_gfs(coords):
        grp = next(gr for gr in W.GF_GROUPS if g in gr)
        scale = max(float(np.abs(ref[q * T:(q + 1) * T]).max()) for q in grp)
        assert np.all(got[g * T:(g + 1) * T] == 0.0), f"{what}: {W.GF_NAMES[g]} not exactly zero"
        assert float(np.abs(ref[g * T:(g + 1) * T]).max()) <= 1e-13 * max(scale, 1e-300), W.GF_NAMES[g]
