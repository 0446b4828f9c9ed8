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
