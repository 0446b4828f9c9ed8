"""The partition plan of the chare decomposition (Sec. 3), on the host: one grid cut into
partitions, each holding its box widened by N_G, filled after every substage by parity copies
(within a partition, or by messages from the source's partition -- the per-chare send lists)
and by halo copies face by face (axis 0, then 1, then 2).

Checked bit-exactly without a GPU, by applying the plan's records with numpy:
* the phase-0 records are the boundary map of nr_build_maps, ghost by ghost (source and
  parity), split over partitions;
* starting from the owned canonical values of a state whose inner ghosts hold the parity
  copies, the records fill every point of every partition's box with the whole grid's value;
* every point a partition owns is owned by exactly one partition, and the boxes cover the grid.
"""
import numpy as np
import pytest

from paper_2505_00097_gb300 import binding as B
from paper_2505_00097_gb300 import workloads as W

TYPES = [4, 5, 6, 7, 8, 9, 4, 5, 6, 7, 8, 9, 0, 0, 1, 2, 3, 1, 2, 3, 1, 2, 3, 0]

CASES = [
    ("cyl-two-point-z3", W.SINH_CYLINDRICAL, (8, 2, 12), 3, (1, 1, 3)),
    ("cyl-two-point-rho2-z2", W.SINH_CYLINDRICAL, (8, 2, 12), 3, (2, 1, 2)),
    ("cyl-general-phi2-z2", W.SINH_CYLINDRICAL, (6, 8, 9), 3, (1, 2, 3)),
    ("sph-general-2x2x2", W.SINH_SPHERICAL, (6, 6, 8), 3, (2, 2, 2)),
    ("sph-theta3", W.SINH_SPHERICAL, (7, 9, 6), 3, (1, 3, 2)),
    ("sph-two-point", W.SINH_SPHERICAL, (9, 8, 2), 3, (3, 2, 1)),
    ("spherical-ragged", W.SPHERICAL, (11, 7, 10), 3, (3, 2, 3)),
    ("cyl-order8", W.SINH_CYLINDRICAL, (10, 2, 16), 5, (2, 1, 3)),
    ("sph-order8", W.SINH_SPHERICAL, (10, 10, 10), 5, (2, 2, 2)),
]


def _boxes(raw, n, NG):
    out = []
    for r in raw:
        lo, hi, olo, ohi, org = r[0:3], r[3:6], r[6:9], r[9:12], r[12:15]
        m = hi - lo + 2 * NG
        out.append(dict(lo=lo, hi=hi, olo=olo, ohi=ohi, org=org, m=m, T=int(np.prod(m))))
    return out


def _global_of(b, n):
    """flat global index of every local point of box b (i0 fastest)"""
    l2, l1, l0 = np.meshgrid(np.arange(b["m"][2]), np.arange(b["m"][1]), np.arange(b["m"][0]), indexing="ij")
    g0, g1, g2 = l0 + b["org"][0], l1 + b["org"][1], l2 + b["org"][2]
    return (g0 + n[0] * (g1 + n[1] * g2)).reshape(-1), (g0.reshape(-1), g1.reshape(-1), g2.reshape(-1))


def _owned_mask(b, g):
    g0, g1, g2 = g
    return ((g0 >= b["olo"][0]) & (g0 < b["ohi"][0]) & (g1 >= b["olo"][1]) & (g1 < b["ohi"][1]) &
            (g2 >= b["olo"][2]) & (g2 < b["ohi"][2]))


@pytest.mark.parametrize("name,coords,N,NG,parts", CASES, ids=[c[0] for c in CASES])
def test_plan_reproduces_the_whole_grid(name, coords, N, NG, parts):
    n = [v + 2 * NG for v in N]
    T = int(np.prod(n))
    src, par, cls = B.build_maps(coords, N, NG)
    raw, recs = B.part_plan(coords, N, NG, parts)
    assert raw.shape[0] == int(np.prod(parts))
    boxes = _boxes(raw, n, NG)
    gidx = [_global_of(b, n) for b in boxes]
    # ownership: a partition of the whole padded grid
    owned = np.zeros(T, dtype=np.int64)
    for b, (gi, g) in zip(boxes, gidx):
        assert np.all((gi >= 0) & (gi < T))
        owned[gi[_owned_mask(b, g)]] += 1
    assert np.all(owned == 1)
    # phase 0 is the boundary map, split over partitions
    r0 = recs[0]
    assert len(r0) == int(np.sum(cls == 2))
    dst_g = np.array([gidx[p][0][l] for p, l in zip(r0[:, 2], r0[:, 3])])
    src_g = np.array([gidx[p][0][l] for p, l in zip(r0[:, 0], r0[:, 1])])
    order = np.argsort(dst_g)
    assert np.array_equal(dst_g[order], np.nonzero(cls == 2)[0])
    assert np.array_equal(src_g[order], src[dst_g[order]])
    mask = np.zeros((len(r0), 10), dtype=np.int8)
    for t in range(10):
        mask[:, t] = np.where((r0[:, 4] >> t) & 1, -1, 1)
    assert np.array_equal(mask[order], par[dst_g[order]])
    for p in range(len(boxes)):               # every fill lands on a point its partition owns
        sel = r0[:, 2] == p
        gi, g = gidx[p]
        assert np.all(_owned_mask(boxes[p], g)[r0[sel, 3]])
    # a whole-grid state with parity-consistent inner ghosts
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((24, T))
    gh = np.nonzero(cls == 2)[0]
    for gf in range(24):
        Y[gf, gh] = par[gh, TYPES[gf]] * Y[gf, src[gh]]
    # each partition starts with its owned canonical values only
    loc = []
    for b, (gi, g) in zip(boxes, gidx):
        a = np.full((24, b["T"]), np.nan)
        keep = _owned_mask(b, g) & (cls[gi] != 2)
        a[:, keep] = Y[:, gi[keep]]
        loc.append(a)
    for ph in range(4):
        r = recs[ph]
        vals = np.stack([loc[sp][:, sl] for sp, sl in zip(r[:, 0], r[:, 1])], axis=1) if len(r) else None
        if ph == 0 and len(r):
            sgn = np.stack([np.where((r[:, 4] >> TYPES[gf]) & 1, -1.0, 1.0) for gf in range(24)])
            vals = vals * sgn
        # within a phase no record reads a point another record of the phase writes
        for k, (dp, dl) in enumerate(zip(r[:, 2], r[:, 3])):
            loc[dp][:, dl] = vals[:, k]
    for b, a, (gi, g) in zip(boxes, loc, gidx):
        assert np.array_equal(a, Y[:, gi]), name


def test_plan_rejects_partitions_thinner_than_the_ghost_layers():
    with pytest.raises(B.NrError) as e:
        B.part_plan(W.SINH_CYLINDRICAL, (8, 2, 12), 3, (1, 2, 1))   # the two-point azimuth
    assert e.value.code == 1
    with pytest.raises(B.NrError):
        B.part_plan(W.SINH_CYLINDRICAL, (8, 2, 12), 3, (1, 1, 5))   # 12 / 5 < 3
    with pytest.raises(B.NrError):
        B.part_plan(W.SINH_CYLINDRICAL, (10, 2, 16), 5, (3, 1, 1))  # 10 / 3 < 5 at 8th order
    B.part_plan(W.SINH_CYLINDRICAL, (8, 2, 12), 3, (1, 1, 4))       # 3 each: allowed


def test_head_on_plan_message_counts():
    """The head-on grid cut into 4 slabs along z: no inner-boundary message (the rho < 0 ghosts map
    within their slab), one halo message per face in each direction, each N_G slices thick."""
    boxes, recs = B.part_plan(W.SINH_CYLINDRICAL, (256, 2, 512), 3, (1, 1, 4))
    assert len(recs[0]) > 0 and len(recs[1]) == 0 and len(recs[2]) == 0
    assert len(recs[3]) == 2 * 3 * (262 * 8 * 3)
    assert np.all(recs[0][:, 0] == recs[0][:, 2])
