"""The partition plan's messages between processes: two gloo ranks (127.0.0.1) each own half of
the partitions of a small grid (partition q on rank q % 2) and carry out the plan's exchange --
parity copies, then halos along axes 0, 1, 2 -- sending every record whose source partition lives
on the other rank through torch.distributed send/recv, in plan order.  Starting from the owned
canonical values only, every point of every partition's box must end with the whole grid's value,
bit for bit: the host side of a one-partition-per-process run, without a GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

TYPES = [4, 5, 6, 7, 8, 9, 4, 5, 6, 7, 8, 9, 0, 0, 1, 2, 3, 1, 2, 3, 1, 2, 3, 0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from paper_2505_00097_gb300 import binding as B

    dist.init_process_group("gloo", rank=rank, world_size=world)
    coords, N, NG, parts = case
    n = [v + 2 * NG for v in N]
    T = int(np.prod(n))
    src, par, cls = B.build_maps(coords, N, NG)
    raw, recs = B.part_plan(coords, N, NG, parts)
    # the same seeded whole-grid state on both ranks, inner ghosts as parity copies
    Y = np.random.default_rng(5).standard_normal((24, T))
    gh = np.nonzero(cls == 2)[0]
    for gf in range(24):
        Y[gf, gh] = par[gh, TYPES[gf]] * Y[gf, src[gh]]
    boxes, loc, gidx = [], {}, {}
    for q, r in enumerate(raw):
        lo, hi, olo, ohi, org = r[0:3], r[3:6], r[6:9], r[9:12], r[12:15]
        m = hi - lo + 2 * NG
        l2, l1, l0 = np.meshgrid(np.arange(m[2]), np.arange(m[1]), np.arange(m[0]), indexing="ij")
        g = (l0 + org[0]).ravel(), (l1 + org[1]).ravel(), (l2 + org[2]).ravel()
        gi = g[0] + n[0] * (g[1] + n[1] * g[2])
        own = np.all([(g[d] >= olo[d]) & (g[d] < ohi[d]) for d in range(3)], axis=0)
        if q % world == rank:
            a = np.full((24, gi.size), np.nan)
            keep = own & (cls[gi] != 2)
            a[:, keep] = Y[:, gi[keep]]
            loc[q], gidx[q] = a, gi
    other = 1 - rank
    for ph in range(4):
        r = recs[ph]
        sgn = (np.stack([np.where((r[:, 4] >> TYPES[gf]) & 1, -1.0, 1.0) for gf in range(24)]) if ph == 0
               else np.ones((24, len(r))))
        mine_src = r[:, 0] % world == rank
        mine_dst = r[:, 2] % world == rank
        send = np.nonzero(mine_src & ~mine_dst)[0]      # to the other rank, in plan order
        recv = np.nonzero(~mine_src & mine_dst)[0]      # from the other rank, in plan order
        payload = torch.from_numpy(np.stack([loc[r[k, 0]][:, r[k, 1]] for k in send], axis=1).copy()
                                   if send.size else np.zeros((24, 0)))
        got = torch.zeros((24, recv.size), dtype=torch.float64)
        if rank == 0:
            dist.send(payload, dst=other) if send.size else None
            dist.recv(got, src=other) if recv.size else None
        else:
            dist.recv(got, src=other) if recv.size else None
            dist.send(payload, dst=other) if send.size else None
        vals = {}
        for j, k in enumerate(recv):
            vals[k] = got[:, j].numpy()
        for k in np.nonzero(mine_src & mine_dst)[0]:
            vals[k] = loc[r[k, 0]][:, r[k, 1]].copy()
        for k, v in vals.items():
            loc[r[k, 2]][:, r[k, 3]] = v * sgn[:, k]
    ok = all(np.array_equal(loc[q], Y[:, gidx[q]]) for q in loc)
    out[rank] = (ok, len(loc), int(sum(len(x) for x in recs)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", [(0, (6, 6, 8), 3, (2, 2, 2)), (1, (8, 6, 12), 3, (2, 2, 2)),
                                  (1, (10, 2, 16), 5, (2, 1, 3))], ids=["sph", "cyl-general", "cyl-order8"])
def test_plan_exchange_between_two_gloo_ranks(case):
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, case, out), nprocs=world, join=True)
    assert out[0][0] and out[1][0]
    assert out[0][1] + out[1][1] == int(np.prod(case[3]))
