"""Domain decomposition bookkeeping on the host (no GPU): the message plan of every subdomain
and the order of the face sites in a message (Sec. IV D: faces are packed by the sender and
unpacked by the receiver in the same order).

The face order is checked against an independent statement of what a halo entry must hold:
for a receiving site x on a cut face, the entry at its half face index (the other three local
coordinates, lexicographic, halved) must be the spinor of the global neighbour x +- mu.  The
two-rank test moves the face payloads (global site indices) between gloo processes in the plan's
order, as the NCCL transport moves the half spinors.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1712_01505_gb300 import dd  # noqa: E402

BC = (1, 1, 1, -1)
GRIDS = [((4, 4, 4, 8), (1, 1, 1, 2)), ((4, 4, 4, 8), (2, 1, 1, 2)), ((8, 4, 4, 4), (4, 1, 1, 1)),
         ((4, 4, 4, 4), (2, 2, 2, 2)), ((6, 4, 2, 4), (3, 2, 1, 1))]


def _coords(l, i):
    c = []
    for m in range(4):
        c.append(i % l[m])
        i //= l[m]
    return c


def _face_half_index(l, x, mu):
    f, stride = 0, 1
    for nu in range(4):
        if nu != mu:
            f += x[nu] * stride
            stride *= l[nu]
    return f >> 1


def _expected_halo(L, P, sid, mu, side, parity_out):
    """Global index of the neighbour that fills each halo entry of a receive message of
    subdomain `sid` (side 0: forward hops of the high face, side 1: backward hops of the
    low face) for output parity `parity_out`."""
    l = dd.local_extents(L, P)
    gs = dd.global_sites(L, P, sid)
    n = int(np.prod(l)) // l[mu] // 2
    want = -np.ones(n, dtype=np.int64)
    for i in range(int(np.prod(l))):
        x = _coords(l, i)
        if sum(x) % 2 != parity_out:
            continue
        if x[mu] != (l[mu] - 1 if side == 0 else 0):
            continue
        g = _coords(L, int(gs[i]))
        g[mu] = (g[mu] + (1 if side == 0 else -1)) % L[mu]
        want[_face_half_index(l, x, mu)] = g[0] + L[0] * (g[1] + L[1] * (g[2] + L[2] * g[3]))
    assert np.all(want >= 0)
    return want


@pytest.mark.parametrize("L,P", GRIDS)
def test_every_send_meets_its_receive(L, P):
    nsub = int(np.prod(P))
    plans = {s: dd.plan(L, P, BC, s) for s in range(nsub)}
    ncut = sum(p > 1 for p in P)
    for s, (sends, recvs) in plans.items():
        assert len(sends) == len(recvs) == 2 * ncut
        for m in sends:
            # the peer receives it on the same side: low face -> forward halo, high face -> backward halo
            match = [r for r in plans[m["peer"]][1] if r["mu"] == m["mu"] and r["side"] == m["side"]]
            assert len(match) == 1 and match[0]["peer"] == s and match[0]["nsites"] == m["nsites"]


@pytest.mark.parametrize("L,P", GRIDS)
def test_face_order_gives_each_boundary_site_its_neighbour(L, P):
    nsub = int(np.prod(P))
    for s in range(nsub):
        _, recvs = dd.plan(L, P, BC, s)
        for r in recvs:
            for par_out in (0, 1):
                # what the peer packs: its face sites of the input parity, in message order
                sent_local = dd.face_sites(L, P, BC, r["mu"], r["side"], 1 - par_out)
                sent_global = dd.global_sites(L, P, r["peer"])[sent_local]
                np.testing.assert_array_equal(sent_global, _expected_halo(L, P, s, r["mu"], r["side"], par_out))


def test_plan_refuses_bad_geometry():
    with pytest.raises(ValueError):
        dd.local_extents((4, 4, 4, 8), (1, 1, 1, 8))  # local extent 1
    from paper_1712_01505_gb300 import qcd

    with pytest.raises(qcd.QCDError):
        dd.plan((4, 4, 4, 6), (1, 1, 1, 2), BC, 0)  # local extent 3 is odd
    with pytest.raises(qcd.QCDError):
        dd.plan((4, 4, 4, 8), (1, 1, 1, 2), BC, 2)  # id out of range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, L, P, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ok = True
        sends, recvs = dd.plan(L, P, BC, rank)
        gs = dd.global_sites(L, P, rank)
        for par_out in (0, 1):
            # the sender's payload for each message: the global indices of its face sites
            reqs, bufs = [], []
            for m in sends:
                payload = torch.from_numpy(gs[dd.face_sites(L, P, BC, m["mu"], m["side"], 1 - par_out)].copy())
                reqs.append(dist.isend(payload, m["peer"], tag=2 * m["mu"] + m["side"]))
            for r in recvs:
                buf = torch.empty(r["nsites"], dtype=torch.int64)
                bufs.append((r, buf))
                reqs.append(dist.irecv(buf, r["peer"], tag=2 * r["mu"] + r["side"]))
            for q in reqs:
                q.wait()
            for r, buf in bufs:
                want = _expected_halo(L, P, rank, r["mu"], r["side"], par_out)
                ok = ok and bool(np.array_equal(buf.numpy(), want))
        out[rank] = ok
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("L,P", [((4, 4, 4, 8), (1, 1, 1, 2)), ((8, 4, 4, 4), (2, 1, 1, 1))])
def test_two_ranks_exchange_the_faces_each_needs(L, P):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, L, P, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] and out[1]
