"""Decomposition along z on the CPU: the partition, and the halo index
logic checked across two gloo ranks.

Each rank builds its own part of a small porous box (its planes plus the
two halo planes at the cut) and the (cell, slot) order of the population
buffers it packs and unpacks, and the catalytic nodes of the hit buffers,
in the order the library's pack kernels use (entries of a plane: cells with
no solid neighbour first, then the cells touching a solid). The ranks send
each other what they pack, as global (cell, slot) ids over gloo; each
receiver checks that this is exactly what it unpacks, element for element:
before an odd step the lower part's real plane goes into the upper part's
halo and the upper part's real plane into the lower part's halo, after it
the halos go back, and the hit buffers name the same nodes. No GPU and no
library call is involved.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1607_02874_gb300 import decomp, lbm


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _mask(nx=9, ny=7, nz=26, seed=3):
    """A porous box whose slab spans the cut (planes 2 .. nz-3 porous; the
    first and last two all fluid, as an inlet and outlet need)."""
    rng = np.random.default_rng(seed)
    m = (rng.random((nz, ny, nx)) < 0.3).astype(np.uint8)
    m[:2] = 0
    m[-2:] = 0
    return m


def test_partition_covers_every_plane_once():
    for nz, parts in ((26, 2), (27, 3), (100, 7), (9, 3)):
        r = decomp.partition(nz, parts)
        assert r[0][0] == 0 and r[-1][1] == nz
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
        assert all(z1 - z0 >= 3 for z0, z1 in r)
    with pytest.raises(ValueError):
        decomp.partition(8, 3)


def test_local_boxes_carry_two_halo_planes_per_cut():
    r = decomp.partition(30, 3)
    assert decomp.local_box(30, r, 0) == (0, r[0][1] + 2, 0, 1)
    assert decomp.local_box(30, r, 1) == (r[1][0] - 2, r[1][1] + 2, 1, 1)
    assert decomp.local_box(30, r, 2) == (r[2][0] - 2, 30, 1, 0)


def test_plane_entries_put_wall_cells_last():
    m = _mask()
    touch = decomp.solid_neighbour_mask(m)
    cells = decomp.plane_entries(m, 10)
    plane = m.shape[1] * m.shape[2]
    t = touch.reshape(-1)[cells]
    # every cell with no solid neighbour comes before every wall cell
    assert not np.any(t[:-1] & ~t[1:])
    assert np.all(m.reshape(-1)[cells] == 0) and len(cells) == int((m[10] == 0).sum())
    assert np.all(cells // plane == 10)


def _global_ids(pairs, box_z0, plane):
    return np.array([(c + box_z0 * plane) * 19 + k for c, k in pairs], np.int64)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = _mask()
        nz, ny, nx = m.shape
        plane = nx * ny
        ranges = decomp.partition(nz, world)
        bz0, bz1, lo, hi = decomp.local_box(nz, ranges, rank)
        local = m[bz0:bz1]
        side = lbm.HALO_HI if rank == 0 else lbm.HALO_LO
        peer = 1 - rank
        ok = {}
        for phase in (lbm.HALO_PRE, lbm.HALO_POST):
            send = _global_ids(decomp.halo_order(local, side, phase, lbm.HALO_PACK), bz0, plane)
            want = _global_ids(decomp.halo_order(local, side, phase, lbm.HALO_UNPACK), bz0, plane)
            n = torch.tensor([len(send)], dtype=torch.int64)
            n_peer = torch.zeros(1, dtype=torch.int64)
            reqs = [dist.isend(n, peer), dist.irecv(n_peer, peer)]
            for q in reqs:
                q.wait()
            got = torch.zeros(int(n_peer.item()), dtype=torch.int64)
            reqs = [dist.isend(torch.from_numpy(send), peer), dist.irecv(got, peer)]
            for q in reqs:
                q.wait()
            ok[phase] = (len(want) > 0, np.array_equal(got.numpy(), want))
        nodes = decomp.node_order(local, side) + bz0 * plane
        got = torch.zeros(len(nodes) + 1, dtype=torch.int64)
        mine = torch.from_numpy(np.concatenate([[len(nodes)], nodes]).astype(np.int64))
        reqs = [dist.isend(mine, peer), dist.irecv(got, peer)]
        for q in reqs:
            q.wait()
        ok["nodes"] = (len(nodes) > 0, np.array_equal(got.numpy(), mine.numpy()))
        out[rank] = ok
    finally:
        dist.destroy_process_group()


def test_halo_buffers_agree_across_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        for key, (nonempty, equal) in res[r].items():
            assert nonempty, (r, key)
            assert equal, (r, key)


def _fake_obs(rng, nz_local):
    o = {k: float(rng.random()) for k in decomp._SUMMED + decomp._INLET + decomp._OUTLET}
    for k in decomp._PROFILES:
        o[k] = rng.random(nz_local)
    return o


def _obs_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nz = 26
        ranges = decomp.partition(nz, world)
        rng = np.random.default_rng(100)
        # every rank draws every part's fake observables (same seed), then
        # contributes its own part's vector to the all-reduce
        boxes = [decomp.local_box(nz, ranges, k) for k in range(world)]
        obs = [_fake_obs(rng, b[1] - b[0]) for b in boxes]
        mine = decomp.contribution(obs[rank], rank, world, *ranges[rank], boxes[rank][0], nz)
        v = torch.from_numpy(mine)
        dist.all_reduce(v)
        got = decomp.from_contributions(v.numpy(), nz)
        total = sum(decomp.contribution(obs[k], k, world, *ranges[k], boxes[k][0], nz) for k in range(world))
        want = decomp.from_contributions(total, nz)
        ok = all(np.allclose(got[k], want[k], rtol=1e-15, atol=0) for k in want)
        # the combination rules themselves
        ok = ok and got["in_R"] == obs[0]["in_R"] and got["out_P"] == obs[-1]["out_P"]
        ok = ok and np.isclose(got["M_R"], sum(o["M_R"] for o in obs), rtol=1e-15)
        prof_ok = all(np.array_equal(got["rhoR_z"][z0:z1], obs[k]["rhoR_z"][z0 - boxes[k][0]:z1 - boxes[k][0]])
                      for k, (z0, z1) in enumerate(ranges))
        eta_ok = got["eta"] == got["rhoP_z"][nz - 2] / got["rhoR_z"][1]
        out[rank] = bool(ok and prof_ok and eta_ok)
    finally:
        dist.destroy_process_group()


def test_observables_all_reduce_across_two_gloo_ranks():
    """Each rank's share of the observables (one FP64 vector) summed by an
    all-reduce gives the whole box's: masses summed, inlet flows from the
    first part, outlet flows from the last, each plane's profile from the
    part that owns it, eta from the global profiles."""
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_obs_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {0: True, 1: True}


class _FakeSim:
    def halo_bytes(self, side):
        return 40, 24


class _FakePart:
    def __init__(self, k, world):
        self.k = k
        self.halo = (int(k > 0), int(k < world - 1))
        self.sim = _FakeSim()


def _swap_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = _FakePart(rank, world)
        ex = decomp.DistExchange(part, dist, device="cpu")
        for (k, side), (pops, hits) in ex.buf.items():
            pops.fill_(10 * rank + side)
            hits.fill_(100 + 10 * rank + side)
        ex.swap(0)
        ex.swap(1)
        got = {side: (int(ex.buf[(rank, side)][0][0]), int(ex.buf[(rank, side)][1][0]),
                      bool((ex.buf[(rank, side)][0] == ex.buf[(rank, side)][0][0]).all()))
               for (_, side) in ex.buf}
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_dist_exchange_trades_cut_buffers_over_gloo():
    """DistExchange, one part per rank with host buffers: after a swap,
    each rank's buffer at a cut holds what the rank across that cut packed
    (rank r's HI side trades with rank r + 1's LO side), for the population
    and the hit buffers alike; the outer ends have no buffer."""
    world = 3
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_swap_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    lo, hi = lbm.HALO_LO, lbm.HALO_HI
    assert set(res[0]) == {hi} and set(res[2]) == {lo} and set(res[1]) == {lo, hi}
    for r in range(world):
        for side, (pops, hits, uniform) in res[r].items():
            peer, peer_side = (r - 1, hi) if side == lo else (r + 1, lo)
            assert pops == 10 * peer + peer_side and hits == 100 + 10 * peer + peer_side and uniform, (r, side)
