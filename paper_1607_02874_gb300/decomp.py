"""Decomposition of one simulation along z (the flow axis) into sub-domains.

The paper closes by noting that the lattice Boltzmann scheme parallelises
well (Conclusions, with a pointer to multi-GPU LB work); this module splits
one box into z slabs, one per device (or several on one device), that step
in lockstep and exchange only what crosses each cut:

- ``partition`` gives each part a contiguous range of planes [z0, z1);
- each part's box holds its planes plus, at each internal cut, two halo
  planes of its neighbour (``lbm_geometry_desc.halo_lo / halo_hi``): the
  inner one exchanges populations and wall hits, the outer one completes the
  catalytic nodes' links;
- around every odd step the 5 populations per array that cross the cut go
  to the neighbour's inner halo (before the step) and back into the
  neighbour's real plane (after it); after every step the wall hits of the
  two shared planes' catalytic nodes are summed on both sides
  (``lbm_halo_pops``, ``lbm_halo_hits``);
- observables combine: masses, hits and profiles are sums over the parts,
  the face flows come from the first and last part, eta from the global
  profiles (``contribution``: one FP64 vector per part, summed in one
  process or by an all-reduce across ranks, ``dist_observables``).

With deterministic wall-hit accumulation every field equals the whole box's
bit for bit (the stochastic rounding of the 16-bit formats draws by global
entry number). The exchange is pluggable: ``LocalExchange`` copies between
parts that live in one process (on one device: the test of the protocol),
``DistExchange`` sends through torch.distributed (NCCL between devices, one
part per rank).
"""
from __future__ import annotations

import numpy as np

from . import lbm

Q = 19
CX = (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0)
CY = (0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1)
CZ = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1)
UP = tuple(k for k in range(Q) if CZ[k] > 0)    # 5, 11, 14, 15, 18
DOWN = tuple(k for k in range(Q) if CZ[k] < 0)  # 6, 12, 13, 16, 17


def partition(nz, parts, min_planes=3):
    """Owned planes [z0, z1) of each part: contiguous, as even as possible,
    at least min_planes each."""
    if parts < 1 or nz < parts * min_planes:
        raise ValueError(f"cannot split {nz} planes into {parts} parts of at least {min_planes}")
    cuts = [round(k * nz / parts) for k in range(parts + 1)]
    return [(cuts[k], cuts[k + 1]) for k in range(parts)]


def local_box(nz, ranges, k):
    """(box_z0, box_z1, halo_lo, halo_hi) of part k: its planes plus two
    halo planes at each internal cut."""
    z0, z1 = ranges[k]
    lo, hi = int(k > 0), int(k < len(ranges) - 1)
    return z0 - 2 * lo, z1 + 2 * hi, lo, hi


def solid_neighbour_mask(mask3):
    """Per cell of a [nz, ny, nx] box (x, y periodic, nothing beyond the z
    ends): whether any of its 18 neighbours is solid, as the library's
    geometry builder computes it for the entry order."""
    nz = mask3.shape[0]
    solid = mask3 != 0
    any_s = np.zeros(mask3.shape, bool)
    for k in range(1, Q):
        sh = np.roll(solid, (-CY[k], -CX[k]), axis=(1, 2))  # value at (y + cy, x + cx)
        out = np.zeros_like(solid)
        if CZ[k] > 0:
            out[: nz - 1] = sh[1:]
        elif CZ[k] < 0:
            out[1:] = sh[: nz - 1]
        else:
            out = sh
        any_s |= out
    return any_s


def plane_entries(mask3, z):
    """Cells of plane z of a box in the order of its lattice entries
    (fluid-only addressing): cells with no solid neighbour first, then the
    cells touching a solid, each in linear order."""
    nyx = mask3.shape[1] * mask3.shape[2]
    fl = mask3[z].reshape(-1) == 0
    touch = solid_neighbour_mask(mask3)[z].reshape(-1)
    cells = np.arange(nyx)
    order = np.concatenate([cells[fl & ~touch], cells[fl & touch]])
    return z * nyx + order


def halo_order(mask3, side, phase, direction):
    """(local cell, slot) pairs of one population buffer of a part's box, in
    buffer order ([5 slots][entries of the plane]), as lbm_halo_pops packs
    or unpacks them (fluid-only addressing)."""
    nz = mask3.shape[0]
    lo = side == lbm.HALO_LO
    zr, zh = (2, 1) if lo else (nz - 3, nz - 2)
    real = (phase == lbm.HALO_PRE) == (direction == lbm.HALO_PACK)
    z = zr if real else zh
    up = real == lo
    cells = plane_entries(mask3, z)
    slots = UP if up else DOWN
    return [(int(c), k) for k in slots for c in cells]


def node_order(mask3, side):
    """Local cells of the catalytic nodes of the two planes a cut shares, in
    the order of lbm_halo_hits' buffers (node number: linear cell order)."""
    nz = mask3.shape[0]
    zlo = 1 if side == lbm.HALO_LO else nz - 3
    plane = mask3.shape[1] * mask3.shape[2]
    m = mask3.reshape(-1)
    # catalytic nodes: catalytic solid with at least one fluid neighbour
    fluid = mask3 == 0
    has_fluid = np.zeros(mask3.shape, bool)
    for k in range(1, Q):
        sh = np.roll(fluid, (-CY[k], -CX[k]), axis=(1, 2))
        out = np.zeros_like(fluid)
        if CZ[k] > 0:
            out[: nz - 1] = sh[1:]
        elif CZ[k] < 0:
            out[1:] = sh[: nz - 1]
        else:
            out = sh
        has_fluid |= out
    node = (m == 1) & has_fluid.reshape(-1)
    idx = np.arange(zlo * plane, (zlo + 2) * plane)
    return idx[node[idx]]


class Part:
    """One sub-domain: its geometry and simulation on the current device."""

    def __init__(self, mask3, ranges, k, *, params, stream=None, seed=1):
        nz, ny, nx = mask3.shape
        bz0, bz1, lo, hi = local_box(nz, ranges, k)
        self.k, self.ranges = k, ranges
        self.z0, self.z1 = ranges[k]
        self.box_z0, self.halo = bz0, (lo, hi)
        local = np.ascontiguousarray(mask3[bz0:bz1])
        fluid_base = int((mask3[:bz0] == 0).sum())
        self.geom = lbm.Geometry(nx, ny, bz1 - bz0, mask=local.reshape(-1), halo=(lo, hi), fluid_base=fluid_base,
                                 z_base=bz0, seed=seed, stream=stream)
        self.sim = lbm.Simulation(self.geom, stream=stream, **params)
        self.mask3 = local

    def real_slice(self):
        """Local planes this part owns."""
        return slice(self.z0 - self.box_z0, self.z1 - self.box_z0)


class LocalExchange:
    """Parts in one process: each buffer is copied straight into the
    neighbour's (device-to-device on one stream)."""

    def __init__(self, parts):
        import torch

        self.torch = torch
        self.parts = parts
        dev = torch.cuda.current_device()
        self.buf = {}
        for p in parts:
            for side in (lbm.HALO_LO, lbm.HALO_HI):
                if not p.halo[side]:
                    continue
                pb, hb = p.sim.halo_bytes(side)
                self.buf[(p.k, side)] = (torch.empty(max(pb, 16), dtype=torch.uint8, device=dev),
                                         torch.empty(max(hb, 16), dtype=torch.uint8, device=dev))

    def swap(self, kind):
        """Exchange buffer `kind` (0 populations, 1 hits) across every cut:
        the lower part's HI buffer and the upper part's LO buffer trade
        contents."""
        for a, b in zip(self.parts[:-1], self.parts[1:]):
            x, y = self.buf[(a.k, lbm.HALO_HI)][kind], self.buf[(b.k, lbm.HALO_LO)][kind]
            t = x.clone()
            n = min(x.numel(), y.numel())
            x[:n].copy_(y[:n])
            y[:n].copy_(t[:n])


def step(parts, exchange, n=1):
    """Advance every part by n steps in lockstep (one process, parts on one
    device and one stream: LocalExchange)."""
    for _ in range(n):
        odd = parts[0].sim.info()["step"] % 2 == 1
        if odd:
            _pops(parts, exchange, lbm.HALO_PRE)
        for p in parts:
            p.sim.step(1)
        if odd:
            _pops(parts, exchange, lbm.HALO_POST)
        for p in parts:
            for side in (lbm.HALO_LO, lbm.HALO_HI):
                if p.halo[side]:
                    p.sim.halo_hits(side, lbm.HALO_PACK, exchange.buf[(p.k, side)][1].data_ptr())
        exchange.swap(1)
        for p in parts:
            for side in (lbm.HALO_LO, lbm.HALO_HI):
                if p.halo[side]:
                    p.sim.halo_hits(side, lbm.HALO_UNPACK, exchange.buf[(p.k, side)][1].data_ptr())


def _pops(parts, exchange, phase):
    for p in parts:
        for side in (lbm.HALO_LO, lbm.HALO_HI):
            if p.halo[side]:
                p.sim.halo_pops(side, phase, lbm.HALO_PACK, exchange.buf[(p.k, side)][0].data_ptr())
    exchange.swap(0)
    for p in parts:
        for side in (lbm.HALO_LO, lbm.HALO_HI):
            if p.halo[side]:
                p.sim.halo_pops(side, phase, lbm.HALO_UNPACK, exchange.buf[(p.k, side)][0].data_ptr())


def refresh(parts, exchange):
    """Make the halos current for reading. After an even step (the next one
    odd) a cell of a cut plane finds the populations that cross the cut
    towards it in the neighbour's slots, which lie in the halo; they arrive
    with the exchange that precedes the next odd step. Doing it now as well
    is harmless: nothing writes those halo slots before that step."""
    if parts[0].sim.info()["step"] % 2 == 1:
        _pops(parts, exchange, lbm.HALO_PRE)


def field(parts, name, nz, exchange):
    """A field of the whole box from the parts' own planes."""
    refresh(parts, exchange)
    ny, nx = parts[0].mask3.shape[1:]
    out = np.zeros((nz, ny, nx), np.float32)
    for p in parts:
        f = p.sim.field(name).reshape(-1, ny, nx)
        out[p.z0:p.z1] = f[p.real_slice()]
    return out.reshape(-1)


_SUMMED = ("M_C", "M_R", "M_P", "hits_R", "hits_P", "reacted", "stuck_R", "stuck_P", "resid_C", "resid_RP")
_INLET = ("in_C", "in_R", "in_P")
_OUTLET = ("out_C", "out_R", "out_P")
_PROFILES = ("rhoC_z", "rhoR_z", "rhoP_z", "phiP_z", "react_z")


def contribution(obs, k, n_parts, z0, z1, box_z0, nz):
    """One part's share of the whole box's observables as one FP64 vector,
    so that the whole box's are the plain sum of the parts' vectors (an
    all-reduce across ranks): masses, hits and residuals add; the inlet
    flows come from the first part and the outlet flows from the last; each
    profile holds the part's own planes at their global z and zeros
    elsewhere."""
    v = np.zeros(len(_SUMMED) + len(_INLET) + len(_OUTLET) + len(_PROFILES) * nz)
    v[: len(_SUMMED)] = [obs[key] for key in _SUMMED]
    o = len(_SUMMED)
    if k == 0:
        v[o:o + 3] = [obs[key] for key in _INLET]
    if k == n_parts - 1:
        v[o + 3:o + 6] = [obs[key] for key in _OUTLET]
    o += 6
    for key in _PROFILES:
        v[o + z0:o + z1] = np.asarray(obs[key])[z0 - box_z0:z1 - box_z0]
        o += nz
    return v


def from_contributions(total, nz):
    """The whole box's observables from the sum of the parts' vectors; eta
    (Sec. 3, Eq. eff) from the global profiles."""
    out = {key: float(total[n]) for n, key in enumerate(_SUMMED)}
    o = len(_SUMMED)
    for n, key in enumerate(_INLET + _OUTLET):
        out[key] = float(total[o + n])
    o += 6
    for key in _PROFILES:
        out[key] = np.array(total[o:o + nz])
        o += nz
    out["eta"] = out["rhoP_z"][nz - 2] / out["rhoR_z"][1] if out["rhoR_z"][1] != 0 else 0.0
    return out


def observables(parts, nz, exchange):
    """Observables of the whole box from the parts' (one process)."""
    refresh(parts, exchange)
    total = 0.0
    for p in parts:
        o = p.sim.observables(profiles=True)
        total = total + contribution(o, p.k, len(p.ranges), p.z0, p.z1, p.box_z0, nz)
    return from_contributions(total, nz)


def dist_observables(part, nz, exchange, dist):
    """Observables of the whole box on every rank, one part per rank: the
    parts' vectors summed by an FP64 all-reduce."""
    import torch

    refresh([part], exchange)
    o = part.sim.observables(profiles=True)
    v = torch.from_numpy(contribution(o, part.k, len(part.ranges), part.z0, part.z1, part.box_z0, nz))
    if exchange.buf and next(iter(exchange.buf.values()))[0].is_cuda:
        v = v.cuda()
    dist.all_reduce(v)
    return from_contributions(v.cpu().numpy(), nz)


class DistExchange:
    """One part per rank: buffers travel through torch.distributed
    (device tensors over NCCL, host tensors over gloo); rank r's HI buffer
    trades with rank r + 1's LO buffer."""

    def __init__(self, part, dist, device="cuda"):
        import torch

        self.torch, self.dist, self.part = torch, dist, part
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.buf = {}
        for side in (lbm.HALO_LO, lbm.HALO_HI):
            if part.halo[side]:
                pb, hb = part.sim.halo_bytes(side)
                self.buf[(part.k, side)] = (torch.empty(max(pb, 16), dtype=torch.uint8, device=device),
                                            torch.empty(max(hb, 16), dtype=torch.uint8, device=device))

    def swap(self, kind):
        ops = []
        torch, dist = self.torch, self.dist
        recv = {}
        for side, peer in ((lbm.HALO_LO, self.rank - 1), (lbm.HALO_HI, self.rank + 1)):
            if (self.part.k, side) not in self.buf:
                continue
            b = self.buf[(self.part.k, side)][kind]
            recv[side] = torch.empty_like(b)
            ops.append(dist.P2POp(dist.isend, b, peer))
            ops.append(dist.P2POp(dist.irecv, recv[side], peer))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        for side, t in recv.items():
            self.buf[(self.part.k, side)][kind].copy_(t)
