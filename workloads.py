"""Seeded synthetic workloads shared by the tests, the benchmark and smoke().

Holds only sizes, parameters and seeded random draws (no lattice Boltzmann
arithmetic): the porous geometry itself is generated independently by the
library and by the oracle from these parameters.

For the three-dimensional samples a thresholded Gaussian random field with
the porosity and correlation length below stands in for the paper's np-Au
reconstructions. The paper's own two-dimensional ingot (pore disks grown to
porosity 0.70 +- 0.005 in a 500 x 250 domain, Sec. 2.1) is rebuilt by
disk_ingot for the reactor replica.
"""
from __future__ import annotations

import numpy as np

# Plain method, small: 32x32x64, slab z in [16, 48), porosity 0.65, corr 6,
# carrier + reactant, Da = 1, 500 steps.
CFG1 = dict(name="cfg1_32x32x64_CR", nx=32, ny=32, nz=64, slab=(16, 48), porosity=0.65, corr_len=6.0, seed=1,
            n_species=1, Da=1.0, tau=0.8, rho_in=1.001, rho_out=1.0, c_in=1.0, steps=500)
# Da sweep: 128x128x256, slab 128 layers thick, porosity 0.60, corr 10, C+R+P.
CFG2 = dict(name="cfg2_128x128x256_CRP", nx=128, ny=128, nz=256, slab=(64, 192), porosity=0.60, corr_len=10.0,
            seed=2, n_species=2, Da_list=(1e-3, 1e-2, 1e-1, 1.0, 10.0), Da=1.0, tau=0.8, rho_in=1.001,
            rho_out=1.0, c_in=1.0, steps=20000)
# Precision: 256x256x512, porosity 0.70, corr 14, Da = 1, 10k steps; oracle
# comparison on a 64^3 crop x, y in [0, 64), z in [96, 160) run as its own box.
CFG3 = dict(name="cfg3_256x256x512_CRP", nx=256, ny=256, nz=512, slab=(128, 384), porosity=0.70, corr_len=14.0,
            seed=3, n_species=2, Da=1.0, tau=0.8, rho_in=1.001, rho_out=1.0, c_in=1.0, steps=10000)
# Large single sample: 512x512x1024, slab 768 layers, porosity 0.65, corr 20,
# Da = 0.1, FP16 storage, fluid-only addressing, 5k steps.
CFG5 = dict(name="cfg5_512x512x1024_CRP", nx=512, ny=512, nz=1024, slab=(128, 896), porosity=0.65,
            corr_len=20.0, seed=5, n_species=2, Da=0.1, tau=0.8, rho_in=1.001, rho_out=1.0, c_in=1.0, steps=5000)

CONFIGS = {c["name"]: c for c in (CFG1, CFG2, CFG3, CFG5)}

# The paper's two-dimensional reactor (Sec. 2.1, Fig. 7, Table 1): 500 x 250
# lattice units, H = 500 across the flow and L = 250 along it, run as a
# one-cell-thick periodic D3Q19 box (nx = 500, ny = 1, nz = 250; with no
# variation along y the D3Q19 populations sum to the D2Q9 weights). The ingot
# is h = 200 across and w along the flow (perpendicular orientation), or w
# across and h along (parallel orientation), centred, porosity 0.70 +- 0.005
# from 30 nm (3 lattice unit) pore disks. Inlet: speed U_in = 0.08 with
# rho_C = 0.8 and rho_R = 0.2; initial rho_C = 0.8 (Sec. 3). tau = 4 (Sec. 2.3,
# Knudsen number paragraph).
REPLICA = dict(name="replica_500x1x250", nx=500, ny=1, nz=250, h=200, w_list=(6, 10, 20, 30), h_list=(100, 150, 200, 250),
               p_list=(0.35, 0.45, 0.55, 0.65), u_in=0.08, rho_C=0.8, c_in=0.2, tau=4.0, porosity=0.70,
               pore_diameter=3.0, pS_R=0.95, pS_P=0.0, steps=30000, seed=11)


# The Appendix's validation channel: 150 lattice units of reactive bottom
# plate, L_y = 50 between the plates, Pe = 253, p = 1 (every reactant that
# reaches the plate reacts), a body force driving the carrier. Run as a
# one-cell-thick box: x across the channel (catalytic plate at x = 0, inert
# plate at x = L_y + 1), z along it (two fluid planes at either end, which the
# inlet/outlet conditions need). Pe = U_max L_y / D with D = cs^2 (tau_s - 1/2)
# (the paper's 4 Pe in its Lévêque formula reads as 6 U_mean = 4 U_max); the
# carrier relaxes with tau = 1 so that the Poiseuille profile develops in a
# few thousand steps, the species with tau_s = 0.55.
LEVEQUE = dict(name="leveque_52x1x154", L=150, L_y=50, Pe=253.0, tau=1.0, tau_s=0.55, steps=30000)


def leveque_force():
    """Body-force acceleration of the Poiseuille flow with U_max = Pe D / L_y:
    g = 8 nu U_max / L_y^2."""
    c = LEVEQUE
    nu, D = (c["tau"] - 0.5) / 3.0, (c["tau_s"] - 0.5) / 3.0
    return 8.0 * nu * (c["Pe"] * D / c["L_y"]) / c["L_y"] ** 2


def leveque_mask():
    """[nz * nx] uint8 (x fastest): catalytic plate (1) at x = 0 and inert
    plate (2) at x = L_y + 1, both over z in [2, L + 2)."""
    c = LEVEQUE
    nx, nz = c["L_y"] + 2, c["L"] + 4
    m = np.zeros((nz, nx), np.uint8)
    m[2:nz - 2, 0] = 1
    m[2:nz - 2, nx - 1] = 2
    return m.reshape(-1)


def ingot_box(nx, nz, h, w, orientation="perpendicular"):
    """[x0, x1) x [z0, z1) of a centred h x w ingot; perpendicular: h across
    the flow (x), w along it (z); parallel: the other way round."""
    ax, az = (h, w) if orientation == "perpendicular" else (w, h)
    x0, z0 = (nx - ax) // 2, (nz - az) // 2
    return x0, x0 + ax, z0, z0 + az


def disk_ingot(nx, nz, box, *, porosity=0.70, diameter=3.0, tol=0.005, seed=0):
    """Solid mask [nz * nx] (uint8, 1 = solid, x fastest) of a one-cell-thick
    box: the rectangle box = (x0, x1, z0, z1) starts solid and pore disks of
    the given diameter are carved out of it one at a time, centres drawn
    uniformly (continuous) in the rectangle, until its porosity reaches
    porosity - tol. A cell belongs to a disk when its centre lies within
    diameter / 2 of the disk's centre. One disk frees at most 9 cells, so for
    a rectangle of at least 9 / (2 tol) cells the porosity ends inside
    porosity +- tol."""
    x0, x1, z0, z1 = box
    m = np.zeros((nz, nx), np.uint8)
    m[z0:z1, x0:x1] = 1
    area = (x1 - x0) * (z1 - z0)
    rng = np.random.default_rng(seed)
    r2 = (diameter / 2.0) ** 2
    reach = int(np.ceil(diameter / 2.0))
    solid = area
    while 1.0 - solid / area < porosity - tol:
        cx, cz = rng.uniform(x0, x1), rng.uniform(z0, z1)
        ix, iz = int(np.floor(cx)), int(np.floor(cz))
        for z in range(max(iz - reach, z0), min(iz + reach + 1, z1)):
            for x in range(max(ix - reach, x0), min(ix + reach + 1, x1)):
                if (x + 0.5 - cx) ** 2 + (z + 0.5 - cz) ** 2 <= r2 and m[z, x]:
                    m[z, x] = 0
                    solid -= 1
    return m.reshape(-1)


def serving_requests(n=256, rate_per_s=20.0, seed=4, base_seed=1000):
    """Serving stream: Poisson arrivals (mean rate_per_s), cubic boxes with
    side uniform in [48, 192], porosity U[0.55, 0.75], correlation length
    U[4, 16], Da log-uniform in [1e-3, 10], slab [L/4, 3L/4), one seed per
    request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for k in range(n):
        L = int(rng.integers(48, 193))
        out.append(dict(id=k, arrival=float(t[k]), nx=L, ny=L, nz=L, slab=(L // 4, 3 * L // 4),
                        porosity=float(rng.uniform(0.55, 0.75)), corr_len=float(rng.uniform(4.0, 16.0)),
                        Da=float(10 ** rng.uniform(-3, 1)), seed=base_seed + k))
    return out


def ragged_case():
    """A small box with sizes that are not multiples of any tile (parity tests)."""
    return dict(name="ragged_37x29x50", nx=37, ny=29, nz=50, slab=(12, 38), porosity=0.6, corr_len=3.0, seed=7)
