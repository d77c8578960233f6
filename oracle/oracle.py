"""ctypes wrapper around the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. The product library never imports it,
and it imports nothing from the product package.

Every function mirrors one function of ``lbm_oracle.c``; see that file for the
paper passage each one follows. Masks hold 0 (fluid), 1 (catalytic solid) or
2 (inert solid). Arrays are numpy, C-contiguous, linear cell
index ``(z * ny + y) * nx + x`` (x fastest); populations are
``[species][19][cell]`` with species 0 = carrier, 1 = reactant R, 2 = product P.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PRESSURE = 0
BC_PERIODIC = 1
Q_NONE, Q_FP16, Q_BF16 = 0, 1, 2
Q = 19


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            sig = {
                "orc_lattice": (None, [P, P, P, P, P]),
                "orc_feq": (None, [f64, f64, f64, f64, P]),
                "orc_round_fp16": (f64, [f64]),
                "orc_round_bf16": (f64, [f64]),
                "orc_splitmix64": (u64, [u64]),
                "orc_noise": (i64, [u64, u64]),
                "orc_box_width": (i32, [f64]),
                "orc_field": (None, [i32, i32, i32, f64, u64, P]),
                "orc_fluid_count": (i64, [f64, i64]),
                "orc_geometry": (None, [i32, i32, i32, i32, i32, f64, f64, u64, P]),
                "orc_active_links": (None, [i32, i32, i32, i32, P, P]),
                "orc_index_maps": (None, [i32, i32, i32, i32, P, P, P, P, P]),
                "orc_links": (i64, [i32, i32, i32, i32, P, P]),
                "orc_chord_length": (f64, [i32, i32, i32, i32, i32, P]),
                "orc_reaction_probability": (f64, [f64, f64]),
                "orc_knudsen": (f64, [f64, f64]),
                "orc_create": (P, [i32, i32, i32, i32, P, i32, f64, f64, f64, f64, f64, f64, f64, i32]),
                "orc_set_random_sputtering": (None, [P, u64]),
                "orc_set_barycentric": (None, [P]),
                "orc_set_velocity_inlet": (None, [P, f64]),
                "orc_set_species_tau": (None, [P, f64]),
                "orc_set_body_force": (None, [P, f64]),
                "orc_set_species_bounceback": (None, [P]),
                "orc_set_desorbing": (None, [P]),
                "orc_rs_choice": (i32, [u64, i64, i32, i64, ctypes.c_uint32]),
                "orc_destroy": (None, [P]),
                "orc_set_populations": (None, [P, i32, P]),
                "orc_get_populations": (None, [P, P]),
                "orc_step": (None, [P, i64]),
                "orc_get_step": (i64, [P]),
                "orc_fields": (None, [P, P]),
                "orc_observables": (None, [P, P, P, P, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def lattice():
    """(c [19,3] int, w [19] float64, opp [19] int) of the oracle's D3Q19."""
    cx, cy, cz = (np.zeros(Q, np.int32) for _ in range(3))
    w = np.zeros(Q, np.float64)
    opp = np.zeros(Q, np.int32)
    lib().orc_lattice(_p(cx), _p(cy), _p(cz), _p(w), _p(opp))
    return np.stack([cx, cy, cz], 1), w, opp


def feq(rho, ux, uy, uz):
    out = np.zeros(Q, np.float64)
    lib().orc_feq(rho, ux, uy, uz, _p(out))
    return out


def round_fp16(x: float) -> float:
    return lib().orc_round_fp16(float(x))


def round_bf16(x: float) -> float:
    return lib().orc_round_bf16(float(x))


def rs_choice(seed: int, cell: int, j: int, t: int, amask: int) -> int:
    """Outgoing link drawn for the population reaching node `cell` along c_j
    at step t under the random sputtering matrix (0: no active link)."""
    return lib().orc_rs_choice(int(seed), int(cell), int(j), int(t), int(amask))


def splitmix64(x: int) -> int:
    return lib().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF)


def noise(seed: int, v: int) -> int:
    return lib().orc_noise(seed, v)


def box_width(corr_len: float) -> int:
    return lib().orc_box_width(corr_len)


def field(nx, ny, nz, corr_len, seed):
    out = np.zeros(nx * ny * nz, np.int64)
    lib().orc_field(nx, ny, nz, corr_len, seed, _p(out))
    return out


def fluid_count(porosity, n_slab):
    return lib().orc_fluid_count(porosity, n_slab)


def geometry(nx, ny, nz, z0, z1, porosity, corr_len, seed):
    """uint8 mask (1 = solid), linear cell order."""
    m = np.zeros(nx * ny * nz, np.uint8)
    lib().orc_geometry(nx, ny, nz, z0, z1, porosity, corr_len, seed, _p(m))
    return m


def active_links(nx, ny, nz, mask, zper=False):
    b = np.zeros(nx * ny * nz, np.int32)
    lib().orc_active_links(nx, ny, nz, int(zper), _p(np.ascontiguousarray(mask, np.uint8)), _p(b))
    return b


def index_maps(nx, ny, nz, mask, zper=False):
    """(fluid_idx, node_idx, n_fluid, n_nodes): -1 where not applicable."""
    n = nx * ny * nz
    fi = np.zeros(n, np.int64)
    ni = np.zeros(n, np.int64)
    nf = ctypes.c_int64()
    nn = ctypes.c_int64()
    lib().orc_index_maps(nx, ny, nz, int(zper), _p(np.ascontiguousarray(mask, np.uint8)), _p(fi), _p(ni),
                         ctypes.byref(nf), ctypes.byref(nn))
    return fi, ni, nf.value, nn.value


def links(nx, ny, nz, mask, zper=False):
    """[n_links, 3] int64: (fluid cell, direction, solid target cell), canonical order."""
    m = np.ascontiguousarray(mask, np.uint8)
    cnt = lib().orc_links(nx, ny, nz, int(zper), _p(m), None)
    out = np.zeros((cnt, 3), np.int64)
    lib().orc_links(nx, ny, nz, int(zper), _p(m), _p(out))
    return out


def chord_length(nx, ny, nz, z0, z1, mask):
    return lib().orc_chord_length(nx, ny, nz, z0, z1, _p(np.ascontiguousarray(mask, np.uint8)))


def reaction_probability(Da, delta):
    return lib().orc_reaction_probability(Da, delta)


def knudsen(tau, delta):
    return lib().orc_knudsen(tau, delta)


N_SCAL = 17
SCALAR_NAMES = [
    "M_C", "M_R", "M_P", "eta", "in_C", "in_R", "in_P", "out_C", "out_R", "out_P",
    "hits_R", "hits_P", "reacted", "stuck_R", "stuck_P", "resid_C", "resid_RP",
]


class Sim:
    """One oracle simulation (two-lattice FP64)."""

    def __init__(self, nx, ny, nz, mask, *, n_species=2, tau=0.8, rho_in=1.001, rho_out=1.0, c_in=1.0,
                 p=1.0, pS_R=0.95, pS_P=0.0, bc=BC_PRESSURE, quant=Q_NONE):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        self.ns = 1 + n_species
        self.mask = np.ascontiguousarray(mask, np.uint8).reshape(-1)
        assert self.mask.size == self.n
        self._h = lib().orc_create(nx, ny, nz, bc, _p(self.mask), n_species, tau, rho_in, rho_out, c_in, p,
                                   pS_R, pS_P, quant)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        lib().orc_step(self._h, n)

    def barycentric(self):
        """Relax every array towards the common barycentric velocity."""
        lib().orc_set_barycentric(self._h)

    def velocity_inlet(self, u_in: float):
        """Inlet plane at the fixed velocity (0, 0, u_in) (with rho_in, c_in)."""
        lib().orc_set_velocity_inlet(self._h, float(u_in))

    def species_tau(self, tau_s: float):
        """Reactant and product relax with 1/tau_s."""
        lib().orc_set_species_tau(self._h, float(tau_s))

    def body_force(self, gz: float):
        """Body-force acceleration gz along z on the carrier (velocity shift)."""
        lib().orc_set_body_force(self._h, float(gz))

    def species_bounceback(self):
        """Species bounce back at every solid (no catalytic node acts)."""
        lib().orc_set_species_bounceback(self._h)

    def desorbing(self):
        """Stuck unreacted reactant desorbs: R re-emitted with (1 - p pS_R)."""
        lib().orc_set_desorbing(self._h)

    def random_sputtering(self, seed: int):
        """Switch to the random one-hot sputtering matrix (see rs_choice)."""
        lib().orc_set_random_sputtering(self._h, int(seed))

    @property
    def t(self) -> int:
        return lib().orc_get_step(self._h)

    def populations(self):
        out = np.zeros((self.ns, Q, self.n), np.float64)
        lib().orc_get_populations(self._h, _p(out))
        return out

    def set_populations(self, a: int, f):
        f = np.ascontiguousarray(f, np.float64).reshape(Q, self.n)
        lib().orc_set_populations(self._h, a, _p(f))

    def fields(self):
        """[ns + 3, n]: rho per species array, then ux, uy, uz (the carrier's,
        or the barycentric velocity after barycentric())."""
        out = np.zeros((self.ns + 3, self.n), np.float64)
        lib().orc_fields(self._h, _p(out))
        return out

    def observables(self, site=False):
        scal = np.zeros(N_SCAL, np.float64)
        prof = np.zeros((5, self.nz), np.float64)
        s = np.zeros(self.n, np.float64) if site else None
        lib().orc_observables(self._h, _p(scal), _p(prof[0]), _p(prof[1]), _p(prof[2]), _p(prof[3]),
                              _p(prof[4]), _p(s))
        d = dict(zip(SCALAR_NAMES, scal.tolist()))
        d["rhoC_z"], d["rhoR_z"], d["rhoP_z"], d["phiP_z"], d["react_z"] = prof
        if site:
            d["site"] = s
        return d
