"""ctypes binding of liblbm (argument marshalling only).

Every call maps one-to-one onto an ``extern "C"`` function of
``include/lbm.h``; all arithmetic of the time step, the boundary conditions
and the reductions runs in the library's CUDA kernels. PyTorch provides the
CUDA stream (``torch.cuda.current_stream()``) and device memory through its
caching allocator. The library must be built (``build.py``); without it, or
without a CUDA device, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the library (the bounds-checked one)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "_lib", "liblbm.so")

FP32, FP16_DEV, BF16_DEV = 0, 1, 2
HALO_LO, HALO_HI = 0, 1
HALO_PRE, HALO_POST = 0, 1
HALO_PACK, HALO_UNPACK = 0, 1
SPUTTER_UNIFORM, SPUTTER_RANDOM, SPUTTER_BOUNCEBACK = 0, 1, 2
VELOCITY_CARRIER, VELOCITY_BARYCENTRIC = 0, 1
INLET_PRESSURE, INLET_VELOCITY = 0, 1
STATE_HEADER_BYTES = 136
LAYOUT_AUTO, LAYOUT_DENSE, LAYOUT_FLUID = 0, 1, 2
BC_PRESSURE, BC_PERIODIC = 0, 1
FIELD_RHO_C, FIELD_RHO_R, FIELD_RHO_P, FIELD_UX, FIELD_UY, FIELD_UZ = range(6)
FIELDS = {"rho_C": 0, "rho_R": 1, "rho_P": 2, "ux": 3, "uy": 4, "uz": 5, "drho_C": 6}

_c_void_p = ctypes.c_void_p
ALLOC_FN = ctypes.CFUNCTYPE(_c_void_p, _c_void_p, ctypes.c_size_t, _c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, _c_void_p, _c_void_p, ctypes.c_size_t, _c_void_p)


class lbm_allocator(ctypes.Structure):
    _fields_ = [("ctx", _c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class lbm_geometry_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("slab_z0", ctypes.c_int32), ("slab_z1", ctypes.c_int32),
        ("porosity", ctypes.c_double), ("corr_len", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("mask", _c_void_p), ("bc_z", ctypes.c_int32),
        ("halo_lo", ctypes.c_int32), ("halo_hi", ctypes.c_int32), ("fluid_base", ctypes.c_int64),
        ("z_base", ctypes.c_int32),
    ]


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
        ("c_in", ctypes.c_double), ("Da", ctypes.c_double), ("p_override", ctypes.c_double),
        ("pS_R", ctypes.c_double), ("pS_P", ctypes.c_double),
        ("n_species", ctypes.c_int32), ("storage", ctypes.c_int32), ("layout", ctypes.c_int32),
        ("deterministic", ctypes.c_int32),
        ("sputter", ctypes.c_int32), ("sputter_seed", ctypes.c_uint64),
        ("velocity", ctypes.c_int32), ("inlet", ctypes.c_int32), ("u_in", ctypes.c_double),
        ("tau_s", ctypes.c_double), ("g_z", ctypes.c_double), ("desorb", ctypes.c_int32),
        ("c_init", ctypes.c_double),
    ]


_PD = ctypes.POINTER(ctypes.c_double)


class lbm_obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64)] + [
        (k, ctypes.c_double) for k in (
            "M_C", "M_R", "M_P", "eta", "in_C", "in_R", "in_P", "out_C", "out_R", "out_P",
            "hits_R", "hits_P", "reacted", "stuck_R", "stuck_P", "resid_C", "resid_RP",
            "delta", "p", "Kn")
    ] + [(k, _PD) for k in ("rhoC_z", "rhoR_z", "rhoP_z", "phiP_z", "react_z")] + [
        ("site_map", ctypes.POINTER(ctypes.c_float))]


SCALARS = ["M_C", "M_R", "M_P", "eta", "in_C", "in_R", "in_P", "out_C", "out_R", "out_P",
           "hits_R", "hits_P", "reacted", "stuck_R", "stuck_P", "resid_C", "resid_RP", "delta", "p", "Kn"]

# exported symbols and their signatures (restype, argtypes)
_P = _c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "lbm_create_geometry": (_I, [ctypes.POINTER(lbm_geometry_desc), _P, ctypes.POINTER(lbm_allocator), ctypes.POINTER(_P)]),
    "lbm_geometry_info": (_I, [_P, _P, _P, _P, _P]),
    "lbm_geometry_export": (_I, [_P, _P, _P, _P, _P, _P]),
    "lbm_geometry_free": (None, [_P]),
    "lbm_footprint": (_I, [_P, ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_request_footprint": (_I, [ctypes.POINTER(lbm_geometry_desc), ctypes.POINTER(lbm_params),
                                   ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_init": (_I, [_P, ctypes.POINTER(lbm_params), _P, ctypes.POINTER(lbm_allocator), ctypes.POINTER(_P)]),
    "lbm_step": (_I, [_P, ctypes.c_int64]),
    "lbm_step_batch": (_I, [_P, _I, ctypes.c_int64, _P]),
    "lbm_step_timed": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int64)]),
    "lbm_halo_bytes": (_I, [_P, _I, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_halo_pops": (_I, [_P, _I, _I, _I, _P]),
    "lbm_halo_hits": (_I, [_P, _I, _I, _P]),
    "lbm_observables": (_I, [_P, ctypes.POINTER(lbm_obs)]),
    "lbm_observables_noalloc": (_I, [_P, ctypes.POINTER(lbm_obs)]),
    "lbm_get_field": (_I, [_P, _I, _P, _I]),
    "lbm_get_populations": (_I, [_P, _P, _I]),
    "lbm_sim_info": (_I, [_P, _P, _P, _P, _P]),
    "lbm_warp_counts": (_I, [_P, _P]),
    "lbm_state_size": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_step_batch_mode": (_I, [_P, ctypes.c_int, ctypes.c_int64, _P, ctypes.c_int]),
    "lbm_selftest_barrier": (_I, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_int)]),
    "lbm_get_state": (_I, [_P, _P, ctypes.c_size_t]),
    "lbm_set_state": (_I, [_P, _P, ctypes.c_size_t]),
    "lbm_check_status": (_I, [ctypes.POINTER(ctypes.c_uint64)]),
    "lbm_destroy": (None, [_P]),
    "lbm_error_string": (ctypes.c_char_p, [_I]),
    "lbm_last_error": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


class LbmError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {code} {library().lbm_error_string(code).decode()} "
                         f"({library().lbm_last_error().decode()})")


def library():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"liblbm.so not built ({LIB_PATH}); run paper_1607_02874_gb300/build.py")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        raise LbmError(rc, what)


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("liblbm needs a CUDA device; no CPU fallback exists")
    return torch


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self):
        torch = _torch()
        self._torch = torch
        self._dev = torch.cuda.current_device()

        def _alloc(ctx, nbytes, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self._dev, stream)
            except Exception:  # reported to the library as an allocation failure
                return None

        def _free(ctx, ptr, nbytes, stream):
            torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = lbm_allocator(None, self._a, self._f)


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream, ctypes.c_void_p(stream.cuda_stream)


def request_footprint(nx, ny, nz, n_species=2, storage=FP32, layout=LAYOUT_AUTO, tau=0.8) -> int:
    """Upper bound of the device bytes of a request (lbm_request_footprint)."""
    d = lbm_geometry_desc(int(nx), int(ny), int(nz), 0, 0, 0.5, 1.0, 0, None, BC_PRESSURE)
    prm = lbm_params(tau, 1.001, 1.0, 1.0, 1.0, -1.0, 0.95, 0.0, int(n_species), int(storage), int(layout), 0)
    out = ctypes.c_size_t()
    _check(library().lbm_request_footprint(ctypes.byref(d), ctypes.byref(prm), ctypes.byref(out)),
           "lbm_request_footprint")
    return out.value


def selftest_barrier(ctas, expected, timeout_s, stream=None):
    """Run the bounded-wait self-test (lbm_selftest_barrier); returns
    (status code, CTAs that passed) without raising."""
    _, sh = _stream_handle(stream)
    passed = ctypes.c_int(-1)
    rc = library().lbm_selftest_barrier(int(ctas), int(expected), float(timeout_s), sh, ctypes.byref(passed))
    return rc, passed.value


BATCH_PER_STEP, BATCH_SINGLE_LAUNCH = 0, 1


def check_status():
    """First out-of-bounds access recorded by a bounds-checked build
    (kind << 56 | element index; 0: none), then cleared. Raises LbmError on
    the default build, which has no checks."""
    w = ctypes.c_uint64()
    _check(library().lbm_check_status(ctypes.byref(w)), "lbm_check_status")
    return w.value


def step_batch(sims, nsteps, stream=None, mode=BATCH_PER_STEP):
    """Advance every simulation in `sims` by `nsteps` steps in batched
    launches (lbm_step_batch_mode): one launch per group and step, or one
    launch per group for up to 1024 steps (BATCH_SINGLE_LAUNCH)."""
    if not sims:
        return
    arr = (ctypes.c_void_p * len(sims))(*[s._h.value for s in sims])
    sh = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(library().lbm_step_batch_mode(ctypes.cast(arr, ctypes.c_void_p), len(sims), int(nsteps), sh, int(mode)),
           "lbm_step_batch_mode")


class Geometry:
    """Device geometry: synthetic np-Au slab (seeded GRF) or a caller mask."""

    def __init__(self, nx, ny, nz, *, slab=(0, 0), porosity=0.65, corr_len=6.0, seed=1, mask=None,
                 bc=BC_PRESSURE, halo=(0, 0), fluid_base=0, z_base=0, stream=None, use_torch_allocator=True):
        """halo, fluid_base, z_base: a sub-domain of a z decomposition (see
        lbm_geometry_desc; decomp.py builds them)."""
        L = library()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz
        self._mask_keep = None
        d = lbm_geometry_desc(self.nx, self.ny, self.nz, int(slab[0]), int(slab[1]), float(porosity),
                              float(corr_len), int(seed), None, int(bc), int(halo[0]), int(halo[1]),
                              int(fluid_base), int(z_base))
        if mask is not None:
            m = np.ascontiguousarray(mask, np.uint8).reshape(-1)
            if m.size != self.n:
                raise ValueError("mask size does not match the box")
            self._mask_keep = m
            d.mask = m.ctypes.data_as(ctypes.c_void_p)
        self.stream, sh = _stream_handle(stream)
        self._alloc = _TorchAllocator() if use_torch_allocator else None
        h = ctypes.c_void_p()
        _check(L.lbm_create_geometry(ctypes.byref(d), sh, ctypes.byref(self._alloc.struct) if self._alloc else None,
                                     ctypes.byref(h)), "lbm_create_geometry")
        self._h = h
        self._mask_keep = None
        self.bc = bc
        self.slab = slab

    @property
    def handle(self):
        return self._h

    def info(self):
        nf, nn, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        dl = ctypes.c_double()
        _check(library().lbm_geometry_info(self._h, ctypes.byref(nf), ctypes.byref(nn), ctypes.byref(nl),
                                           ctypes.byref(dl)), "lbm_geometry_info")
        return {"n_fluid": nf.value, "n_nodes": nn.value, "n_links": nl.value, "delta": dl.value}

    def export(self, links=False):
        info = self.info()
        mask = np.zeros(self.n, np.uint8)
        fi = np.zeros(self.n, np.int32)
        ni = np.zeros(self.n, np.int32)
        b = np.zeros(self.n, np.int32)
        lk = np.zeros((info["n_links"], 3), np.int64) if links else None
        p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        _check(library().lbm_geometry_export(self._h, p(mask), p(fi), p(ni), p(b), p(lk)), "lbm_geometry_export")
        out = {"mask": mask, "fluid_idx": fi, "node_idx": ni, "b": b}
        if links:
            out["links"] = lk
        return out

    def close(self):
        if getattr(self, "_h", None):
            library().lbm_geometry_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """One resident simulation on the device."""

    def __init__(self, geom: Geometry, *, tau=0.8, rho_in=1.001, rho_out=1.0, c_in=1.0, Da=1.0, p=None,
                 pS_R=0.95, pS_P=0.0, n_species=2, storage=FP32, layout=LAYOUT_AUTO, deterministic=False,
                 sputter=SPUTTER_UNIFORM, sputter_seed=0, velocity=VELOCITY_CARRIER, u_in=None, tau_s=None,
                 g_z=0.0, desorb=False, c_init=0.0, stream=None, use_torch_allocator=True):
        """u_in: None for the pressure inlet (rho_in at the velocity of the
        first interior plane), else the fixed inlet speed along +z.
        tau_s: relaxation time of the reactant and product (None: tau).
        g_z: body-force acceleration of the carrier along +z.
        desorb: the stuck, unreacted reactant desorbs instead of being lost.
        c_init: initial reactant density in the fluid (0: none, the paper's
        start)."""
        L = library()
        self.geom = geom
        self.prm = lbm_params(float(tau), float(rho_in), float(rho_out), float(c_in), float(Da),
                              -1.0 if p is None else float(p), float(pS_R), float(pS_P), int(n_species),
                              int(storage), int(layout), int(bool(deterministic)), int(sputter),
                              int(sputter_seed), int(velocity), INLET_PRESSURE if u_in is None else INLET_VELOCITY,
                              0.0 if u_in is None else float(u_in), 0.0 if tau_s is None else float(tau_s),
                              float(g_z), int(bool(desorb)), float(c_init))
        self.stream, sh = _stream_handle(stream)
        self._alloc = _TorchAllocator() if use_torch_allocator else None
        h = ctypes.c_void_p()
        _check(L.lbm_init(geom.handle, ctypes.byref(self.prm), sh,
                          ctypes.byref(self._alloc.struct) if self._alloc else None, ctypes.byref(h)), "lbm_init")
        self._h = h
        self.ns = 1 + int(n_species)

    @staticmethod
    def footprint(geom: Geometry, **kw) -> int:
        prm = lbm_params(kw.get("tau", 0.8), 1.001, 1.0, 1.0, 1.0, -1.0, 0.95, 0.0, kw.get("n_species", 2),
                         kw.get("storage", FP32), kw.get("layout", LAYOUT_AUTO), int(kw.get("deterministic", 0)),
                         int(kw.get("sputter", SPUTTER_UNIFORM)), 0, int(kw.get("velocity", VELOCITY_CARRIER)))
        out = ctypes.c_size_t()
        _check(library().lbm_footprint(geom.handle, ctypes.byref(prm), ctypes.byref(out)), "lbm_footprint")
        return out.value

    def step(self, n=1):
        _check(library().lbm_step(self._h, int(n)), "lbm_step")

    # halo exchange of a sub-domain (lbm_halo_*; decomp.py drives them)
    def halo_bytes(self, side):
        pb, hb = ctypes.c_size_t(), ctypes.c_size_t()
        _check(library().lbm_halo_bytes(self._h, int(side), ctypes.byref(pb), ctypes.byref(hb)), "lbm_halo_bytes")
        return pb.value, hb.value

    def halo_pops(self, side, phase, direction, dev_ptr):
        _check(library().lbm_halo_pops(self._h, int(side), int(phase), int(direction), ctypes.c_void_p(dev_ptr)),
               "lbm_halo_pops")

    def halo_hits(self, side, direction, dev_ptr):
        _check(library().lbm_halo_hits(self._h, int(side), int(direction), ctypes.c_void_p(dev_ptr)),
               "lbm_halo_hits")

    def step_timed(self):
        """One step (lbm_step_timed): ((fast ms, general ms, node kernels ms),
        (fast entries, general entries))."""
        ms = (ctypes.c_float * 3)()
        ent = (ctypes.c_int64 * 2)()
        _check(library().lbm_step_timed(self._h, ms, ent), "lbm_step_timed")
        return (ms[0], ms[1], ms[2]), (ent[0], ent[1])

    def warp_counts(self):
        """Lattice warps per kernel class (lbm_warp_counts): plain, region,
        wall and general warps."""
        c = (ctypes.c_int64 * 4)()
        _check(library().lbm_warp_counts(self._h, c), "lbm_warp_counts")
        return {"plain": c[0], "region": c[1], "wall": c[2], "general": c[3]}

    def info(self):
        t, st, ly, p = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(library().lbm_sim_info(self._h, ctypes.byref(t), ctypes.byref(st), ctypes.byref(ly), ctypes.byref(p)),
               "lbm_sim_info")
        return {"step": t.value, "storage": st.value, "layout": ly.value, "p": p.value}

    def observables(self, profiles=True, site_map=False, check=True):
        nz = self.geom.nz
        o = lbm_obs()
        prof = np.zeros((5, nz), np.float64) if profiles else None
        if profiles:
            for k, name in enumerate(("rhoC_z", "rhoR_z", "rhoP_z", "phiP_z", "react_z")):
                setattr(o, name, prof[k].ctypes.data_as(_PD))
        site = None
        if site_map:
            site = np.zeros(max(self.geom.info()["n_nodes"], 1), np.float32)
            o.site_map = site.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        rc = library().lbm_observables(self._h, ctypes.byref(o))
        if check:
            _check(rc, "lbm_observables")
        d = {k: getattr(o, k) for k in SCALARS}
        d["step"] = o.step
        d["status"] = rc
        if profiles:
            d["rhoC_z"], d["rhoR_z"], d["rhoP_z"], d["phiP_z"], d["react_z"] = prof
        if site_map:
            d["site_map"] = site[: self.geom.info()["n_nodes"]]
        return d

    def observables_noalloc(self, profiles=False):
        """Observables without any device allocation (lbm_observables_noalloc)."""
        nz = self.geom.nz
        o = lbm_obs()
        prof = np.zeros((5, nz), np.float64) if profiles else None
        if profiles:
            for k, name in enumerate(("rhoC_z", "rhoR_z", "rhoP_z", "phiP_z", "react_z")):
                setattr(o, name, prof[k].ctypes.data_as(_PD))
        _check(library().lbm_observables_noalloc(self._h, ctypes.byref(o)), "lbm_observables_noalloc")
        d = {k: getattr(o, k) for k in SCALARS}
        d["step"] = o.step
        if profiles:
            d["rhoC_z"], d["rhoR_z"], d["rhoP_z"], d["phiP_z"], d["react_z"] = prof
        return d

    def field(self, name):
        out = np.zeros(self.geom.n, np.float32)
        _check(library().lbm_get_field(self._h, FIELDS[name], out.ctypes.data_as(ctypes.c_void_p), 0),
               "lbm_get_field")
        return out

    def field_into(self, name, dst_tensor):
        """Write a field into a caller device tensor (float32, n elements)."""
        _check(library().lbm_get_field(self._h, FIELDS[name], ctypes.c_void_p(dst_tensor.data_ptr()), 1),
               "lbm_get_field")

    def get_state(self) -> bytes:
        """Checkpoint: the complete resumable state as bytes (lbm_get_state)."""
        n = ctypes.c_size_t()
        _check(library().lbm_state_size(self._h, ctypes.byref(n)), "lbm_state_size")
        buf = (ctypes.c_char * n.value)()
        _check(library().lbm_get_state(self._h, ctypes.cast(buf, ctypes.c_void_p), n.value), "lbm_get_state")
        return bytes(buf)

    def set_state(self, state: bytes):
        """Restore a checkpoint taken from a simulation of the same geometry
        and parameters (lbm_set_state)."""
        buf = ctypes.create_string_buffer(state, len(state))
        _check(library().lbm_set_state(self._h, ctypes.cast(buf, ctypes.c_void_p), len(state)), "lbm_set_state")

    def populations(self):
        out = np.zeros((self.ns, 19, self.geom.n), np.float32)
        _check(library().lbm_get_populations(self._h, out.ctypes.data_as(ctypes.c_void_p), 0),
               "lbm_get_populations")
        return out

    def close(self):
        if getattr(self, "_h", None):
            library().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
