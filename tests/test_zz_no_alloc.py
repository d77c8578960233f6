"""lbm_observables_noalloc: observables for callers that cannot allocate.

A caller that runs simulations inside a fixed device-memory budget (for
example a serving loop that admits each simulation by its lbm_footprint)
must be able to poll conversion without the library allocating behind its
back. This test drives the C ABI directly. The simulation gets a counting
device allocator, the new entry point is called twice in a row with steps
in between, and each time its results must equal lbm_observables' (same
kernels and summation order, so the FP64 results agree to the last bit). No
allocation may happen during the calls. Oversized boxes and site-map
requests are refused with LBM_ERR_ARG.

This file sorts last so that a run stopping at the first failure has run
every other test before it.
"""
import ctypes
import gc

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LBM_ERR_ARG = -1


class _Counting:
    """lbm_allocator that forwards to torch's caching allocator and counts."""

    def __init__(self, torch, lbm):
        self.n_alloc = 0
        self.n_free = 0
        dev = torch.cuda.current_device()

        def _alloc(ctx, nbytes, stream):
            self.n_alloc += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)

        def _free(ctx, ptr, nbytes, stream):
            self.n_free += 1
            torch.cuda.caching_allocator_delete(ptr)

        self._a = lbm.ALLOC_FN(_alloc)
        self._f = lbm.FREE_FN(_free)
        self.struct = lbm.lbm_allocator(None, self._a, self._f)


def _obs(lbm, nz):
    o = lbm.lbm_obs()
    prof = np.zeros((5, nz), np.float64)
    for k, name in enumerate(("rhoC_z", "rhoR_z", "rhoP_z", "phiP_z", "react_z")):
        setattr(o, name, prof[k].ctypes.data_as(lbm._PD))
    return o, prof


def _sim(torch, lbm, geom, alloc, **kw):
    prm = lbm.lbm_params(0.8, 1.001, 1.0, 1.0, 1.0, kw.get("p", 0.45), 0.95, kw.get("pS_P", 0.1),
                         kw.get("n_species", 2), kw.get("storage", 0), kw.get("layout", 2))
    h = ctypes.c_void_p()
    stream = torch.cuda.current_stream()
    rc = lbm.library().lbm_init(geom.handle, ctypes.byref(prm), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(alloc.struct), ctypes.byref(h))
    assert rc == 0, rc
    return h


@pytest.mark.parametrize("layout,storage", [(2, 0), (1, 1)], ids=["fluid-fp32", "dense-fp16"])
def test_noalloc_observables_equal_lbm_observables(layout, storage):
    torch = pytest.importorskip("torch")
    from paper_1607_02874_gb300 import lbm

    L = lbm.library()
    nx, ny, nz = 29, 23, 41
    geom = lbm.Geometry(nx, ny, nz, slab=(10, 31), porosity=0.62, corr_len=3.0, seed=13)
    alloc = _Counting(torch, lbm)
    h = _sim(torch, lbm, geom, alloc, layout=layout, storage=storage)
    try:
        for steps in (37, 64):  # two calls in a row, odd then even step count
            assert L.lbm_step(h, steps) == 0
            ref, ref_prof = _obs(lbm, nz)
            assert L.lbm_observables(h, ctypes.byref(ref)) == 0
            got, got_prof = _obs(lbm, nz)
            # the garbage collector must not release other tests' device
            # memory between the two readings
            gc.collect()
            gc.disable()
            try:
                before = (alloc.n_alloc, alloc.n_free, torch.cuda.memory_allocated())
                assert L.lbm_observables_noalloc(h, ctypes.byref(got)) == 0
                assert (alloc.n_alloc, alloc.n_free, torch.cuda.memory_allocated()) == before
            finally:
                gc.enable()
            assert got.step == ref.step
            # same kernels, same summation order, FP64 adds without fusion:
            # the two entry points agree to the last bit
            for k in lbm.SCALARS:
                a, b = getattr(got, k), getattr(ref, k)
                assert a == b, (k, a, b)
            np.testing.assert_array_equal(got_prof, ref_prof)
            assert ref.M_R > 0 and ref.hits_R > 0
    finally:
        L.lbm_destroy(h)
        geom.close()


def test_noalloc_refuses_site_map_and_oversized_boxes():
    torch = pytest.importorskip("torch")
    from paper_1607_02874_gb300 import lbm

    L = lbm.library()
    geom = lbm.Geometry(16, 12, 20, slab=(6, 14), porosity=0.6, corr_len=2.0, seed=3)
    alloc = _Counting(torch, lbm)
    h = _sim(torch, lbm, geom, alloc)
    try:
        L.lbm_step(h, 3)
        o, _ = _obs(lbm, 20)
        site = np.zeros(max(geom.info()["n_nodes"], 1), np.float32)
        o.site_map = site.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        assert L.lbm_observables_noalloc(h, ctypes.byref(o)) == LBM_ERR_ARG
        assert L.lbm_observables_noalloc(None, ctypes.byref(o)) == LBM_ERR_ARG
    finally:
        L.lbm_destroy(h)
        geom.close()
    # more planes than the fixed scratch holds (LBM_NOALLOC_MAX_PLANES = 4096)
    tall = lbm.Geometry(1, 1, 4100, mask=np.zeros(4100, np.uint8), bc=lbm.BC_PERIODIC)
    h = _sim(torch, lbm, tall, alloc, n_species=1)
    try:
        o, _ = _obs(lbm, 4100)
        assert L.lbm_observables_noalloc(h, ctypes.byref(o)) == LBM_ERR_ARG
        ref, _ = _obs(lbm, 4100)
        assert L.lbm_observables(h, ctypes.byref(ref)) == 0  # the allocating entry point still serves it
    finally:
        L.lbm_destroy(h)
        tall.close()
