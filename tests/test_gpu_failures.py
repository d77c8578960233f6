"""Failure detection on the GPU, with every failure made on the host:
- an allocator that refuses its k-th request, for every allocation site of
  lbm_create_geometry and lbm_init: the call answers LBM_ERR_OOM and hands
  every block it did get back to the allocator;
- a state whose populations are NaN, loaded through lbm_set_state: the step
  runs on, and lbm_observables / lbm_observables_noalloc answer
  LBM_ERR_DIVERGED;
- after either, the context and the library keep working.
No kernel is made to fault, trap or hang."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOX = dict(n=(24, 20, 40), slab=(10, 30), phi=0.62, l=3.0, seed=31)


class CountingAllocator:
    """Device memory from torch's caching allocator; refuses request number
    `fail_at` (0-based) and records what is outstanding."""

    def __init__(self, lbm, torch, fail_at=None):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        dev = torch.cuda.current_device()

        def _alloc(ctx, nbytes, stream):
            k = self.calls
            self.calls += 1
            if k == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            self.live[p] = int(nbytes)
            return p

        def _free(ctx, ptr, nbytes, stream):
            assert ptr in self.live, "freed a block it was not given"
            assert self.live.pop(ptr) == nbytes, "freed with another size"
            torch.cuda.caching_allocator_delete(ptr)

        self._a = lbm.ALLOC_FN(_alloc)
        self._f = lbm.FREE_FN(_free)
        self.struct = lbm.lbm_allocator(None, self._a, self._f)


def _desc(lbm):
    return lbm.lbm_geometry_desc(*BOX["n"], *BOX["slab"], BOX["phi"], BOX["l"], BOX["seed"], None, lbm.BC_PRESSURE)


def _params(lbm):
    return lbm.lbm_params(0.8, 1.001, 1.0, 1.0, 1.0, -1.0, 0.95, 0.0, 2, lbm.FP32, lbm.LAYOUT_FLUID, 0)


def test_allocation_failure_at_every_site_is_reported_and_leaks_nothing():
    import torch

    from paper_1607_02874_gb300 import lbm

    L = lbm.library()
    stream = torch.cuda.current_stream()
    sh = ctypes.c_void_p(stream.cuda_stream)
    d = _desc(lbm)
    prm = _params(lbm)
    # count the allocations of a run that succeeds
    ok = CountingAllocator(lbm, torch)
    g = ctypes.c_void_p()
    assert L.lbm_create_geometry(ctypes.byref(d), sh, ctypes.byref(ok.struct), ctypes.byref(g)) == 0
    n_geo = ok.calls
    s = ctypes.c_void_p()
    assert L.lbm_init(g, ctypes.byref(prm), sh, ctypes.byref(ok.struct), ctypes.byref(s)) == 0
    n_sim = ok.calls - n_geo
    assert n_geo >= 8 and n_sim >= 5
    L.lbm_destroy(s)
    L.lbm_geometry_free(g)
    torch.cuda.synchronize()
    assert not ok.live

    for k in range(n_geo):
        a = CountingAllocator(lbm, torch, fail_at=k)
        h = ctypes.c_void_p()
        assert L.lbm_create_geometry(ctypes.byref(d), sh, ctypes.byref(a.struct), ctypes.byref(h)) == -2, k
        assert b"allocation" in L.lbm_last_error()
        torch.cuda.synchronize()
        assert not a.live, (k, a.live)

    good = lbm.Geometry(*BOX["n"], slab=BOX["slab"], porosity=BOX["phi"], corr_len=BOX["l"], seed=BOX["seed"])
    for k in range(n_sim):
        a = CountingAllocator(lbm, torch, fail_at=k)
        h = ctypes.c_void_p(1234)
        assert L.lbm_init(good.handle, ctypes.byref(prm), sh, ctypes.byref(a.struct), ctypes.byref(h)) == -2, k
        assert h.value is None  # no handle on failure
        torch.cuda.synchronize()
        assert not a.live, (k, a.live)

    # the library and the context still work
    sim = lbm.Simulation(good, n_species=2, layout=lbm.LAYOUT_FLUID)
    sim.step(20)
    assert sim.observables(profiles=False)["M_C"] > 0


def test_nan_state_is_reported_as_divergence():
    from paper_1607_02874_gb300 import lbm

    g = lbm.Geometry(*BOX["n"], slab=BOX["slab"], porosity=BOX["phi"], corr_len=BOX["l"], seed=BOX["seed"])
    s = lbm.Simulation(g, n_species=2, storage=lbm.FP32, layout=lbm.LAYOUT_FLUID)
    s.step(10)
    st = bytearray(s.get_state())
    n = len(st) - lbm.STATE_HEADER_BYTES
    # every float32 after the header becomes a quiet NaN (0xFFFFFFFF); the
    # FP64 bookkeeping becomes NaN too
    st[lbm.STATE_HEADER_BYTES:] = b"\xff" * n
    s.set_state(bytes(st))
    s.step(2)  # a NaN state steps without fault
    for call in (lambda: s.observables(profiles=False), lambda: s.observables_noalloc()):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.code == -4
        assert b"diverged" in lbm.library().lbm_error_string(e.value.code)
    # a fresh simulation on the same geometry is unaffected
    t = lbm.Simulation(g, n_species=2, storage=lbm.FP32, layout=lbm.LAYOUT_FLUID)
    t.step(10)
    o = t.observables(profiles=False)
    assert np.isfinite(o["M_R"]) and o["M_C"] > 0
