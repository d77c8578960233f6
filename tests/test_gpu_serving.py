"""Continuous batching on the GPU: a simulation advanced inside batched
launches with others (different sizes, porosities, Da, step parities; one
launch per step or one launch for many steps) ends in the bit-identical state
it reaches alone; the step is reproducible run to run; the bounded wait of the
single-launch mode reports a timeout; and a short real serving run completes
every request."""
import numpy as np
import pytest

from tests.gpu_common import FIELDS

pytestmark = pytest.mark.gpu

CASES = [
    dict(n=(24, 20, 40), slab=(10, 30), phi=0.62, l=3.0, seed=31, Da=1.0),
    dict(n=(33, 17, 28), slab=(7, 21), phi=0.70, l=2.0, seed=32, Da=0.05),
    dict(n=(16, 16, 52), slab=(13, 39), phi=0.55, l=4.0, seed=33, Da=10.0),
]


def _make(lbm, c, storage, stream=None):
    g = lbm.Geometry(*c["n"], slab=c["slab"], porosity=c["phi"], corr_len=c["l"], seed=c["seed"], stream=stream)
    s = lbm.Simulation(g, Da=c["Da"], n_species=2, storage=storage, layout=lbm.LAYOUT_FLUID, deterministic=True,
                       stream=stream)
    return g, s


def _fields(s):
    return {k: s.field(k).astype(np.float64) for k in FIELDS}


@pytest.mark.parametrize("mode", [0, 1], ids=["per-step", "single-launch"])
@pytest.mark.parametrize("storage", [0, 1], ids=["fp32", "fp16"])
def test_alone_equals_mix(storage, mode):
    from paper_1607_02874_gb300 import lbm

    alone = []
    for k, c in enumerate(CASES):
        g, s = _make(lbm, c, storage)
        s.step(k + 150)  # different step counts, so different parities in the mix
        alone.append((g, s, _fields(s), s.observables(profiles=False)))
    mix = [_make(lbm, c, storage) for c in CASES]
    for k, (g, s) in enumerate(mix):
        s.step(k + 50)  # bring the three to different parities first
    lbm.step_batch([s for _, s in mix], 100, mode=mode)
    for k, (g, s) in enumerate(mix):
        assert s.info()["step"] == k + 150
        got = _fields(s)
        ref = alone[k][2]
        mask = g.export()["mask"]
        nz = CASES[k]["n"][2]
        plane = CASES[k]["n"][0] * CASES[k]["n"][1]
        z = np.arange(mask.size) // plane
        sel = (mask == 0) & (z > 0) & (z < nz - 1)
        # the step is deterministic (fixed-point wall-hit sums, per-block
        # FP64 bookkeeping), so batching changes nothing: bit-identical
        for f in FIELDS:
            np.testing.assert_array_equal(got[f][sel], ref[f][sel], err_msg=f"case {k} field {f}")
        o = s.observables(profiles=False)
        for key in ("M_R", "M_P", "hits_R", "eta", "in_R", "out_R"):
            assert o[key] == alone[k][3][key], (k, key)


def test_step_is_reproducible():
    from paper_1607_02874_gb300 import lbm

    runs = []
    for _ in range(2):
        g, s = _make(lbm, CASES[0], 0)
        s.step(77)
        runs.append((_fields(s), s.observables(profiles=False)))
    for f in FIELDS:
        np.testing.assert_array_equal(runs[0][0][f], runs[1][0][f])
    assert runs[0][1]["hits_R"] == runs[1][1]["hits_R"]


def test_serving_run_completes():
    from paper_1607_02874_gb300 import lbm
    from paper_1607_02874_gb300.serving import LbmBackend, Request, ServingLoop

    reqs = [Request(id=i, arrival=0.02 * i, nx=c["n"][0], ny=c["n"][1], nz=c["n"][2], slab=c["slab"],
                    porosity=c["phi"], corr_len=c["l"], Da=c["Da"], seed=c["seed"]) for i, c in enumerate(CASES * 2)]
    be = LbmBackend(storage=lbm.FP16_DEV, layout=lbm.LAYOUT_FLUID)
    budget = 3 * max(be.footprint(r) for r in reqs)  # at most ~3 resident at once
    loop = ServingLoop(be, budget_bytes=budget, steps_per_tick=100, check_every=500, max_steps=1500, tol=1e-8)
    out = loop.run(reqs)
    assert out["requests"] == len(reqs)
    assert all(np.isfinite(r["finished"]) and r["steps"] > 0 for r in out["records"])
    assert out["p99_s"] >= out["p50_s"] > 0
    ticks = [e for e in loop.trace if e[1] == "tick"]
    assert max(e[2] for e in ticks) >= 2  # several simulations shared launches


BIG = [
    dict(n=(96, 96, 96), slab=(24, 72), phi=0.65, l=5.0, seed=41, Da=0.1, storage=1, layout=2),
    dict(n=(64, 80, 72), slab=(18, 54), phi=0.60, l=4.0, seed=42, Da=1.0, storage=0, layout=2),
    dict(n=(40, 40, 48), slab=(12, 36), phi=0.70, l=3.0, seed=43, Da=3.0, storage=0, layout=1),
    dict(n=(48, 32, 64), slab=(16, 48), phi=0.62, l=3.0, seed=44, Da=0.5, storage=1, layout=2),
]


def _make_big(lbm, c):
    g = lbm.Geometry(*c["n"], slab=c["slab"], porosity=c["phi"], corr_len=c["l"], seed=c["seed"])
    s = lbm.Simulation(g, Da=c["Da"], n_species=2, storage=c["storage"], layout=c["layout"], deterministic=True)
    return g, s


@pytest.mark.parametrize("mode", [0, 1], ids=["per-step", "single-launch"])
def test_multistep_batch_is_bit_identical(mode):
    """One launch covers many steps (CTAs ordered by tickets, far more CTAs
    than fit on the GPU at once), three launch groups (storage x layout), and
    a step count that spans two launches (1024 + 6): every simulation ends
    bit-identical to stepping it alone."""
    from paper_1607_02874_gb300 import lbm

    steps = 1030
    alone = []
    for c in BIG:
        g, s = _make_big(lbm, c)
        s.step(steps + 1)
        alone.append(_fields(s))
        s.close()
        g.close()
    mix = [_make_big(lbm, c) for c in BIG]
    mix[0][1].step(1)
    mix[1][1].step(1)
    mix[2][1].step(1)
    lbm.step_batch([s for _, s in mix[:3]], steps, mode=mode)  # at odd parity
    mix[3][1].step(steps)
    lbm.step_batch([mix[3][1]], 1, mode=mode)
    for k, (g, s) in enumerate(mix):
        assert s.info()["step"] == steps + 1
        got = _fields(s)
        for f in FIELDS:
            np.testing.assert_array_equal(got[f], alone[k][f], err_msg=f"case {k} field {f}")


def test_bounded_wait_reports_timeout():
    """The step-ordering wait of the batched launch is bounded: a wait that can
    never end (it expects more CTA arrivals than CTAs were launched) gives up
    after its limit with LBM_ERR_TIMEOUT, and the context keeps working."""
    import time

    from paper_1607_02874_gb300 import lbm

    assert lbm.selftest_barrier(2, 2, 0.5) == (0, 2)
    assert lbm.selftest_barrier(4, 1, 0.5) == (0, 4)
    t0 = time.perf_counter()
    rc, passed = lbm.selftest_barrier(3, 4, 0.05)
    dt = time.perf_counter() - t0
    assert rc == -6 and passed == 0
    assert 0.04 < dt < 5.0
    assert b"limit" in lbm.library().lbm_last_error()
    g, s = _make(lbm, CASES[0], 0)
    s.step(10)
    assert s.observables(profiles=False)["M_C"] > 0
