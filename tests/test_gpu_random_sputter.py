"""The random sputtering matrix on the GPU (through the C ABI) against the
FP64 oracle's, which draws the same one-hot columns from the same
counter-based hash:

  - FP32 fields within 1e-5 and the wall hits, flows and masses, in both
    addressings and both step parities (a different draw anywhere would move
    the species fields next to that wall node by order one);
  - the step index the draw depends on is the same in a batched launch (one
    launch per step, or one launch for many steps): bit-identical to lbm_step
    alone, with deterministic accumulation;
  - a checkpoint of a random-matrix simulation restores its per-link
    accumulators: bit-identical continuation.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_common import FIELDS, field_errors, interior, oracle_case

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
SEED = 2024


def _orc_mask(orc, case):
    return orc.geometry(case["nx"], case["ny"], case["nz"], case["slab"][0], case["slab"][1], case["porosity"],
                        case["corr_len"], case["seed"])


def _geometry(lbm, case):
    return lbm.Geometry(case["nx"], case["ny"], case["nz"], slab=case["slab"], porosity=case["porosity"],
                        corr_len=case["corr_len"], seed=case["seed"])


@pytest.mark.parametrize("layout,steps,det", [(1, 201, False), (2, 201, False), (2, 120, True)],
                         ids=["dense-odd", "fluid-odd", "fluid-even-det"])
def test_random_matrix_matches_oracle(orc, layout, steps, det):
    from paper_1607_02874_gb300 import lbm

    case = workloads.ragged_case()
    mask = _orc_mask(orc, case)
    g = _geometry(lbm, case)
    s = lbm.Simulation(g, n_species=2, p=0.45, pS_P=0.1, layout=layout, deterministic=det,
                       sputter=lbm.SPUTTER_RANDOM, sputter_seed=SEED)
    s.step(steps)
    gp = {k: s.field(k).astype(np.float64) for k in FIELDS}
    sim = orc.Sim(case["nx"], case["ny"], case["nz"], mask, n_species=2, p=0.45, pS_P=0.1)
    sim.random_sputtering(SEED)
    sim.step(steps)
    fl = sim.fields()
    oc = {"drho_C": fl[0] - 1.0, "rho_R": fl[1], "rho_P": fl[2], "ux": fl[3], "uy": fl[4], "uz": fl[5]}
    errs = field_errors(gp, oc, interior(case, mask))
    print("random sputtering field errors", layout, steps, errs)
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    go, oo = s.observables(), sim.observables()
    for k in ("M_R", "M_P"):
        assert go[k] == pytest.approx(oo[k], rel=FP32_TOL)
    for k in ("hits_R", "hits_P", "in_R", "out_R", "reacted"):
        assert abs(go[k] - oo[k]) <= FP32_TOL * max(abs(oo[k]), abs(oo["in_R"])), (k, go[k], oo[k])
    # and the random matrix is really in use: the uniform one gives other fields
    u = oracle_case(orc, case, mask, n_species=2, steps=steps, p=0.45, pS_P=0.1)
    assert max(field_errors(gp, u, interior(case, mask))[k] for k in ("rho_R", "rho_P")) > 1e-3


@pytest.mark.parametrize("mode", [0, 1], ids=["per-step", "single-launch"])
def test_random_matrix_alone_equals_batched(mode):
    from paper_1607_02874_gb300 import lbm

    cases = [workloads.ragged_case(), workloads.CFG1]
    alone = []
    for c in cases:
        g = _geometry(lbm, c)
        s = lbm.Simulation(g, n_species=2, p=0.3, storage=lbm.FP16_DEV, layout=lbm.LAYOUT_FLUID, deterministic=True,
                           sputter=lbm.SPUTTER_RANDOM, sputter_seed=SEED)
        s.step(91)
        alone.append({k: s.field(k) for k in FIELDS})
    mix = []
    for c in cases:
        g = _geometry(lbm, c)
        mix.append((g, lbm.Simulation(g, n_species=2, p=0.3, storage=lbm.FP16_DEV, layout=lbm.LAYOUT_FLUID,
                                      deterministic=True, sputter=lbm.SPUTTER_RANDOM, sputter_seed=SEED)))
    mix[0][1].step(1)  # different parities inside the batch
    lbm.step_batch([s for _, s in mix], 90, mode=mode)
    mix[1][1].step(1)
    for k, (g, s) in enumerate(mix):
        for f in FIELDS:
            np.testing.assert_array_equal(s.field(f), alone[k][f], err_msg=f"case {k} field {f}")


def test_random_matrix_checkpoint_restores_links():
    from paper_1607_02874_gb300 import lbm

    case = workloads.ragged_case()
    g = _geometry(lbm, case)
    mk = lambda: lbm.Simulation(g, n_species=2, p=0.45, layout=lbm.LAYOUT_FLUID, deterministic=True,
                                sputter=lbm.SPUTTER_RANDOM, sputter_seed=SEED)
    a = mk()
    a.step(33)
    st = a.get_state()
    a.step(40)
    ref = {k: a.field(k) for k in FIELDS}
    b = mk()
    b.set_state(st)
    b.step(40)
    for f in FIELDS:
        np.testing.assert_array_equal(b.field(f), ref[f], err_msg=f)
    # a uniform-matrix simulation refuses the state
    u = lbm.Simulation(g, n_species=2, p=0.45, layout=lbm.LAYOUT_FLUID, deterministic=True)
    with pytest.raises(lbm.LbmError):
        u.set_state(st)
