"""The barycentric velocity option on the GPU (through the C ABI) against the
FP64 oracle's (Appendix, velocity equation: every array relaxes towards
feq(rho_a, u) with u = sum_a j_a / sum_a rho_a):

  - FP32 fields within 1e-5, masses, flows, wall hits and the Phi_P profile
    (which takes the same u), in both addressings, both step parities, with
    the uniform and the random sputtering matrix; the option is really in
    use: the carrier-velocity oracle gives other fields;
  - FP16 storage within the reduced-precision field bound;
  - a batched launch that mixes barycentric and carrier-velocity simulations
    keeps them apart: each comes out bit-identical to stepping it alone;
  - a checkpoint records the option: a carrier-velocity simulation refuses
    a barycentric state.

With the barycentric velocity the species' mass joins the mixture's
pressure, so the inlet reactant density is kept small (c_in = 0.05): at the
default c_in = 1 the inlet is a pressure step of the order of the density
itself, and BGK diverges (the oracle too).
"""
import numpy as np
import pytest

import workloads
from tests.gpu_common import FIELDS, field_errors, interior

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP16_FIELD_TOL = 4e-3  # the FP16 field bound of the reduced-precision tests
SEED = 31
C_IN = 0.05


def _orc_mask(orc, case):
    return orc.geometry(case["nx"], case["ny"], case["nz"], case["slab"][0], case["slab"][1], case["porosity"],
                        case["corr_len"], case["seed"])


def _geometry(lbm, case):
    return lbm.Geometry(case["nx"], case["ny"], case["nz"], slab=case["slab"], porosity=case["porosity"],
                        corr_len=case["corr_len"], seed=case["seed"])


def _oracle(orc, case, mask, steps, *, bary, sputter):
    sim = orc.Sim(case["nx"], case["ny"], case["nz"], mask, n_species=2, p=0.45, pS_P=0.1, c_in=C_IN)
    if bary:
        sim.barycentric()
    if sputter:
        sim.random_sputtering(SEED)
    sim.step(steps)
    fl = sim.fields()
    return {"drho_C": fl[0] - 1.0, "rho_R": fl[1], "rho_P": fl[2], "ux": fl[3], "uy": fl[4], "uz": fl[5]}, sim


@pytest.mark.parametrize("layout,steps,det,sputter,storage", [
    (1, 201, False, 0, 0), (2, 201, False, 0, 0), (2, 120, True, 0, 0), (2, 151, False, 1, 0), (2, 200, False, 0, 1)],
    ids=["dense-odd", "fluid-odd", "fluid-even-det", "fluid-random-matrix", "fluid-fp16"])
def test_barycentric_matches_oracle(orc, layout, steps, det, sputter, storage):
    from paper_1607_02874_gb300 import lbm

    case = workloads.ragged_case()
    mask = _orc_mask(orc, case)
    g = _geometry(lbm, case)
    s = lbm.Simulation(g, n_species=2, p=0.45, pS_P=0.1, c_in=C_IN, layout=layout, deterministic=det, storage=storage,
                       sputter=sputter, sputter_seed=SEED, velocity=lbm.VELOCITY_BARYCENTRIC)
    s.step(steps)
    gp = {k: s.field(k).astype(np.float64) for k in FIELDS}
    oc, sim = _oracle(orc, case, mask, steps, bary=True, sputter=sputter)
    sel = interior(case, mask)
    errs = field_errors(gp, oc, sel)
    print("barycentric field errors", layout, steps, sputter, storage, errs)
    tol = FP32_TOL if storage == 0 else FP16_FIELD_TOL
    for k, e in errs.items():
        assert e <= tol, (k, e)
    if storage == 0:
        go, oo = s.observables(), sim.observables()
        for k in ("M_C", "M_R", "M_P"):
            assert go[k] == pytest.approx(oo[k], rel=FP32_TOL)
        for k in ("hits_R", "hits_P", "in_R", "out_R", "reacted"):
            assert abs(go[k] - oo[k]) <= FP32_TOL * max(abs(oo[k]), abs(oo["in_R"])), (k, go[k], oo[k])
        for k in ("rhoR_z", "phiP_z"):
            den = np.abs(oo[k]).max()
            assert np.abs(go[k] - oo[k]).max() <= FP32_TOL * den, k
    # the option is really in use: the carrier's velocity gives other fields
    cv, _ = _oracle(orc, case, mask, steps, bary=False, sputter=sputter)
    assert max(field_errors(gp, cv, sel)[k] for k in ("ux", "uz")) > 1e-2


@pytest.mark.parametrize("mode", [0, 1], ids=["per-step", "single-launch"])
def test_mixed_batch_equals_alone(mode):
    from paper_1607_02874_gb300 import lbm

    cases = [workloads.ragged_case(), workloads.CFG1, workloads.ragged_case()]
    vel = [lbm.VELOCITY_BARYCENTRIC, lbm.VELOCITY_BARYCENTRIC, lbm.VELOCITY_CARRIER]
    mk = lambda c, v: lbm.Simulation(_geometry(lbm, c), n_species=2, p=0.3, c_in=C_IN, storage=lbm.FP16_DEV,
                                     layout=lbm.LAYOUT_FLUID, deterministic=True, velocity=v)
    alone = []
    for c, v in zip(cases, vel):
        s = mk(c, v)
        s.step(61)
        alone.append({k: s.field(k) for k in FIELDS})
    mix = [mk(c, v) for c, v in zip(cases, vel)]
    mix[0].step(1)  # different parities inside the batch
    lbm.step_batch(mix, 60, mode=mode)
    mix[1].step(1)
    mix[2].step(1)
    for k, s in enumerate(mix):
        for f in FIELDS:
            assert np.isfinite(alone[k][f]).all()
            np.testing.assert_array_equal(s.field(f), alone[k][f], err_msg=f"case {k} field {f}")
    # the two options really differ on the same geometry
    assert not np.array_equal(alone[0]["ux"], alone[2]["ux"])


def test_checkpoint_records_the_option():
    from paper_1607_02874_gb300 import lbm

    case = workloads.ragged_case()
    g = _geometry(lbm, case)
    mk = lambda v: lbm.Simulation(g, n_species=2, p=0.45, c_in=C_IN, layout=lbm.LAYOUT_FLUID, deterministic=True,
                                  velocity=v)
    a = mk(lbm.VELOCITY_BARYCENTRIC)
    a.step(21)
    st = a.get_state()
    a.step(30)
    ref = {k: a.field(k) for k in FIELDS}
    b = mk(lbm.VELOCITY_BARYCENTRIC)
    b.set_state(st)
    b.step(30)
    for f in FIELDS:
        np.testing.assert_array_equal(b.field(f), ref[f], err_msg=f)
    with pytest.raises(lbm.LbmError):
        mk(lbm.VELOCITY_CARRIER).set_state(st)
