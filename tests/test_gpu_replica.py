"""The paper's two-dimensional reactor (Sec. 2.1, Sec. 3, Table 1) on the GPU
(through the C ABI) against the FP64 oracle: a one-cell-thick D3Q19 box with
a disk-grown ingot, the velocity inlet (U_in = 0.08, rho_C = 0.8,
rho_R = 0.2), the barycentric velocity and tau = 4.

  - plug flow: with no solid, a column started at rest reaches rho_in, U_in
    and c_in at every interior cell (the oracle's closed-form steady state),
    with either velocity option;
  - a reduced replica (100 x 1 x 60, ingot 40 x 6) in both orientations and
    both addressings, and the full 500 x 1 x 250 domain with the w = 10
    ingot: FP32 fields within 1e-5, masses, flows and the Phi_P profile;
  - the library refuses a velocity inlet on a z-periodic geometry.

In a one-cell-thick box u_y is zero up to rounding on both sides (the
populations of each +y/-y pair are equal in exact arithmetic), so it is
checked against an absolute bound instead of the max-normalised error.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import FIELDS, field_errors, interior

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
R = W.REPLICA


def _errors(gp, oc, sel):
    errs = field_errors(gp, oc, sel)
    errs.pop("uy")
    assert np.abs(gp["uy"][sel]).max() <= 1e-6 and np.abs(oc["uy"][sel]).max() <= 1e-12
    return errs


def _pair(lbm, orc, nx, nz, mask, slab, *, steps, layout=2, p=0.45, bary=True, storage=0):
    g = lbm.Geometry(nx, 1, nz, slab=slab, mask=mask)
    s = lbm.Simulation(g, tau=R["tau"], rho_in=R["rho_C"], rho_out=R["rho_C"], c_in=R["c_in"], p=p, pS_R=R["pS_R"],
                       pS_P=R["pS_P"], n_species=2, storage=storage, layout=layout, u_in=R["u_in"],
                       velocity=lbm.VELOCITY_BARYCENTRIC if bary else lbm.VELOCITY_CARRIER)
    s.step(steps)
    gp = {k: s.field(k).astype(np.float64) for k in FIELDS}
    o = orc.Sim(nx, 1, nz, mask, n_species=2, tau=R["tau"], rho_in=R["rho_C"], rho_out=R["rho_C"], c_in=R["c_in"],
                p=p, pS_R=R["pS_R"], pS_P=R["pS_P"])
    o.velocity_inlet(R["u_in"])
    if bary:
        o.barycentric()
    o.step(steps)
    fl = o.fields()
    oc = {"drho_C": fl[0] - 1.0, "rho_R": fl[1], "rho_P": fl[2], "ux": fl[3], "uy": fl[4], "uz": fl[5]}
    return g, s, gp, o, oc


def _check_obs(go, oo):
    for k in ("M_C", "M_R", "M_P"):
        assert go[k] == pytest.approx(oo[k], rel=FP32_TOL), k
    for k in ("in_C", "in_R", "out_C", "hits_R", "reacted"):
        assert abs(go[k] - oo[k]) <= FP32_TOL * max(abs(oo[k]), abs(oo["in_R"])), (k, go[k], oo[k])
    for k in ("rhoR_z", "phiP_z"):
        den = np.abs(oo[k]).max()
        if den > 0:
            assert np.abs(go[k] - oo[k]).max() <= FP32_TOL * den, k


@pytest.mark.parametrize("bary", [False, True], ids=["carrier-u", "barycentric-u"])
def test_plug_flow(orc, bary):
    from paper_1607_02874_gb300 import lbm

    nx, nz = 3, 40
    mask = np.zeros(nx * nz, np.uint8)
    g, s, gp, o, oc = _pair(lbm, orc, nx, nz, mask, (0, 0), steps=4000, bary=bary)
    sel = interior(dict(nx=nx, ny=1, nz=nz), mask)
    # FP32 state: the stored deviations round every step (~1.5e-6 after
    # 4000 steps at rho_C = 0.8)
    assert np.abs(gp["uz"][sel] - R["u_in"]).max() <= 1e-5
    assert np.abs(gp["drho_C"][sel] + 1.0 - R["rho_C"]).max() <= 1e-5
    assert np.abs(gp["rho_R"][sel] - R["c_in"]).max() <= 1e-5
    assert np.abs(gp["rho_P"][sel]).max() == 0.0
    # In this steady flow every cell rounds the same stored values the same
    # way at every step, and the reactant's FP32 rounding (~1 ulp of 0.2 per
    # cell) accumulates along the 38 cells of the flow path: a float32
    # emulation of the step gives 1.0e-5 to 1.3e-5 of c_in at the outlet for
    # every arrangement of the collision's roundings. Bound: twice the FP32
    # field tolerance.
    for k, e in _errors(gp, oc, sel).items():
        assert e <= 2 * FP32_TOL, (k, e)


@pytest.mark.parametrize("orientation,layout", [("perpendicular", 1), ("perpendicular", 2), ("parallel", 2)],
                         ids=["perpendicular-dense", "perpendicular-fluid", "parallel-fluid"])
def test_reduced_replica_matches_oracle(orc, orientation, layout):
    from paper_1607_02874_gb300 import lbm

    nx, nz = 100, 60
    box = W.ingot_box(nx, nz, 40, 6, orientation)
    mask = W.disk_ingot(nx, nz, box, porosity=R["porosity"], seed=R["seed"])
    g, s, gp, o, oc = _pair(lbm, orc, nx, nz, mask, (box[2], box[3]), steps=601, layout=layout)
    errs = _errors(gp, oc, interior(dict(nx=nx, ny=1, nz=nz), mask))
    print("reduced replica errors", orientation, layout, errs)
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    _check_obs(s.observables(), o.observables())
    assert s.observables()["hits_R"] > 0 and gp["rho_P"].max() > 0  # the reactant reached the ingot


def test_full_replica_domain_matches_oracle(orc):
    from paper_1607_02874_gb300 import lbm

    nx, nz = R["nx"], R["nz"]
    box = W.ingot_box(nx, nz, R["h"], 10)
    mask = W.disk_ingot(nx, nz, box, porosity=R["porosity"], seed=R["seed"] + 10)
    g, s, gp, o, oc = _pair(lbm, orc, nx, nz, mask, (box[2], box[3]), steps=900)
    errs = _errors(gp, oc, interior(dict(nx=nx, ny=1, nz=nz), mask))
    print("full replica errors", errs)
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    _check_obs(s.observables(), o.observables())
    assert s.observables()["hits_R"] > 0


def test_velocity_inlet_needs_open_z():
    from paper_1607_02874_gb300 import lbm

    g = lbm.Geometry(8, 8, 16, slab=(4, 12), porosity=0.6, corr_len=2.0, seed=1, bc=lbm.BC_PERIODIC)
    with pytest.raises(lbm.LbmError):
        lbm.Simulation(g, u_in=0.05)
