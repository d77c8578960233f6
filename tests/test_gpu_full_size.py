"""The full 512x512x1024 sample in the configuration bench.py times (FP16
deviation storage, fluid-only addressing, one launch per step):

  - the geometry's fluid count is exactly what the threshold rule gives:
    everything outside the slab, and round-half-even(porosity x slab cells)
    inside it;
  - after 20 steps the disturbance from the inlet and the outlet has moved at
    most 20 planes (one lattice link per step): every cell further from both
    is still exactly at rest. This checks every entry of the 22.6 GB
    population arrays and the 64-bit addressing behind them;
  - the first 20 planes depend only on the first 40, which lie upstream of
    the slab (all fluid). The FP64 oracle runs that 512 x 512 x 48 all-fluid
    inlet region; its outlet influence cannot reach plane 20 in 20 steps. The
    sampled planes match within the 16-bit storage bound;
  - the mass budgets close.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_common import field_errors

pytestmark = pytest.mark.gpu

STEPS = 20
FP16_FIELD_TOL = 4e-3  # the FP16 field bound of the reduced-precision tests


@pytest.fixture(scope="module")
def full():
    from paper_1607_02874_gb300 import lbm

    c = workloads.CFG5
    g = lbm.Geometry(c["nx"], c["ny"], c["nz"], slab=c["slab"], porosity=c["porosity"], corr_len=c["corr_len"],
                     seed=c["seed"])
    s = lbm.Simulation(g, tau=c["tau"], rho_in=c["rho_in"], rho_out=c["rho_out"], c_in=c["c_in"], Da=c["Da"],
                       n_species=2, storage=lbm.FP16_DEV, layout=lbm.LAYOUT_FLUID)
    s.step(STEPS)
    fields = {k: s.field(k) for k in ("drho_C", "ux", "uy", "uz", "rho_R", "rho_P")}
    yield c, g, s, fields
    s.close()
    g.close()


def test_fluid_count_is_exact(full):
    c, g, s, _ = full
    plane = c["nx"] * c["ny"]
    n_slab = plane * (c["slab"][1] - c["slab"][0])
    outside = plane * c["nz"] - n_slab
    assert g.info()["n_fluid"] == outside + round(c["porosity"] * n_slab)  # round() rounds half to even


def test_far_cells_untouched(full):
    c, g, s, f = full
    nz, plane = c["nz"], c["nx"] * c["ny"]
    lo, hi = STEPS + 2, nz - STEPS - 3  # planes the inlet/outlet cannot have reached
    for k, v in f.items():
        mid = v.reshape(nz, plane)[lo:hi + 1]
        assert np.count_nonzero(mid) == 0, k


def test_inlet_region_against_oracle(full, orc):
    c, g, s, f = full
    nx, ny, nzs = c["nx"], c["ny"], 48
    assert c["slab"][0] >= 2 * STEPS + 8  # the region upstream of the slab is all fluid
    o = orc.Sim(nx, ny, nzs, np.zeros(nx * ny * nzs, np.uint8), n_species=2, tau=c["tau"], rho_in=c["rho_in"],
                rho_out=c["rho_out"], c_in=c["c_in"], p=s.info()["p"])
    o.step(STEPS)
    fl = o.fields()
    plane = nx * ny
    sl = slice(plane, (STEPS + 1) * plane)  # planes 1 .. 20
    ref = {"drho_C": fl[0][sl] - 1.0, "rho_R": fl[1][sl], "rho_P": fl[2][sl], "ux": fl[3][sl], "uy": fl[4][sl],
           "uz": fl[5][sl]}
    got = {k: v[sl].astype(np.float64) for k, v in f.items()}
    errs = field_errors(got, ref, np.ones(sl.stop - sl.start, bool))
    print("inlet region errors", errs)
    for k in ("drho_C", "uz", "rho_R"):
        assert errs[k] <= FP16_FIELD_TOL, (k, errs[k])
    # no catalytic node upstream of the slab: no product yet
    assert np.abs(got["rho_P"]).max() == 0.0


def test_mass_budgets_close(full):
    c, g, s, _ = full
    o = s.observables(profiles=False)
    assert np.isfinite(o["M_C"]) and o["M_R"] > 0
    assert abs(o["resid_C"]) <= 1e-6 * o["M_C"]
    assert abs(o["resid_RP"]) <= 1e-3 * o["in_R"]
