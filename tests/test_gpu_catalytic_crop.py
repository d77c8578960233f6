"""The sputtering boundary condition live on a crop of the 512x512x1024
sample's slab front, against the FP64 oracle.

The crop is x, y in [0, 64), z in [96, 160) of the oracle's own mask of the
full sample (the porous slab starts at z = 128, so the crop holds 32 open
planes and 32 slab planes), run as its own box with the same boundary types
and two fluid planes added at each end. Both sides start with reactant at
density 1 at rest in every fluid cell (the oracle through its population
setter, the library through c_init; the populations that arrive from
catalytic solid start at zero on both sides, since the walls have
re-emitted nothing yet), so that every gas-solid link of the slab carries
wall hits from the first step; 300 steps. Bounds, as for the
reduced-precision crop of the 256x256x512 sample:
  - FP32 storage: fields 2e-5 (max-normalised), reacted mass 2e-5;
  - FP16 storage (species rounded stochastically): fields 4e-3, reacted
    mass 1e-3.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_common import FIELDS, field_errors

pytestmark = pytest.mark.gpu

STEPS = 300
C_INIT = 1.0


@pytest.fixture(scope="module")
def crop(orc):
    c = workloads.CFG5
    full = orc.geometry(c["nx"], c["ny"], c["nz"], c["slab"][0], c["slab"][1], c["porosity"], c["corr_len"],
                        c["seed"]).reshape(c["nz"], c["ny"], c["nx"])
    sub = np.ascontiguousarray(full[96:160, 0:64, 0:64])
    del full
    pad = np.zeros((2, 64, 64), np.uint8)
    m = np.concatenate([pad, sub, pad]).astype(np.uint8)
    nz = m.shape[0]
    mask = m.reshape(-1)
    delta = orc.chord_length(64, 64, nz, 2 + 128 - 96, nz - 2, mask)
    p = orc.reaction_probability(c["Da"], delta)
    o = orc.Sim(64, 64, nz, mask, n_species=2, p=p)
    # reactant at rest in every fluid cell, except the populations that
    # arrive from catalytic solid: the walls have re-emitted nothing yet
    cq, w, _ = orc.lattice()
    m3 = mask.reshape(nz, 64, 64)
    f0 = np.zeros((19, nz, 64, 64))
    for i in range(19):
        up = np.roll(m3, (cq[i, 2], cq[i, 1], cq[i, 0]), axis=(0, 1, 2))  # mask at x - c_i (x, y periodic)
        if cq[i, 2] > 0:
            up[0] = 0  # upwind outside the box: the inlet plane, reset every step
        elif cq[i, 2] < 0:
            up[-1] = 0
        f0[i] = np.where((m3 == 0) & (up != 1), w[i] * C_INIT, 0.0)
    o.set_populations(1, f0.reshape(19, -1))
    o.step(STEPS)
    fl = o.fields()
    ref = {"drho_C": fl[0] - 1.0, "rho_R": fl[1], "rho_P": fl[2], "ux": fl[3], "uy": fl[4], "uz": fl[5]}
    obs = o.observables()
    z = np.arange(mask.size) // (64 * 64)
    sel = (mask == 0) & (z > 0) & (z < nz - 1)
    return nz, mask, p, ref, obs, sel


@pytest.mark.parametrize("storage,field_tol,react_tol", [(0, 2e-5, 2e-5), (1, 4e-3, 1e-3)], ids=["fp32", "fp16"])
def test_catalytic_front_against_oracle(crop, storage, field_tol, react_tol):
    from paper_1607_02874_gb300 import lbm

    nz, mask, p, ref, obs, sel = crop
    assert obs["reacted"] > 0 and obs["M_P"] > 0  # the boundary condition is live
    g = lbm.Geometry(64, 64, nz, mask=mask)
    s = lbm.Simulation(g, n_species=2, p=p, storage=storage, layout=lbm.LAYOUT_FLUID, c_init=C_INIT)
    s.step(STEPS)
    got = {k: s.field(k).astype(np.float64) for k in FIELDS}
    errs = field_errors(got, ref, sel)
    o = s.observables()
    react_err = abs(o["reacted"] - obs["reacted"]) / obs["reacted"]
    print("storage", storage, "field errors", errs, "reacted error", react_err, "reacted", obs["reacted"])
    for k, e in errs.items():
        assert e <= field_tol, (k, e)
    assert react_err <= react_tol
    assert abs(o["M_P"] - obs["M_P"]) <= react_tol * obs["M_P"]
