"""Decomposition along z on one GPU, through the C ABI: a box split into 2
or 3 parts that step in lockstep and exchange only their halo planes
(lbm_halo_pops before and after odd steps, lbm_halo_hits after every step,
copied between the parts on the device) evolves exactly as the whole box.

The porous slab spans every cut, and the reactant starts inside the pores,
so that catalytic nodes of the cut planes collect wall hits from both
sides from the first step. With deterministic (fixed-point) wall hits every
field of every part's own planes equals the whole box's bit for bit, in
FP32 and in FP16 storage (whose stochastic rounding draws by global entry
number); the observables, summed over the parts in another grouping, agree
to FP64 rounding.
"""
import numpy as np
import pytest

import workloads
from paper_1607_02874_gb300 import decomp, lbm

pytestmark = pytest.mark.gpu

FIELDS = ("drho_C", "ux", "uy", "uz", "rho_R", "rho_P")


@pytest.mark.parametrize("storage,layout", [(lbm.FP32, lbm.LAYOUT_FLUID), (lbm.FP16_DEV, lbm.LAYOUT_FLUID),
                                            (lbm.FP32, lbm.LAYOUT_DENSE)], ids=["fp32", "fp16", "fp32-dense"])
@pytest.mark.parametrize("n_parts", [2, 3])
def test_parts_step_as_the_whole_box(storage, layout, n_parts):
    c = workloads.ragged_case()
    g = lbm.Geometry(c["nx"], c["ny"], c["nz"], slab=c["slab"], porosity=c["porosity"], corr_len=c["corr_len"],
                     seed=c["seed"])
    mask3 = g.export()["mask"].reshape(c["nz"], c["ny"], c["nx"])
    params = dict(n_species=2, p=0.4, pS_P=0.05, storage=storage, layout=layout, deterministic=True, c_init=0.5)
    whole = lbm.Simulation(g, **params)
    ranges = decomp.partition(c["nz"], n_parts)
    assert all(c["slab"][0] < z0 < c["slab"][1] for z0, _ in ranges[1:])  # every cut inside the slab
    parts = [decomp.Part(mask3, ranges, k, params=params, seed=c["seed"]) for k in range(n_parts)]
    ex = decomp.LocalExchange(parts)
    for n in (37, 1):  # end after an odd step, then after an even one
        whole.step(n)
        decomp.step(parts, ex, n)
        for f in FIELDS:
            got, want = decomp.field(parts, f, c["nz"], ex), whole.field(f)
            bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
            planes = sorted(set((bad // (c["nx"] * c["ny"])).tolist()))
            assert bad.size == 0, (f, n, len(bad), "planes", planes[:20], "cuts", [z0 for z0, _ in ranges[1:]])
    o, w = decomp.observables(parts, c["nz"], ex), whole.observables()
    assert w["hits_R"] > 0 and w["M_P"] > 0
    for k in ("M_C", "M_R", "M_P", "hits_R", "hits_P", "reacted", "in_C", "out_C", "in_R", "out_R", "out_P"):
        assert o[k] == pytest.approx(w[k], rel=1e-9, abs=1e-12), k
    assert o["eta"] == pytest.approx(w["eta"], rel=1e-9, abs=1e-15)
    for k in ("rhoR_z", "rhoP_z", "react_z"):
        np.testing.assert_allclose(o[k], np.asarray(w[k]), rtol=1e-12, atol=1e-12)


def test_halo_calls_refuse_a_whole_box():
    g = lbm.Geometry(12, 10, 20, slab=(6, 14), porosity=0.6, corr_len=2.0, seed=4)
    s = lbm.Simulation(g, n_species=2)
    with pytest.raises(lbm.LbmError):
        s.halo_bytes(lbm.HALO_LO)
    m = g.export()["mask"].reshape(20, 10, 12)
    parts = [decomp.Part(m, decomp.partition(20, 2), k, params=dict(n_species=2), seed=4) for k in range(2)]
    with pytest.raises(lbm.LbmError):
        parts[0].sim.halo_bytes(lbm.HALO_LO)  # the first part has no halo below
    assert parts[0].sim.halo_bytes(lbm.HALO_HI)[0] > 0
