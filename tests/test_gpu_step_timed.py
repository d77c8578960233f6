"""lbm_step_timed: one step exactly as lbm_step, with its launches timed
apart. The timed step leaves the same state as an untimed one (bit for bit,
deterministic hits), its three times are positive (the node kernels' too,
where the box has catalytic nodes), and the two entry counts cover every
lattice entry."""
import numpy as np
import pytest

import workloads
from tests.gpu_common import FIELDS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", ["fluid", "dense"])
@pytest.mark.parametrize("storage", [0, 1], ids=["fp32", "fp16"])
def test_timed_step_equals_step(storage, layout):
    from paper_1607_02874_gb300 import lbm

    c = workloads.ragged_case()
    g = lbm.Geometry(c["nx"], c["ny"], c["nz"], slab=c["slab"], porosity=c["porosity"], corr_len=c["corr_len"],
                     seed=c["seed"])
    ly = lbm.LAYOUT_FLUID if layout == "fluid" else lbm.LAYOUT_DENSE
    a = lbm.Simulation(g, n_species=2, storage=storage, layout=ly, deterministic=True, c_init=0.5)
    b = lbm.Simulation(g, n_species=2, storage=storage, layout=ly, deterministic=True, c_init=0.5)
    info = g.info()
    n_lat = info["n_fluid"] if layout == "fluid" else c["nx"] * c["ny"] * c["nz"]
    for _ in range(5):  # both parities
        a.step(1)
        ms, entries = b.step_timed()
        assert len(ms) == 3 and all(m > 0 for m in ms), ms
        assert entries[0] + entries[1] == n_lat
        assert entries[0] > 0 and entries[1] > 0
    for f in FIELDS:
        np.testing.assert_array_equal(a.field(f), b.field(f), err_msg=f)
    oa, ob = a.observables(), b.observables()
    assert oa["hits_R"] == ob["hits_R"] and oa["hits_R"] > 0


@pytest.mark.parametrize("layout", ["fluid", "dense"])
def test_warp_counts(layout):
    """Every warp with a live entry is in exactly one class. Fluid-only
    addressing finds region warps in the all-fluid planes below and above
    the slab (their odd steps form neighbour entries by arithmetic, in a
    launch of their own); dense addressing has none."""
    from paper_1607_02874_gb300 import lbm

    c = workloads.ragged_case()
    g = lbm.Geometry(c["nx"], c["ny"], c["nz"], slab=c["slab"], porosity=c["porosity"], corr_len=c["corr_len"],
                     seed=c["seed"])
    ly = lbm.LAYOUT_FLUID if layout == "fluid" else lbm.LAYOUT_DENSE
    s = lbm.Simulation(g, n_species=2, layout=ly)
    w = s.warp_counts()
    _, entries = s.step_timed()
    n_fast = w["plain"] + w["region"] + w["wall"]
    assert n_fast * 32 >= entries[0] > (n_fast - 1) * 32
    if layout == "fluid":
        assert n_fast + w["general"] == (g.info()["n_fluid"] + 31) // 32
        # below the slab, planes 2 .. slab[0] - 3 see only all-fluid planes
        # numbered in cell order (and as many above it)
        plane = c["nx"] * c["ny"]
        assert w["region"] * 32 > (c["slab"][0] - 5) * plane - 64
    else:
        assert w["region"] == 0
