"""Degenerate inputs, GPU (through the C ABI) against the FP64 oracle:

  - a slab with no solid at all: no catalytic node, no wall hit, in both
    addressings and with the random sputtering matrix;
  - a fully solid slab: the box splits into an inlet and an outlet region
    with no path between them;
  - the smallest box the library accepts, a 1 x 1 x 8 column (x and y wrap
    onto the cell itself);
  - one species (C + R) with the random sputtering matrix.
"""
import numpy as np
import pytest

from tests.gpu_common import FIELDS, field_errors, interior

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _run(lbm, orc, case, *, layout, steps, n_species=2, sputter=0, p=0.45, mask=None):
    nx, ny, nz = case["n"]
    g = lbm.Geometry(nx, ny, nz, slab=case["slab"], porosity=case["phi"], corr_len=case["l"], seed=case["seed"],
                     mask=mask)
    s = lbm.Simulation(g, n_species=n_species, p=p, pS_P=0.1, layout=layout, sputter=sputter, sputter_seed=7)
    s.step(steps)
    gp = {k: s.field(k).astype(np.float64) for k in FIELDS if n_species == 2 or k != "rho_P"}
    if n_species == 1:
        gp["rho_P"] = np.zeros(g.n)
    m = g.export()["mask"]
    sim = orc.Sim(nx, ny, nz, m, n_species=n_species, p=p, pS_P=0.1)
    if sputter:
        sim.random_sputtering(7)
    sim.step(steps)
    fl = sim.fields()
    ns = 1 + n_species
    oc = {"drho_C": fl[0] - 1.0, "rho_R": fl[1], "rho_P": fl[2] if ns > 2 else np.zeros(sim.n),
          "ux": fl[ns], "uy": fl[ns + 1], "uz": fl[ns + 2]}
    box = {"nx": nx, "ny": ny, "nz": nz}
    return g, s, gp, oc, sim.observables(), field_errors(gp, oc, interior(box, m))


@pytest.mark.parametrize("layout,sputter", [(1, 0), (2, 0), (2, 1)], ids=["dense", "fluid", "fluid-random"])
def test_slab_without_solid(orc, layout, sputter):
    from paper_1607_02874_gb300 import lbm

    case = dict(n=(21, 13, 40), slab=(10, 30), phi=1.0, l=3.0, seed=5)
    g, s, gp, oc, oo, errs = _run(lbm, orc, case, layout=layout, steps=101, sputter=sputter)
    assert g.info()["n_nodes"] == 0 and g.info()["n_fluid"] == 21 * 13 * 40
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    o = s.observables(site_map=True)
    assert o["hits_R"] == 0.0 and o["hits_P"] == 0.0 and oo["hits_R"] == 0.0
    assert o["M_R"] == pytest.approx(oo["M_R"], rel=FP32_TOL)


def test_fully_solid_slab(orc):
    from paper_1607_02874_gb300 import lbm

    case = dict(n=(16, 12, 40), slab=(12, 28), phi=0.0, l=3.0, seed=6)
    g, s, gp, oc, oo, errs = _run(lbm, orc, case, layout=2, steps=121)
    assert g.info()["n_fluid"] == 16 * 12 * 24
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    # no flow crosses the slab: nothing of R reaches the outlet side
    o = s.observables()
    assert o["hits_R"] > 0
    rho_R = gp["rho_R"].reshape(40, 12, 16)
    assert np.abs(rho_R[28:]).max() == 0.0


def test_single_column(orc):
    from paper_1607_02874_gb300 import lbm

    case = dict(n=(1, 1, 8), slab=(0, 0), phi=1.0, l=1.0, seed=1)
    for layout in (1, 2):
        g, s, gp, oc, oo, errs = _run(lbm, orc, case, layout=layout, steps=57)
        for k, e in errs.items():
            assert e <= FP32_TOL, (layout, k, e)


@pytest.mark.parametrize("layout", [1, 2], ids=["dense", "fluid"])
def test_single_species_random_matrix(orc, layout):
    from paper_1607_02874_gb300 import lbm

    case = dict(n=(23, 19, 44), slab=(12, 32), phi=0.62, l=2.5, seed=9)
    g, s, gp, oc, oo, errs = _run(lbm, orc, case, layout=layout, steps=150, n_species=1, sputter=1)
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    o = s.observables()
    assert o["hits_R"] == pytest.approx(oo["hits_R"], rel=FP32_TOL)
    assert o["reacted"] == pytest.approx(oo["reacted"], rel=FP32_TOL)
