"""The catalytic path live at full size: the 512x512x1024 sample in the
configuration bench.py times (FP16 deviation storage, fluid-only addressing),
started with reactant at density 1 in every fluid cell, so that every
gas-solid link of the slab carries wall hits from the first step (the
sputtering law, Appendix, Eq. f_P_in).

  - after 60 steps reactant has reached catalytic nodes throughout the slab
    and product has formed: hits, reacted mass and product mass are positive,
    and the per-layer reaction is non-zero on every slab plane;
  - the carrier and the R + P budgets close at the 16-bit storage bound with
    the wall hits, reaction and sticking losses included;
  - the per-node site map (p pS_R A^R of the last step) sums to the per-layer
    reaction profile, and is zero outside the slab's nodes' planes.

The oracle comparison of this sample's front, with the same initial
reactant, is in test_gpu_catalytic_crop.py.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

STEPS = 60


@pytest.fixture(scope="module")
def live():
    from paper_1607_02874_gb300 import lbm

    c = workloads.CFG5
    g = lbm.Geometry(c["nx"], c["ny"], c["nz"], slab=c["slab"], porosity=c["porosity"], corr_len=c["corr_len"],
                     seed=c["seed"])
    s = lbm.Simulation(g, tau=c["tau"], rho_in=c["rho_in"], rho_out=c["rho_out"], c_in=c["c_in"], Da=c["Da"],
                       n_species=2, storage=lbm.FP16_DEV, layout=lbm.LAYOUT_FLUID, c_init=1.0)
    o0 = s.observables(profiles=False)
    s.step(STEPS)
    o = s.observables(profiles=True, site_map=True)
    yield c, g, s, o0, o
    s.close()
    g.close()


def test_initial_reactant_fills_the_fluid(live):
    c, g, s, o0, o = live
    nf = g.info()["n_fluid"]
    plane = c["nx"] * c["ny"]
    # interior planes 1 .. nz-2 hold every fluid cell except the two open
    # planes, each with density 1 less the weights of its links from
    # catalytic solid (the walls have re-emitted nothing yet): at most 1/36
    # to 1/18 per link
    full = nf - 2 * plane
    links = g.info()["n_links"]
    assert full - links / 18.0 <= o0["M_R"] <= full - links / 36.0 + 1e-6 * full
    assert o0["M_P"] == 0.0 and o0["hits_R"] == 0.0


def test_catalysis_is_live(live):
    c, g, s, o0, o = live
    assert o["hits_R"] > 0 and o["reacted"] > 0 and o["M_P"] > 0
    react = np.asarray(o["react_z"])
    z0, z1 = c["slab"]
    assert np.all(react[z0:z1] > 0)           # every slab plane reacts
    assert np.all(react[: z0 - 1] == 0) and np.all(react[z1 + 1:] == 0)  # no node outside the slab
    # the reacted mass is p pS_R of the reactant that reached the walls
    assert o["reacted"] == pytest.approx(o["p"] * 0.95 * o["hits_R"], rel=1e-12)


def test_budgets_close_with_reaction(live):
    c, g, s, o0, o = live
    assert abs(o["resid_C"]) <= 1e-6 * o["M_C"]
    # R + P lost only to sticking, gained only through the faces; FP16 species
    # round stochastically (unbiased), so the residual is a random walk far
    # below the reacted mass
    assert abs(o["resid_RP"]) <= 1e-6 * o0["M_R"]
    assert abs(o["resid_RP"]) <= 1e-3 * o["reacted"]


def test_site_map_matches_layer_profile(live):
    c, g, s, o0, o = live
    site = np.asarray(o["site_map"], np.float64)
    # (over-relaxation can leave a species population slightly negative, so
    # a few nodes may hold small negative hits)
    assert site.size == g.info()["n_nodes"] and site.sum() > 0 and np.mean(site > 0) > 0.99
    react = np.asarray(o["react_z"])
    assert site.sum() == pytest.approx(react.sum(), rel=1e-5)
