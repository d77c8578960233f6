"""Pins of the oracle's two wall variants:

  - species bounce-back everywhere (the non-reactive reference) is the same
    computation as marking every solid cell inert: populations bit-identical,
    no wall hit, and the species mass budget closes with nothing stuck;
  - desorbing reactant (the stuck, unreacted reactant goes back into the gas,
    re-emitted with 1 - p pS_R instead of 1 - pS_R; Appendix, the remark that
    the printed law conserves R + P only without sticking): R + P is then
    conserved in a closed box at any p when pS_P = 0, while the printed law
    loses exactly the stuck mass; at p = 1 the two laws coincide bit for bit.
"""
import numpy as np

from tests.test_oracle_physics import _closed_box


def _porous(orc, values):
    nx, ny, nz = 14, 11, 30
    m = orc.geometry(nx, ny, nz, 8, 22, 0.6, 2.0, 4)
    return nx, ny, nz, (m * values).astype(np.uint8)


def test_species_bounceback_is_all_inert(orc):
    nx, ny, nz, m1 = _porous(orc, 1)
    _, _, _, m2 = _porous(orc, 2)
    a = orc.Sim(nx, ny, nz, m1, n_species=2, p=0.45, pS_P=0.1)
    a.species_bounceback()
    b = orc.Sim(nx, ny, nz, m2, n_species=2, p=0.45, pS_P=0.1)
    a.step(150)
    b.step(150)
    assert np.array_equal(a.populations(), b.populations())
    oa = a.observables()
    assert oa["hits_R"] == 0.0 and oa["reacted"] == 0.0 and oa["stuck_R"] == 0.0
    assert abs(oa["resid_RP"]) <= 1e-12 * oa["in_R"]
    assert oa["M_R"] > 0
    # the catalytic law really differs
    c = orc.Sim(nx, ny, nz, m1, n_species=2, p=0.45, pS_P=0.1)
    c.step(150)
    assert not np.array_equal(a.populations()[1], c.populations()[1])


def test_desorbing_conserves_reactant_plus_product(orc):
    for desorb in (True, False):
        sim = _closed_box(orc, 5, p=0.45, pS_R=0.95, pS_P=0.0)
        if desorb:
            sim.desorbing()
        o0 = sim.observables()
        sim.step(80)
        o1 = sim.observables()
        tot0, tot1 = o0["M_R"] + o0["M_P"], o1["M_R"] + o1["M_P"]
        assert o1["hits_R"] > 0
        if desorb:
            assert abs(tot1 - tot0) <= 1e-12 * tot0
            assert o1["stuck_R"] == 0.0
        else:
            assert tot0 - tot1 > 1e-3 * tot0
            assert abs((tot0 - tot1) - o1["stuck_R"]) <= 1e-12 * tot0


def test_desorbing_equals_printed_law_at_p1(orc):
    nx, ny, nz, m = _porous(orc, 1)
    a = orc.Sim(nx, ny, nz, m, n_species=2, p=1.0, pS_P=0.1)
    a.desorbing()
    b = orc.Sim(nx, ny, nz, m, n_species=2, p=1.0, pS_P=0.1)
    a.step(120)
    b.step(120)
    assert np.array_equal(a.populations(), b.populations())
