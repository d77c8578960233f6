"""Physics pins of the oracle's time step.

  - worked single-node example of the sputtering law (Appendix, Eq. f_P_in)
    with S_ij = 1/b(x), in exact rationals;
  - conservation: carrier mass always; R and P each when nothing sticks; R+P
    when p = 1 and the product never sticks (Appendix: R+P is conserved only
    when both sticking probabilities vanish; with p = 1 every stuck reactant
    returns as product);
  - Poiseuille flow in a slit against the parabola G/(2 nu) x (h - x),
    nu = cs^2 (tau - 1/2) (Appendix);
  - a reactive slit with a reservoir at one end and a no-flux end against the
    Thiele profile cosh(phi (1 - z/L)) / cosh(phi);
  - Table 1 and Table nondimpar numbers for the Da -> p and Kn formulas;
  - the open-box mass balance closes to rounding.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_table1.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


def _single_node_case(orc, pS_R, pS_P, p, rhoP0):
    nx = ny = nz = 5
    n = nx * ny * nz
    mask = np.zeros(n, np.uint8)
    s = (2 * ny + 2) * nx + 2
    mask[s] = 1
    sim = orc.Sim(nx, ny, nz, mask, n_species=2, p=p, pS_R=pS_R, pS_P=pS_P, bc=orc.BC_PERIODIC)
    c, w, _ = orc.lattice()
    R = np.repeat(w[:, None], n, 1) * 1.0
    P = np.repeat(w[:, None], n, 1) * rhoP0
    R[:, s] = 0
    P[:, s] = 0
    sim.set_populations(1, R)
    sim.set_populations(2, P)
    sim.step(1)
    return sim, s, c, w


@pytest.mark.parametrize("pS_R,pS_P,p", [(0.95, 0.0, 0.45), (0.3, 0.2, 0.7), (1.0, 1.0, 1.0)])
def test_sputter_single_node_worked_example(orc, pS_R, pS_P, p):
    # carrier and species at rest: collision changes nothing, so every fluid
    # neighbour of the solid node sends w_j rho towards it. Gathered:
    # A^R = rho_R sum_{j=1..18} w_j = 2/3, A^P = rho_P0 * 2/3, b = 18, and each
    # of the 18 emission directions gets (Eq. f_P_in, S_ij = 1/18):
    #   R: (1 - pS_R) A^R / 18,  P: (p pS_R A^R + (1 - pS_P) A^P) / 18
    rhoP0 = 0.5
    sim, s, c, w = _single_node_case(orc, pS_R, pS_P, p, rhoP0)
    f = sim.populations()
    nx = ny = nz = 5
    A_R = Fraction(2, 3)
    A_P = Fraction(1, 2) * Fraction(2, 3)
    F = lambda x: Fraction(x).limit_denominator(10 ** 6)
    eR = (1 - F(pS_R)) * A_R / 18
    eP = (F(p) * F(pS_R) * A_R + (1 - F(pS_P)) * A_P) / 18
    W = [Fraction(1, 3)] + [Fraction(1, 18)] * 6 + [Fraction(1, 36)] * 12
    for i in range(1, 19):
        x, y, z = 2 + c[i][0], 2 + c[i][1], 2 + c[i][2]
        y_cell = (z * ny + y) * nx + x
        assert abs(f[1, i, y_cell] - float(eR)) < 1e-15
        assert abs(f[2, i, y_cell] - float(eP)) < 1e-15
        # carrier: halfway bounce-back of its own (rest) population
        assert abs(f[0, i, y_cell] - float(W[i])) < 1e-15
    # column-stochastic S: everything not stuck comes back
    obs = sim.observables()
    assert obs["hits_R"] == pytest.approx(float(A_R), rel=1e-14)
    assert obs["hits_P"] == pytest.approx(float(A_P), rel=1e-14)


def _closed_box(orc, seed, **kw):
    nx, ny, nz = 12, 10, 14
    mask = orc.geometry(nx, ny, nz, 0, nz, 0.6, 1.5, seed)
    sim = orc.Sim(nx, ny, nz, mask, n_species=2, bc=orc.BC_PERIODIC, **kw)
    n = nx * ny * nz
    c, w, _ = orc.lattice()
    rng = np.random.default_rng(seed)
    fluid = mask == 0
    R = w[:, None] * rng.uniform(0.2, 1.0, n)[None, :] * fluid
    P = w[:, None] * rng.uniform(0.0, 0.5, n)[None, :] * fluid
    C = w[:, None] * rng.uniform(0.99, 1.01, n)[None, :] * fluid
    sim.set_populations(0, C)
    sim.set_populations(1, R)
    sim.set_populations(2, P)
    return sim


def test_conservation_no_sticking(orc):
    sim = _closed_box(orc, 11, p=0.6, pS_R=0.0, pS_P=0.0)
    o0 = sim.observables()
    sim.step(60)
    o1 = sim.observables()
    for k in ("M_C", "M_R", "M_P"):
        assert abs(o1[k] - o0[k]) < 1e-12 * o0[k], k
    assert o1["hits_R"] > 0  # species really did hit the walls


def test_conservation_full_conversion(orc):
    # p = 1, pS_P = 0: every stuck reactant returns as product, R + P conserved
    sim = _closed_box(orc, 12, p=1.0, pS_R=0.95, pS_P=0.0)
    o0 = sim.observables()
    sim.step(60)
    o1 = sim.observables()
    rp0, rp1 = o0["M_R"] + o0["M_P"], o1["M_R"] + o1["M_P"]
    assert abs(rp1 - rp0) < 1e-12 * rp0
    assert o1["M_R"] < 0.5 * o0["M_R"]  # the reaction really ran
    assert abs(o1["M_C"] - o0["M_C"]) < 1e-12 * o0["M_C"]


def test_nonconservation_matches_stuck_mass(orc):
    # general case: R + P loses exactly the stuck mass (Appendix: not conserved)
    sim = _closed_box(orc, 13, p=0.4, pS_R=0.7, pS_P=0.3)
    o0 = sim.observables()
    sim.step(40)
    o1 = sim.observables()
    lost = (o0["M_R"] + o0["M_P"]) - (o1["M_R"] + o1["M_P"])
    assert lost > 0
    assert lost == pytest.approx(o1["stuck_R"] + o1["stuck_P"], rel=1e-11)
    assert abs(o1["resid_RP"]) < 1e-11 * (o0["M_R"] + o0["M_P"])


def test_open_box_mass_balance(orc):
    m = orc.geometry(16, 16, 40, 12, 28, 0.65, 3.0, 21)
    sim = orc.Sim(16, 16, 40, m, n_species=2, p=0.3, pS_R=0.95, pS_P=0.1)
    sim.step(300)
    o = sim.observables()
    assert abs(o["resid_C"]) < 1e-10 * o["M_C"]
    assert abs(o["resid_RP"]) < 1e-10 * (o["M_R"] + o["M_P"])
    assert o["in_R"] > 0 and o["reacted"] > 0


@pytest.mark.slow
def test_poiseuille_slit(orc):
    # slit of h = 16 fluid cells between solid planes x = 0 (periodic in x, so
    # the plane bounds both sides), pressure-driven along z. Halfway
    # bounce-back puts the walls at x = 0.5 and x = 16.5.
    h, ny, nz, tau = 16, 1, 48, 0.8
    nx = h + 1
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, :, 0] = 1
    sim = orc.Sim(nx, ny, nz, mask.reshape(-1), n_species=1, tau=tau, rho_in=1.002, rho_out=1.0,
                  p=1.0, pS_R=0.0, pS_P=0.0)
    sim.step(12000)
    fl = sim.fields().reshape(5, nz, ny, nx)
    rho, uz = fl[0], fl[4]
    zc = nz // 2
    # pressure gradient from the density along the centre line, p = cs^2 rho
    zs = np.arange(zc - 6, zc + 7)
    G = -np.polyfit(zs, rho[zs, 0, h // 2 + 1], 1)[0] / 3.0
    nu = (tau - 0.5) / 3.0
    x = np.arange(1, h + 1) - 0.5
    ref = G / (2 * nu) * x * (h - x) / rho[zc, 0, 1:].mean()
    got = uz[zc, 0, 1:]
    err = np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())
    assert err < 0.01, err


def _sine_decay_rate(orc, nx, nz, mask, steps0=300, steps=2000):
    """Diffusivity from the decay of the first z-mode of R in a z-periodic box
    (no sticking): amplitude ~ exp(-D k^2 t)."""
    _, w, _ = orc.lattice()
    s = orc.Sim(nx, 1, nz, mask, n_species=1, bc=orc.BC_PERIODIC, p=0.0, pS_R=0.0, pS_P=0.0)
    z = np.arange(nz)
    cz = 1 + 0.1 * np.sin(2 * np.pi * z / nz)
    s.set_populations(1, w[:, None] * np.repeat(cz, nx)[None, :] * (mask == 0))

    def amp():
        fl = s.fields()[1].reshape(nz, nx)[:, mask.reshape(nz, nx)[0] == 0].mean(1)
        return np.abs(np.fft.rfft(fl)[1])

    s.step(steps0)
    a1 = amp()
    s.step(steps)
    a2 = amp()
    return -np.log(a2 / a1) / steps / (2 * np.pi / nz) ** 2


def test_species_diffusivity(orc):
    # advection-diffusion LB at rest: D = cs^2 (tau - 1/2) (Appendix, same tau for all species)
    D = _sine_decay_rate(orc, 1, 64, np.zeros(64, np.uint8), 200, 1000)
    assert D == pytest.approx((0.8 - 0.5) / 3.0, rel=2e-3)


def test_wall_hit_rate(orc):
    # uniform R in a periodic slit of width h: the wall-ward populations of the
    # two wall layers carry sum w = 1/6 each, so hits per step = 2 c / 6 per
    # unit wall area, i.e. a fraction 1/(3h) of the slit's mass, and the mass
    # decays at k = pS_R / (3 h) per step (p = 0: all stuck reactant is lost).
    _, w, _ = orc.lattice()
    h, nz, pS = 4, 8, 1e-3
    nx = h + 1
    mask = np.zeros((nz, 1, nx), np.uint8)
    mask[:, :, 0] = 1
    mask = mask.reshape(-1)
    s = orc.Sim(nx, 1, nz, mask, n_species=1, bc=orc.BC_PERIODIC, p=0.0, pS_R=pS, pS_P=0.0)
    s.set_populations(1, w[:, None] * (mask == 0)[None, :])
    s.step(200)
    o1 = s.observables()
    s.step(100)
    o2 = s.observables()
    hits = (o2["hits_R"] - o1["hits_R"]) / 100
    assert hits / o1["M_R"] == pytest.approx(1 / (3 * h), rel=0.01)
    assert -np.log(o2["M_R"] / o1["M_R"]) / 100 == pytest.approx(pS / (3 * h), rel=0.01)


@pytest.mark.slow
@pytest.mark.parametrize("phi", [2.0, 3.0])
def test_thiele_reactive_slit(orc, phi):
    # gas at rest (rho_in = rho_out), reservoir c_in = 1 at the inlet plane. A
    # slit of width h = 4 between catalytic walls removes R at the
    # homogenised first-order rate k = pS_R / (3 h) (test_wall_hit_rate).
    # The steady profile must solve D_eff c'' = k c, i.e. be a pure
    # combination of exp(+-m z) with the Thiele decay constant
    # m = sqrt(k / D_eff) = phi / L. In the discrete profile that reads
    # c(z+1) + c(z-1) = 2 cosh(m) c(z) at every interior plane, whatever the
    # end conditions. D_eff is the slit's own axial diffusivity (the uniform
    # re-emission over all of a wall node's active links adds to it), taken
    # from a separate non-reactive decay run.
    h, tau, L, gap = 4, 0.8, 64, 2
    nx, nz = h + 1, L + 2 * gap
    mask = np.zeros((nz, 1, nx), np.uint8)
    mask[gap:nz - gap, :, 0] = 1
    per = np.zeros((64, 1, nx), np.uint8)
    per[:, :, 0] = 1
    D_eff = _sine_decay_rate(orc, nx, 64, per.reshape(-1))
    assert D_eff > (tau - 0.5) / 3.0
    k = D_eff * (phi / L) ** 2
    pS_R = 3 * h * k
    sim = orc.Sim(nx, 1, nz, mask.reshape(-1), n_species=1, tau=tau, rho_in=1.0, rho_out=1.0, c_in=1.0,
                  p=0.0, pS_R=pS_R, pS_P=0.0)
    sim.step(60000)
    cR = sim.fields().reshape(5, nz, 1, nx)[1][:, 0, 1:].mean(1)
    zz = np.arange(gap + 8, nz - gap - 8)
    md = np.arccosh((cR[zz + 1] + cR[zz - 1]) / (2 * cR[zz]))
    assert md.max() / md.min() - 1 < 2e-3  # a pure cosh/exp profile
    assert md.mean() == pytest.approx(phi / L, rel=0.01)
    # and it decays: front-loaded like cosh(phi (1 - z/L)) / cosh(phi)
    assert cR[nz - gap - 1] / cR[gap] < 1.3 / np.cosh(phi)


def test_da_to_p_table1(orc):
    g = _golden()
    cs = g["v_bar"]
    assert cs == pytest.approx(1 / math.sqrt(3), rel=1e-15)
    assert g["tau_tr"] == pytest.approx(g["delta"] / cs, rel=1e-15)  # tau_tr = delta / v
    # Table 1: tau_ch = 2 with tau_tr = 3 sqrt(3) gives Da = 2 / (3 sqrt(3)) ~ 0.385 ~ 0.4 (nondimpar)
    Da = g["tau_ch"] / g["tau_tr"]
    assert Da == pytest.approx(g["Da"], abs=0.02)
    assert orc.reaction_probability(Da, g["delta"]) == pytest.approx(1 / g["tau_ch"], rel=1e-14)
    # p = 0.45 (Table 1) corresponds to tau_ch = 1/0.45 ~ 2.2 ("2 ~")
    Da45 = (1 / g["p"]) * cs / g["delta"]
    assert orc.reaction_probability(Da45, g["delta"]) == pytest.approx(g["p"], rel=1e-14)
    assert Da45 == pytest.approx(g["Da"], abs=0.05)
    # Da -> 0 is the transport-limited end: p saturates at 1
    assert orc.reaction_probability(1e-3, 3.0) == 1.0
    # Kn = cs (tau - 1/2) / delta ~ 0.6 for tau ~ 4, delta ~ 3 (Sec. 2.3)
    assert orc.knudsen(g["tau_for_Kn"], g["delta"]) == pytest.approx(g["Kn"], rel=0.15)


def test_eta_and_flux_definitions(orc):
    # hand-built state: uniform carrier flow u_z, R only at plane 1, P only at
    # plane nz-2 -> eta = M_P(nz-2) / M_R(1) (Eq. eff), Phi_P = sum rho_P u_z (Eq. Phi_P)
    nx, ny, nz = 4, 3, 8
    n = nx * ny * nz
    mask = np.zeros(n, np.uint8)
    sim = orc.Sim(nx, ny, nz, mask, n_species=2)
    uz = 0.01
    fC = np.repeat(orc.feq(1.0, 0.0, 0.0, uz)[:, None], n, 1)
    rng = np.random.default_rng(1)
    rR = np.zeros((nz, ny, nx))
    rR[1] = rng.uniform(0.1, 1.0, (ny, nx))
    rP = np.zeros((nz, ny, nx))
    rP[nz - 2] = rng.uniform(0.1, 1.0, (ny, nx))
    _, w, _ = orc.lattice()
    sim.set_populations(0, fC)
    sim.set_populations(1, w[:, None] * rR.reshape(1, -1))
    sim.set_populations(2, w[:, None] * rP.reshape(1, -1))
    o = sim.observables()
    assert o["eta"] == pytest.approx(rP[nz - 2].sum() / rR[1].sum(), rel=1e-14)
    assert o["phiP_z"][nz - 2] == pytest.approx(rP[nz - 2].sum() * uz, rel=1e-12)
    assert o["rhoR_z"][1] == pytest.approx(rR[1].sum(), rel=1e-14)
