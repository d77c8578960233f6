"""Pins of the oracle's validation-channel ingredients (Appendix, validation
of the numerical model: a body-force-driven channel, reactive bottom plate,
inert top plate):

  - species relaxation time of their own: a sine mode of R decays at
    D = cs^2 (tau_s - 1/2) while the carrier keeps tau;
  - inert solid (mask 2) bounces every array back as the carrier: in a closed
    periodic box with inert obstacles and an uneven flow, a reactant started
    proportional to the carrier (same tau, same velocity) stays exactly
    proportional, with no wall hit; mixed with catalytic solid, only the
    catalytic nodes are nodes and the species mass is conserved without
    sticking;
  - body force (Guo forcing): in a periodic box without walls a uniform
    gas accelerates exactly, u_z(t) = g (t + 1/2) (rho g of momentum per
    step, the velocity taken half a step on); a slit driven along z settles
    to a profile whose second differences are exactly -g/nu (the momentum
    balance of the Poiseuille parabola) and which lies within 1% of the
    no-slip parabola u = g/(2 nu) (x - a)(b - x) with the walls halfway
    between the solid and fluid rows (halfway bounce-back leaves an O(nu/h^2)
    slip); and one collision in a uniform box leaves the second moment the
    Guo source must give, rho (u g + g u) added to the BGK relaxation.
"""
import numpy as np
import pytest

from tests.test_oracle_physics import _sine_decay_rate


def test_species_tau(orc):
    nz = 64
    _, w, _ = orc.lattice()
    s = orc.Sim(1, 1, nz, np.zeros(nz, np.uint8), n_species=1, bc=orc.BC_PERIODIC, tau=0.8, p=0.0, pS_R=0.0)
    s.species_tau(0.6)
    z = np.arange(nz)
    s.set_populations(1, w[:, None] * (1 + 0.1 * np.sin(2 * np.pi * z / nz))[None, :])

    def amp():
        return np.abs(np.fft.rfft(s.fields()[1])[1])

    s.step(200)
    a1 = amp()
    s.step(1000)
    a2 = amp()
    D = -np.log(a2 / a1) / 1000 / (2 * np.pi / nz) ** 2
    assert D == pytest.approx((0.6 - 0.5) / 3.0, rel=2e-3)
    # the default is the carrier's tau
    assert _sine_decay_rate(orc, 1, nz, np.zeros(nz, np.uint8), 200, 1000) == pytest.approx(0.1, rel=2e-3)


def _obstacle_box(orc, value, seed=3):
    nx, ny, nz = 10, 8, 12
    mask = orc.geometry(nx, ny, nz, 0, nz, 0.7, 1.5, seed) * value
    return nx, ny, nz, mask.astype(np.uint8)


def test_inert_solid_bounces_species_like_the_carrier(orc):
    nx, ny, nz, mask = _obstacle_box(orc, 2)
    n = nx * ny * nz
    fluid = mask == 0
    rng = np.random.default_rng(1)
    C = np.stack([orc.feq(1.0 + 0.01 * rng.standard_normal(), *(0.02 * rng.standard_normal(3))) for _ in range(n)], 1)
    C *= fluid
    kappa = 0.37
    s = orc.Sim(nx, ny, nz, mask, n_species=1, bc=orc.BC_PERIODIC, p=1.0, pS_R=0.9)
    s.set_populations(0, C)
    s.set_populations(1, kappa * C)
    s.step(150)
    f = s.populations()
    assert np.abs(f[1] - kappa * f[0]).max() <= 1e-14
    o = s.observables()
    assert o["hits_R"] == 0.0 and o["reacted"] == 0.0
    assert np.abs(f[0] - C).max() > 1e-4  # the flow really moved
    # the inert cells are not nodes, and have no active links
    _, node_idx, _, n_nodes = orc.index_maps(nx, ny, nz, mask, True)
    assert n_nodes == 0 and orc.links(nx, ny, nz, mask, True).shape[0] == 0
    # catalytic solid in the same places gives nodes, and other species fields
    s2 = orc.Sim(nx, ny, nz, (mask > 0).astype(np.uint8), n_species=1, bc=orc.BC_PERIODIC, p=1.0, pS_R=0.9)
    s2.set_populations(0, C)
    s2.set_populations(1, kappa * C)
    s2.step(150)
    assert np.abs(s2.populations()[1] - kappa * s2.populations()[0]).max() > 1e-4


def test_mixed_solid_conserves_species_and_hits_only_catalytic(orc):
    nx, ny, nz, m1 = _obstacle_box(orc, 1)
    z = np.arange(nx * ny * nz) // (nx * ny)
    mask = np.where((m1 == 1) & (z >= nz // 2), 2, m1).astype(np.uint8)
    assert (mask == 2).any() and (mask == 1).any()
    _, w, _ = orc.lattice()
    s = orc.Sim(nx, ny, nz, mask, n_species=2, bc=orc.BC_PERIODIC, p=0.5, pS_R=0.0, pS_P=0.0)
    R = w[:, None] * (mask == 0)[None, :] * 0.5
    s.set_populations(1, R)
    o0 = s.observables()
    s.step(120)
    o1 = s.observables(site=True)
    for k in ("M_C", "M_R", "M_P"):
        assert abs(o1[k] - o0[k]) <= 1e-12 * max(o0[k], 1.0), k
    assert o1["hits_R"] > 0
    fi, ni, nf, nn = orc.index_maps(nx, ny, nz, mask, True)
    _, ni1, _, nn1 = orc.index_maps(nx, ny, nz, m1, True)
    b = orc.active_links(nx, ny, nz, mask, True)
    assert nn < nn1 and np.array_equal(ni >= 0, (mask == 1) & (b > 0))
    assert np.all(b[mask == 2] == 0)
    links = orc.links(nx, ny, nz, mask, True)
    assert np.all(mask[links[:, 2]] == 1) and links.shape[0] == b.sum()


def test_body_force_uniform_acceleration(orc):
    nz, g = 6, 2e-6
    s = orc.Sim(3, 2, nz, np.zeros(3 * 2 * nz, np.uint8), n_species=1, bc=orc.BC_PERIODIC, tau=0.7, p=1.0)
    s.body_force(g)
    for t in range(0, 40, 7):
        fl = s.fields()
        assert np.abs(fl[4] - g * (t + 0.5)).max() <= 1e-9 * g * (t + 0.5), t
        assert np.abs(fl[0] - 1.0).max() <= 1e-14
        s.step(7)


@pytest.mark.parametrize("tau", [0.5 + np.sqrt(3) / 4, 0.8, 1.2])
def test_body_force_poiseuille(orc, tau):
    h, nz, g = 16, 4, 1e-6
    nx = h + 2
    mask = np.zeros((nz, 1, nx), np.uint8)
    mask[:, :, 0] = 1
    mask[:, :, nx - 1] = 2
    s = orc.Sim(nx, 1, nz, mask.reshape(-1), n_species=1, bc=orc.BC_PERIODIC, tau=tau, rho_out=1.0, p=1.0)
    s.body_force(g)
    s.step(40000)
    fl = s.fields().reshape(5, nz, 1, nx)
    nu = (tau - 0.5) / 3.0
    u = fl[4][:, 0, 1:nx - 1]
    d2 = u[:, 2:] - 2 * u[:, 1:-1] + u[:, :-2]
    assert np.abs(d2 * nu / g + 1.0).max() <= 1e-9
    x = np.arange(1, nx - 1)
    ref = g / (2 * nu) * (x - 0.5) * (nx - 1.5 - x)
    assert np.abs(u - ref[None, :]).max() <= 1e-2 * ref.max()
    assert np.abs(u - u[:, ::-1]).max() <= 1e-12 * ref.max()
    assert np.abs(fl[2]).max() < 1e-12 and np.abs(fl[3]).max() < 1e-12


def test_guo_source_second_moment(orc):
    # in a uniform periodic box one step is one collision, so the populations'
    # second moment after it is (1 - omega) Pi(f) + omega Pi_eq(u*) +
    # (1 - omega/2) rho (u* g + g u*), u* = u0 + g/2 the forced velocity: the
    # (c.u)(c.F) part of the source makes the last term (without it the
    # source's second moment would be -(u.F) I instead)
    tau, gz, rho = 0.7, 3e-4, 1.1
    omega = 1.0 / tau
    u0 = np.array([0.02, -0.01, 0.015])
    n = 2 * 3 * 4
    s = orc.Sim(2, 3, 4, np.zeros(n, np.uint8), n_species=1, bc=orc.BC_PERIODIC, tau=tau, p=1.0)
    s.body_force(gz)
    f0 = orc.feq(rho, *u0)
    s.set_populations(0, np.repeat(f0[:, None], n, 1))
    s.step(1)
    c, _, _ = orc.lattice()
    c = c.astype(np.float64)
    f1 = s.populations()[0][:, 0]
    pi = np.einsum("qa,qb,q->ab", c, c, f1)
    pi0 = np.einsum("qa,qb,q->ab", c, c, f0)
    g = np.array([0.0, 0.0, gz])
    us = u0 + 0.5 * g
    pi_eq = rho / 3.0 * np.eye(3) + rho * np.outer(us, us)
    want = (1 - omega) * pi0 + omega * pi_eq + (1 - 0.5 * omega) * rho * (np.outer(us, g) + np.outer(g, us))
    assert np.abs(pi - want).max() <= 1e-15
    # and the momentum gained is rho g exactly
    assert np.allclose(np.einsum("qa,q->a", c, f1), rho * (u0 + g), rtol=0, atol=1e-16)
