"""Pins of the oracle's barycentric velocity option (Appendix, velocity
equation: u = sum_a rho_a u_a / sum_a rho_a, every array relaxed towards
feq(rho_a, u)):

  - closed form: in a spatially uniform periodic box streaming does nothing,
    and BGK moves each array's momentum linearly, j_a -> j_a + omega (rho_a u
    - j_a), because the second-order equilibrium carries momentum rho_a u
    exactly on D3Q19. The barycentric u is then constant and every array's
    velocity approaches it as (1 - omega)^t; with the carrier's velocity
    instead, the carrier keeps its own and the species approach that;
  - in a closed periodic box with an uneven flow, the total momentum over all
    arrays is conserved and the carrier's alone is not; with the carrier's
    velocity it is the other way round;
  - with no species mass anywhere the two options step bit-identically.
"""
import numpy as np

RHO = (1.0, 0.3, 0.2)
U0 = ((0.01, 0.0, -0.005), (0.03, -0.02, 0.01), (-0.02, 0.015, 0.04))


def _uniform_box(orc, bary):
    nx, ny, nz = 4, 3, 5
    n = nx * ny * nz
    sim = orc.Sim(nx, ny, nz, np.zeros(n, np.uint8), n_species=2, tau=0.8, bc=orc.BC_PERIODIC)
    if bary:
        sim.barycentric()
    for a in range(3):
        sim.set_populations(a, np.repeat(orc.feq(RHO[a], *U0[a])[:, None], n, 1))
    return sim


def _momenta(orc, sim):
    """[3 arrays, 3 components, n cells] momentum and [3, n] density."""
    c, _, _ = orc.lattice()
    f = sim.populations()
    return np.einsum("qi,aqn->ain", c.astype(np.float64), f), f.sum(axis=1)


def test_uniform_box_closed_form(orc):
    omega = 1.0 / 0.8
    rho = np.array(RHO)
    u0 = np.array(U0)
    u_bary = (rho[:, None] * u0).sum(0) / rho.sum()
    for bary in (True, False):
        sim = _uniform_box(orc, bary)
        target = u_bary if bary else u0[0]
        for t in range(1, 9):
            sim.step(1)
            j, r = _momenta(orc, sim)
            assert np.allclose(r, rho[:, None], rtol=0, atol=1e-15)
            g = (1.0 - omega) ** t
            for a in range(3):
                want = target + (u0[a] - target) * g
                if not bary and a == 0:
                    want = u0[0]
                got = j[a] / rho[a]
                assert np.abs(got - want[:, None]).max() < 1e-15, (bary, t, a)
            fl = sim.fields()
            assert np.abs(fl[3:6] - target[:, None]).max() < 1e-15, (bary, t)


def _wavy_box(orc, bary):
    nx, ny, nz = 8, 6, 10
    n = nx * ny * nz
    sim = orc.Sim(nx, ny, nz, np.zeros(n, np.uint8), n_species=2, tau=0.7, bc=orc.BC_PERIODIC)
    if bary:
        sim.barycentric()
    x = np.arange(n) % nx
    z = np.arange(n) // (nx * ny)
    rng = np.random.default_rng(3)
    for a in range(3):
        rho = RHO[a] * (1.0 + 0.05 * np.sin(2 * np.pi * (z + a) / nz))
        ux = 0.02 * (a - 1) * np.cos(2 * np.pi * x / nx) + 0.005 * rng.standard_normal(n)
        uz = 0.01 * (1 - a) * np.sin(2 * np.pi * z / nz)
        f = np.stack([orc.feq(rho[k], ux[k], 0.0, uz[k]) for k in range(n)], 1)
        sim.set_populations(a, f)
    return sim


def test_momentum_budget_closed_box(orc):
    for bary in (True, False):
        sim = _wavy_box(orc, bary)
        j0, r0 = _momenta(orc, sim)
        sim.step(40)
        j1, r1 = _momenta(orc, sim)
        assert np.allclose(r1.sum(1), r0.sum(1), rtol=1e-13, atol=0)  # each array's mass
        tot0, tot1 = j0.sum(axis=(0, 2)), j1.sum(axis=(0, 2))
        car0, car1 = j0[0].sum(1), j1[0].sum(1)
        scale = np.abs(j0).sum()
        if bary:
            assert np.abs(tot1 - tot0).max() < 1e-13 * scale
            assert np.abs(car1 - car0).max() > 1e-4 * scale
        else:
            assert np.abs(car1 - car0).max() < 1e-13 * scale
            assert np.abs(tot1 - tot0).max() > 1e-4 * scale


def test_no_species_mass_is_bit_identical(orc):
    nx, ny, nz = 12, 10, 24
    mask = orc.geometry(nx, ny, nz, 8, 16, 0.6, 1.5, 4)
    out = []
    for bary in (False, True):
        sim = orc.Sim(nx, ny, nz, mask, n_species=2, c_in=0.0, p=0.5)
        if bary:
            sim.barycentric()
        sim.step(30)
        out.append((sim.populations(), sim.fields()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.abs(out[0][0][0] - orc.lattice()[1][:, None] * (~mask.astype(bool))).max() > 1e-6  # the flow moved
