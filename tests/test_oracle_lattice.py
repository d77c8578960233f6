"""Pins of the oracle's lattice, equilibrium, collision and storage rounding.

Each check is fixed by mathematics or by a library routine, not by the
oracle's own formulas:
  - the D3Q19 weights must satisfy the constraints of the paper's Appendix
    (sum w = 1, sum w c = 0, sum w c c = cs^2 I) exactly, in rationals, plus
    the fourth-order isotropy any Navier-Stokes lattice needs;
  - the equilibrium (Appendix, Eq. feq) must reproduce its defining moments
    rho, rho u and rho cs^2 I + rho u u;
  - BGK collision (Appendix, Eq. LBE) must conserve carrier mass and momentum;
  - the FP16/BF16 storage emulation must agree with numpy's float16 and
    torch's bfloat16 round-to-nearest-even conversions.
"""
from fractions import Fraction

import numpy as np
import pytest


def test_lattice_constraints_exact(orc):
    c, w, opp = orc.lattice()
    assert c.shape == (19, 3)
    # distinct speeds: 1 rest, 6 of |c|^2 = 1, 12 of |c|^2 = 2
    assert len({tuple(v) for v in c}) == 19
    norms = sorted((c * c).sum(1).tolist())
    assert norms == [0] + [1] * 6 + [2] * 12
    W = [Fraction(x).limit_denominator(1000) for x in w]
    assert all(abs(float(Wi) - wi) < 1e-16 for Wi, wi in zip(W, w))
    assert sum(W) == 1
    for a in range(3):
        assert sum(Wi * int(ci[a]) for Wi, ci in zip(W, c)) == 0
        for b in range(3):
            s = sum(Wi * int(ci[a]) * int(ci[b]) for Wi, ci in zip(W, c))
            assert s == (Fraction(1, 3) if a == b else 0)
    # fourth-order isotropy: sum w c_a c_b c_c c_d = cs^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    d = lambda i, j: 1 if i == j else 0
    for a in range(3):
        for b in range(3):
            for e in range(3):
                for g in range(3):
                    s = sum(Wi * int(ci[a]) * int(ci[b]) * int(ci[e]) * int(ci[g]) for Wi, ci in zip(W, c))
                    assert s == Fraction(1, 9) * (d(a, b) * d(e, g) + d(a, e) * d(b, g) + d(a, g) * d(b, e))
    # opposite directions
    for i in range(19):
        assert (c[opp[i]] == -c[i]).all()
        assert opp[opp[i]] == i


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(orc, seed):
    rng = np.random.default_rng(seed)
    c, w, _ = orc.lattice()
    rho = rng.uniform(0.2, 2.0)
    u = rng.uniform(-0.1, 0.1, 3)
    f = orc.feq(rho, *u)
    assert abs(f.sum() - rho) <= 1e-15 * rho * 4
    np.testing.assert_allclose(c.T @ f, rho * u, rtol=0, atol=1e-15 * rho * 8)
    P = (c[:, :, None] * c[:, None, :] * f[:, None, None]).sum(0)
    np.testing.assert_allclose(P, rho / 3 * np.eye(3) + rho * np.outer(u, u), rtol=0, atol=1e-15 * rho * 8)


def test_collision_conserves_carrier_mass_and_momentum(orc):
    # fully fluid periodic box with random positive populations: one step
    nx, ny, nz = 6, 5, 4
    n = nx * ny * nz
    rng = np.random.default_rng(7)
    mask = np.zeros(n, np.uint8)
    sim = orc.Sim(nx, ny, nz, mask, n_species=2, bc=orc.BC_PERIODIC)
    c, w, _ = orc.lattice()
    f0 = w[:, None] * rng.uniform(0.8, 1.2, (19, n))
    sim.set_populations(0, f0)
    sim.set_populations(1, w[:, None] * rng.uniform(0.0, 1.0, (19, n)))
    m0 = f0.sum()
    j0 = c.T @ f0.sum(1)
    sim.step(3)
    f = sim.populations()[0]
    assert abs(f.sum() - m0) < 1e-12 * m0
    np.testing.assert_allclose(c.T @ f.sum(1), j0, rtol=0, atol=1e-12 * m0)


def test_fp16_rounding_matches_numpy(orc):
    rng = np.random.default_rng(3)
    vals = np.concatenate([
        rng.standard_normal(4000) * 10.0 ** rng.integers(-9, 4, 4000),
        # exact halfway cases between float16 neighbours, both parities
        (1.0 + (2 * np.arange(1, 200) + 1) * 2.0 ** -11),
        -(1.0 + (2 * np.arange(1, 200)) * 2.0 ** -11 + 2.0 ** -11),
        np.array([2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 6.1e-5, 65504.0, 0.0, -0.0]),
    ])
    for v in vals:
        ref = float(np.float64(v).astype(np.float16))
        got = orc.round_fp16(float(v))
        assert got == ref, (v, got, ref)


def test_bf16_rounding_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    # values exactly representable in fp32, so torch's fp32->bf16 RNE is the reference
    vals = (rng.standard_normal(4000) * 10.0 ** rng.integers(-20, 6, 4000)).astype(np.float32)
    ties = (1.0 + (2 * np.arange(1, 100) + 1) * 2.0 ** -8).astype(np.float32)
    vals = np.concatenate([vals, ties, -ties])
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([orc.round_bf16(float(v)) for v in vals])
    np.testing.assert_array_equal(got, ref)
