"""Pins of the oracle's random sputtering matrix (Appendix, the random S_ij of
Eq. f_P_in, read as one-hot columns):

  - every draw is one of the node's active links, and the draws are uniform
    over them (binomial bounds on many keys);
  - on a single catalytic node with 18 fluid neighbours, every incoming
    population comes back whole along the link drawn for it, and the
    emissions add up to what arrived (unit column sums);
  - mass: R and P are each conserved when nothing sticks, R + P when p = 1
    and the product never sticks, as with the uniform matrix;
  - the ensemble mean over seeds of the emitted populations is the uniform
    matrix's 1/b share, within the binomial spread.
"""
import numpy as np
import pytest

from tests.test_oracle_physics import _closed_box


def test_draw_is_an_active_link_and_uniform(orc):
    rng = np.random.default_rng(5)
    masks = [sum(1 << i for i in range(1, 19)), (1 << 3), (1 << 2) | (1 << 7) | (1 << 18)]
    masks += [int(sum(1 << i for i in range(1, 19) if rng.random() < 0.4)) | (1 << 1) for _ in range(3)]
    for m in masks:
        active = [i for i in range(1, 19) if (m >> i) & 1]
        counts = {i: 0 for i in active}
        draws = 0
        for cell in range(0, 4000, 7):
            for j in (1, 6, 11, 18):
                k = orc.rs_choice(99, cell, j, cell % 13, m)
                assert k in counts, (m, k)
                counts[k] += 1
                draws += 1
        b = len(active)
        mean = draws / b
        sd = np.sqrt(draws * (1 / b) * (1 - 1 / b))
        for i, n in counts.items():
            assert abs(n - mean) <= 5 * sd + 1, (m, i, n, mean)
    # no active link: no draw; the same key gives the same draw
    assert orc.rs_choice(1, 5, 3, 2, 0) == 0
    assert orc.rs_choice(3, 1234, 5, 77, masks[0]) == orc.rs_choice(3, 1234, 5, 77, masks[0])
    seq = lambda seed: [orc.rs_choice(seed, c, 4, 0, masks[0]) for c in range(64)]
    assert seq(1) != seq(2)


def _single_node(orc, seed, pS_R, pS_P, p, rhoP0):
    nx = ny = nz = 5
    n = nx * ny * nz
    mask = np.zeros(n, np.uint8)
    s = (2 * ny + 2) * nx + 2
    mask[s] = 1
    sim = orc.Sim(nx, ny, nz, mask, n_species=2, p=p, pS_R=pS_R, pS_P=pS_P, bc=orc.BC_PERIODIC)
    sim.random_sputtering(seed)
    c, w, _ = orc.lattice()
    R = np.repeat(w[:, None], n, 1) * 1.0
    P = np.repeat(w[:, None], n, 1) * rhoP0
    R[:, s] = 0
    P[:, s] = 0
    sim.set_populations(1, R)
    sim.set_populations(2, P)
    sim.step(1)
    return sim, s, c, w


@pytest.mark.parametrize("seed,pS_R,pS_P,p", [(3, 0.95, 0.0, 0.45), (4, 0.3, 0.2, 0.7), (5, 0.0, 0.0, 1.0)])
def test_single_node_one_hot_columns(orc, seed, pS_R, pS_P, p):
    # fluid at rest: the neighbour s - c_j sends w_j rho along c_j; the node
    # re-emits it whole along the drawn link k(j) into cell s + c_k as
    # population k
    rhoP0 = 0.5
    sim, s, c, w = _single_node(orc, seed, pS_R, pS_P, p, rhoP0)
    f = sim.populations()
    nx = ny = 5
    full = sum(1 << i for i in range(1, 19))
    gotR = np.zeros(19)
    gotP = np.zeros(19)
    for j in range(1, 19):
        k = orc.rs_choice(seed, s, j, 0, full)
        gotR[k] += w[j] * 1.0
        gotP[k] += w[j] * rhoP0
    for i in range(1, 19):
        x, y, z = 2 + c[i][0], 2 + c[i][1], 2 + c[i][2]
        cell = (z * ny + y) * nx + x
        assert f[1, i, cell] == pytest.approx((1 - pS_R) * gotR[i], abs=1e-16)
        assert f[2, i, cell] == pytest.approx(p * pS_R * gotR[i] + (1 - pS_P) * gotP[i], abs=1e-16)
    emitted = sum(f[1, i, (2 + c[i][2]) * 25 + (2 + c[i][1]) * 5 + 2 + c[i][0]] for i in range(1, 19))
    assert emitted == pytest.approx((1 - pS_R) * 2 / 3, rel=1e-14)  # unit column sums
    assert sim.observables()["hits_R"] == pytest.approx(2 / 3, rel=1e-14)


def test_conservation_no_sticking(orc):
    sim = _closed_box(orc, 21, p=0.6, pS_R=0.0, pS_P=0.0)
    sim.random_sputtering(8)
    o0 = sim.observables()
    sim.step(60)
    o1 = sim.observables()
    for k in ("M_C", "M_R", "M_P"):
        assert abs(o1[k] - o0[k]) < 1e-12 * o0[k], k
    assert o1["hits_R"] > 0


def test_conservation_full_conversion(orc):
    sim = _closed_box(orc, 22, p=1.0, pS_R=0.95, pS_P=0.0)
    sim.random_sputtering(9)
    o0 = sim.observables()
    sim.step(60)
    o1 = sim.observables()
    rp0, rp1 = o0["M_R"] + o0["M_P"], o1["M_R"] + o1["M_P"]
    assert abs(rp1 - rp0) < 1e-12 * rp0
    assert o1["M_R"] < 0.5 * o0["M_R"]


def test_ensemble_mean_is_the_uniform_matrix(orc):
    # per direction i the emission is sum_j w_j [k(j) = i]: mean sum_j w_j / 18
    # = (2/3) / 18, variance sum_j w_j^2 (1/18)(17/18) per draw set
    c, w, _ = orc.lattice()
    K = 300
    acc = np.zeros(19)
    for seed in range(K):
        sim, s, c, w = _single_node(orc, 1000 + seed, 0.0, 0.0, 1.0, 0.0)
        f = sim.populations()
        for i in range(1, 19):
            acc[i] += f[1, i, (2 + c[i][2]) * 25 + (2 + c[i][1]) * 5 + 2 + c[i][0]]
    mean = acc[1:] / K
    sd = np.sqrt((w[1:] ** 2).sum() * (1 / 18) * (17 / 18) / K)
    assert np.all(np.abs(mean - (2 / 3) / 18) < 5 * sd)
    assert abs(mean.sum() - 2 / 3) < 1e-13  # every draw set returns all the mass
