"""Pins of the oracle's synthetic geometry and derived integer structures.

  - SplitMix64 against its published output sequence (seed 0);
  - the white noise against the Irwin-Hall moments;
  - the box-filtered field against scipy's periodic integer convolution;
  - the threshold against a brute-force sort on (value, index);
  - b(x), the fluid / interface-node numbering, the link list and the mean
    chord length against brute-force numpy/Python re-derivations written
    from their definitions (the paper's Appendix defines b(x) as the number
    of active links of a node; every solid node touching gas is catalytic).
"""
import itertools

import numpy as np
import pytest

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def test_splitmix64_published_vectors(orc):
    gamma = 0x9E3779B97F4A7C15
    # first three outputs of SplitMix64 seeded with 0
    assert orc.splitmix64(0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(gamma) == 0x6E789E6AA1B965F4
    assert orc.splitmix64((2 * gamma) % 2 ** 64) == 0x06C45D188009454F


def test_noise_moments(orc):
    v = np.array([orc.noise(123, k) for k in range(40000)], np.float64)
    # sum of 12 U{0..65535} minus 12 * 32768: mean -6, variance 12 (65536^2 - 1) / 12
    var = 65536.0 ** 2 - 1
    assert abs(v.mean() + 6.0) < 4 * np.sqrt(var / v.size)
    assert abs(v.var() / var - 1.0) < 0.03
    assert v.min() >= -12 * 32768 and v.max() <= 12 * 32767


@pytest.mark.parametrize("l,W", [(6, 9), (10, 15), (14, 19), (20, 29), (4, 5), (16, 23)])
def test_box_width(orc, l, W):
    assert orc.box_width(float(l)) == W
    # odd, and the closest odd integer to sqrt(2 l^2 + 1) (3-pass variance 3 (W^2-1)/12 ~ l^2/2)
    t = np.sqrt(2 * l * l + 1)
    assert W % 2 == 1 and all(abs(W - t) <= abs(k - t) for k in range(1, 200, 2))


def test_field_is_periodic_box_filtered_noise(orc):
    nx, ny, nz, l, seed = 12, 10, 14, 3.0, 99
    W = orc.box_width(l)
    noise = np.array([orc.noise(seed, k) for k in range(nx * ny * nz)], np.int64).reshape(nz, ny, nx)
    ref = noise.copy()
    k = np.ones(W, np.int64)
    for axis in (2, 1, 0):  # x, y, z
        for _ in range(3):
            ref = scipy_ndimage.convolve1d(ref, k, axis=axis, mode="wrap")
    got = orc.field(nx, ny, nz, l, seed).reshape(nz, ny, nx)
    np.testing.assert_array_equal(got, ref)


def test_threshold_brute_force(orc):
    nx, ny, nz, z0, z1, phi, l, seed = 10, 9, 16, 4, 12, 0.62, 2.0, 5
    fld = orc.field(nx, ny, nz, l, seed)
    plane = nx * ny
    idx = np.arange(z0 * plane, z1 * plane)
    order = np.lexsort((idx, fld[idx]))  # by value, then index
    K = int(np.round(phi * idx.size))  # numpy rounds half to even
    ref = np.zeros(nx * ny * nz, np.uint8)
    ref[idx] = 1
    ref[idx[order[:K]]] = 0
    got = orc.geometry(nx, ny, nz, z0, z1, phi, l, seed)
    np.testing.assert_array_equal(got, ref)
    assert orc.fluid_count(phi, idx.size) == K


def test_config1_fluid_count(orc):
    # 32x32x64, slab z in [16, 48), porosity 0.65: 32768 slab cells,
    # round(0.65 * 32768 = 21299.2) = 21299 fluid in the slab
    m = orc.geometry(32, 32, 64, 16, 48, 0.65, 6.0, 1)
    assert int((m == 0).sum()) == 32768 + 21299
    assert m[: 16 * 1024].sum() == 0 and m[48 * 1024:].sum() == 0


def _random_mask(rng, nx, ny, nz, frac=0.35):
    return (rng.random(nx * ny * nz) < frac).astype(np.uint8)


def _shift(m3, c, sgn, zper):
    """value of m3 at (cell + sgn * c); out of z range -> fluid-less (solid=2 marker)."""
    cx, cy, cz = (int(v) for v in c)
    out = np.roll(m3, shift=(-sgn * cz, -sgn * cy, -sgn * cx), axis=(0, 1, 2)).copy()
    if not zper and cz != 0:
        nz = m3.shape[0]
        z = np.arange(nz) + sgn * cz
        out[(z < 0) | (z >= nz)] = 2
    return out


@pytest.mark.parametrize("zper", [False, True])
@pytest.mark.parametrize("seed", [1, 2])
def test_structures_brute_force(orc, zper, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = 7, 6, 9
    mask = _random_mask(rng, nx, ny, nz)
    m3 = mask.reshape(nz, ny, nx)
    c, _, _ = orc.lattice()
    # b(s): fluid cells at s - c_j, j != 0
    b = np.zeros_like(m3, dtype=np.int32)
    for j in range(1, 19):
        b += (_shift(m3, c[j], -1, zper) == 0)
    b = np.where(m3 == 1, b, 0).reshape(-1)
    np.testing.assert_array_equal(orc.active_links(nx, ny, nz, mask, zper), b)
    fi, ni, nf, nn = orc.index_maps(nx, ny, nz, mask, zper)
    ref_fi = np.where(mask == 0, np.cumsum(mask == 0) - 1, -1)
    iface = (mask == 1) & (b > 0)
    ref_ni = np.where(iface, np.cumsum(iface) - 1, -1)
    np.testing.assert_array_equal(fi, ref_fi)
    np.testing.assert_array_equal(ni, ref_ni)
    assert nf == int((mask == 0).sum()) and nn == int(iface.sum())
    # link list: (fluid cell, i, target) for every solid target, cell-major then i
    ref_links = []
    for cell in range(mask.size):
        if mask[cell]:
            continue
        z, y, x = cell // (nx * ny), (cell // nx) % ny, cell % nx
        for i in range(1, 19):
            zz = z + c[i][2]
            if not zper and not (0 <= zz < nz):
                continue
            t = ((zz % nz) * ny + (y + c[i][1]) % ny) * nx + (x + c[i][0]) % nx
            if mask[t]:
                ref_links.append((cell, i, t))
    np.testing.assert_array_equal(orc.links(nx, ny, nz, mask, zper), np.array(ref_links, np.int64).reshape(-1, 3))


def _runs_periodic(line):
    if all(v == 0 for v in line):
        return 1
    if all(v == 1 for v in line):
        return 0
    # rotate so the line starts right after a solid cell, then count fluid groups
    k = int(np.argmax(np.asarray(line) == 1))
    rot = list(line[k:]) + list(line[:k])
    return sum(1 for key, _ in itertools.groupby(rot) if key == 0)


def _runs_open(line):
    return sum(1 for key, _ in itertools.groupby(line) if key == 0)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_chord_length_brute_force(orc, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz, z0, z1 = 8, 7, 10, 2, 8
    mask = _random_mask(rng, nx, ny, nz, 0.4)
    mask.reshape(nz, ny, nx)[3, 2, :] = 0  # a fully fluid periodic row
    m3 = mask.reshape(nz, ny, nx)[z0:z1]
    runs = 0
    for z in range(m3.shape[0]):
        for y in range(ny):
            runs += _runs_periodic(m3[z, y, :].tolist())
        for x in range(nx):
            runs += _runs_periodic(m3[z, :, x].tolist())
    for y in range(ny):
        for x in range(nx):
            runs += _runs_open(m3[:, y, x].tolist())
    nf = int((m3 == 0).sum())
    assert orc.chord_length(nx, ny, nz, z0, z1, mask) == pytest.approx(3 * nf / runs, rel=1e-15)
