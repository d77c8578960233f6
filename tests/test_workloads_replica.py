"""The seeded inputs of the two-dimensional reactor replica (Sec. 2.1: pore
disks of 30 nm = 3 lattice units grown at random centres in a centred
rectangle until its porosity is 0.70 +- 0.005):

  - for every ingot of the thickness sweep and both orientations the
    rectangle's porosity lies in the window and everything outside it is
    fluid;
  - every pore cell inside the rectangle has a pore neighbourhood of disk
    size: the 3 x 3 block around it holds at least 4 pore cells (a disk of
    diameter 3 frees at least 4 cells whatever its centre);
  - the draw is reproducible from its seed and changes with it.
"""
import numpy as np
import pytest

import workloads as W

R = W.REPLICA


@pytest.mark.parametrize("orientation", ["perpendicular", "parallel"])
def test_porosity_window_and_outside_fluid(orientation):
    for w in R["w_list"]:
        box = W.ingot_box(R["nx"], R["nz"], R["h"], w, orientation)
        x0, x1, z0, z1 = box
        m = W.disk_ingot(R["nx"], R["nz"], box, porosity=R["porosity"], seed=R["seed"] + w).reshape(R["nz"], R["nx"])
        sub = m[z0:z1, x0:x1]
        phi = 1.0 - sub.mean()
        assert abs(phi - R["porosity"]) <= 0.005, (orientation, w, phi)
        outside = m.copy()
        outside[z0:z1, x0:x1] = 0
        assert outside.sum() == 0
        assert (x1 - x0) * (z1 - z0) == R["h"] * w
        assert z0 >= 2 and z1 <= R["nz"] - 2  # planes 0, 1, nz-2, nz-1 fluid


def test_pores_come_in_disks():
    box = W.ingot_box(R["nx"], R["nz"], R["h"], 30)
    x0, x1, z0, z1 = box
    m = W.disk_ingot(R["nx"], R["nz"], box, seed=3).reshape(R["nz"], R["nx"])
    pore = np.zeros((R["nz"] + 2, R["nx"] + 2), int)
    pore[1:-1, 1:-1] = 1 - m
    for z in range(z0, z1):
        for x in range(x0, x1):
            if not m[z, x]:
                assert pore[z:z + 3, x:x + 3].sum() >= 4, (z, x)


def test_seeded():
    box = W.ingot_box(R["nx"], R["nz"], R["h"], 10)
    a = W.disk_ingot(R["nx"], R["nz"], box, seed=5)
    assert np.array_equal(a, W.disk_ingot(R["nx"], R["nz"], box, seed=5))
    assert not np.array_equal(a, W.disk_ingot(R["nx"], R["nz"], box, seed=6))
