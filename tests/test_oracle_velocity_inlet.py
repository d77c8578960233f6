"""Pins of the oracle's velocity inlet (Sec. 3: carrier and reactant injected
at a constant speed U_in with fixed densities; here the inlet plane's
equilibria take the velocity (0, 0, u_in)):

  - with no solid and equal inlet and outlet densities, uniform plug flow
    feq(rho, U_in) is a fixed point of streaming and collision; a column
    started at rest converges to it: carrier density rho_in, u_z = U_in and
    reactant density c_in at every interior cell, to rounding, with either
    velocity option;
  - the carrier inflow per step is then rho_in U_in per cell of the inlet
    face, the first moment of the inlet equilibrium;
  - the pressure inlet at equal densities drives nothing: the column stays
    at rest.
"""
import numpy as np
import pytest

RHO, C_IN, U_IN = 0.8, 0.2, 0.08


def _column(orc, *, vel, bary=False, nx=1, ny=1, nz=40):
    n = nx * ny * nz
    s = orc.Sim(nx, ny, nz, np.zeros(n, np.uint8), n_species=2, tau=0.8, rho_in=RHO, rho_out=RHO, c_in=C_IN,
                p=0.5)
    if vel:
        s.velocity_inlet(U_IN)
    if bary:
        s.barycentric()
    return s


@pytest.mark.parametrize("bary", [False, True], ids=["carrier-u", "barycentric-u"])
def test_plug_flow_steady_state(orc, bary):
    nx, ny, nz = 2, 3, 40
    s = _column(orc, vel=True, bary=bary, nx=nx, ny=ny, nz=nz)
    s.step(4000)
    fl = s.fields()
    z = np.arange(nx * ny * nz) // (nx * ny)
    inner = (z > 0) & (z < nz - 1)
    assert np.abs(fl[0][inner] - RHO).max() < 1e-13
    assert np.abs(fl[1][inner] - C_IN).max() < 1e-13
    assert np.abs(fl[2][inner]).max() == 0.0
    assert np.abs(fl[3][inner]).max() < 1e-15 and np.abs(fl[4][inner]).max() < 1e-15
    assert np.abs(fl[5][inner] - U_IN).max() < 1e-13
    a = s.observables()["in_C"]
    s.step(100)
    b = s.observables()["in_C"]
    assert (b - a) / 100 == pytest.approx(RHO * U_IN * nx * ny, rel=1e-11)


def test_pressure_inlet_at_equal_densities_stays_at_rest(orc):
    s = _column(orc, vel=False)
    s.step(500)
    fl = s.fields()
    assert np.abs(fl[5][1:-1]).max() < 1e-15
    assert np.abs(fl[0][1:-1] - RHO).max() < 1e-15
