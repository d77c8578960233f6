"""The host-side analysis of the Lévêque study (Appendix, validation), no GPU:

  - the reference gradient follows from Lévêque's similarity solution, here
    rebuilt independently: c/c_in = int_0^eta exp(-s^3) ds / int_0^inf
    exp(-s^3) ds with eta = y (gamma / (9 D x))^(1/3), gamma = 4 U_max / L_y
    the wall shear of the Poiseuille profile; its wall slope, made
    dimensionless with L_y, must equal leveque_gradients' G_L at every node;
  - the measured gradient is the wall flux over D, in units of c_in / L_y: a
    site map of D / L_y per node gives G = 1;
  - the comparison window lies inside the plate.
"""
import numpy as np
import pytest

import workloads


def test_reference_gradient_is_the_similarity_solution():
    from scipy.integrate import quad

    from paper_1607_02874_gb300 import studies

    c = workloads.LEVEQUE
    D = (c["tau_s"] - 0.5) / 3.0
    u_max = c["Pe"] * D / c["L_y"]
    gamma = 4.0 * u_max / c["L_y"]
    norm, _ = quad(lambda s: np.exp(-s ** 3), 0.0, np.inf)
    x = np.arange(c["L"]) + 0.5
    # d(c/c_in)/dy at y = 0 is (gamma / (9 D x))^(1/3) / norm; times L_y
    ref = c["L_y"] * (gamma / (9.0 * D * x)) ** (1.0 / 3.0) / norm
    _, GL = studies.leveque_gradients(np.zeros(c["L"]))
    assert np.allclose(GL, ref, rtol=1e-10)


def test_measured_gradient_units():
    from paper_1607_02874_gb300 import studies

    c = workloads.LEVEQUE
    D = (c["tau_s"] - 0.5) / 3.0
    G, _ = studies.leveque_gradients(np.full(c["L"] + 3, D / c["L_y"]))
    assert G.shape == (c["L"],) and np.allclose(G, 1.0, rtol=1e-12)


def test_window_inside_the_plate():
    from paper_1607_02874_gb300 import studies

    a, b = studies.LEVEQUE_WINDOW
    assert 0 < a < b < workloads.LEVEQUE["L"]
    assert workloads.leveque_force() == pytest.approx(
        8 * (workloads.LEVEQUE["tau"] - 0.5) / 3 * 253.0 * (0.05 / 3) / 50 / 50 ** 2, rel=1e-12)
