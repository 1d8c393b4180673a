"""Host-side parts of the gradient module: the pressure-energy window weight, the window in
front of the outlet, and the copy of a case with other inlet modes."""
import numpy as np
import pytest

from paper_1907_04034_gb300 import cases, gradient


def test_window_weight_vanishes_smoothly_at_both_edges():
    x0, x1 = 2.0, 3.0
    x = np.array([1.0, 2.0, 2.25, 2.5, 2.75, 3.0 - 1e-12, 3.0, 4.0])
    w = gradient.window_weight(x, x0, x1)
    np.testing.assert_allclose(w, [0.0, 0.0, 0.5, 1.0, 0.5, 0.0, 0.0, 0.0], atol=1e-20)
    # continuous (and with zero slope) at the edges: tiny steps inside give tiny weights
    assert gradient.window_weight(x0 + 1e-6, x0, x1) < 1e-10
    assert gradient.window_weight(x1 - 1e-6, x0, x1) < 1e-10


def test_pressure_energy_window_is_the_layer_in_front_of_the_outlet():
    c = cases.cylinder(dx=1.0 / 25.0)
    x0, x1 = gradient.pressure_energy_window(c)
    assert x1 == c.params.x_out
    assert x1 - x0 == pytest.approx(6.0 * c.params.hdx * c.params.dx)  # two support radii


def test_case_with_other_modes_sets_the_profile_and_leaves_the_original():
    c = cases.cylinder(dx=1.0 / 25.0)
    a = np.zeros(gradient.N_MODES)
    a[0] = 0.05
    d = gradient._with_modes(c, a)
    assert c.params.inlet_modes == () and np.all(c.u[c.tag == cases.INLET] == c.params.U)
    assert d.params.inlet_modes[0] == 0.05 and len(d.params.inlet_modes) == gradient.N_MODES
    sel = d.tag == cases.INLET
    y = (d.y[sel] - d.params.inlet_y0) / d.params.inlet_h
    np.testing.assert_allclose(d.u[sel], d.params.U + 0.05 * np.sin(np.pi * y), rtol=0, atol=1e-14)
    assert np.array_equal(d.u[~sel], c.u[~sel])
