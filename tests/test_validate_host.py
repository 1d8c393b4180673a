"""Host-side analysis of the long-run physics driver (`validate.py`), on synthetic signals
whose coefficients are known: the drag and lift coefficients and the Strouhal number that
the Table clcd and Table hybridconv tests compare, and the L2 error of Eq. l2norm."""
import math

import numpy as np
import pytest

from paper_1907_04034_gb300 import validate


def test_moving_average_keeps_constants_and_lines():
    a = np.full(50, 2.5)
    np.testing.assert_allclose(validate.moving_average(a), a, rtol=1e-15)
    b = 0.3 * np.arange(50) - 1.0
    m = validate.moving_average(b)
    np.testing.assert_allclose(m[2:-2], b[2:-2], rtol=0, atol=1e-13)  # centred: exact inside
    assert m[0] == pytest.approx(np.mean(b[:3]))  # the ends average the available points


@pytest.mark.parametrize("St,cd,cl,D,U,rho0", [(0.2, 1.5, 0.72, 1.0, 1.0, 1.0),
                                               (0.21, 1.32, 0.4, 2.0, 1.0, 1000.0)])
def test_coefficients_of_a_synthetic_shedding_history(St, cd, cl, D, U, rho0):
    """Forces F_x = q (c_d + 0.02 sin 2wt), F_y = q c_l sin(wt + 0.3), q = rho0 U^2 D / 2,
    w = 2 pi St U / D, sampled every step of a 75 D/U run: the mean drag, the lift amplitude
    (least-squares sinusoid) and St (the lift spectrum's peak) come back."""
    dt = 0.002 * D / U
    n = int(75 * D / U / dt)
    t = (np.arange(n) + 1) * dt
    w = 2 * math.pi * St * U / D
    q = 0.5 * rho0 * U * U * D
    fx = q * (cd + 0.02 * np.sin(2 * w * t))
    fy = q * cl * np.sin(w * t + 0.3)
    out = validate.coefficients(fx, fy, dt, D, U, rho0, t_from=45 * D / U)
    assert out["cd_mean"] == pytest.approx(cd, abs=2e-3)
    assert out["cl_amp_fit"] == pytest.approx(cl, rel=1e-2)
    assert out["St"] == pytest.approx(St, rel=1e-2)
    # the mean of a sinusoid over a window of 30 St periods is at most its amplitude / (pi periods)
    assert abs(out["cl_mean"]) < cl / (math.pi * 30 * St)
    assert out["window"][0] == pytest.approx(45 * D / U, abs=dt)


def test_coefficients_reject_a_short_window():
    with pytest.raises(ValueError):
        validate.coefficients(np.ones(100), np.zeros(100), 0.01, 1.0, 1.0, 1.0, t_from=0.95)


def test_l2_error_of_a_scaled_and_of_a_shifted_signal():
    """Eq. l2norm: a signal scaled by 1 + e has error |e|; one with an added constant c has
    error |c| sqrt(n / sum f^2)."""
    f = np.sin(np.linspace(0.0, 7.0, 400)) + 0.1
    assert validate.l2_error(1.03 * f, f) == pytest.approx(0.03, rel=1e-12)
    assert validate.l2_error(f + 0.01, f) == pytest.approx(0.01 * math.sqrt(len(f) / np.sum(f * f)),
                                                            rel=1e-12)
    assert validate.l2_error(f, f) == 0.0
