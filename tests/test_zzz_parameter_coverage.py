"""GPU parity over parameters the other cases leave at their defaults (rho0, moving walls, the
inlet profile's origin and height), against the oracle with the tolerances of
`test_gpu_parity.py`."""
import pytest

import oracle
from paper_1907_04034_gb300 import binding, cases
from test_gpu_parity import PRECS, _compare_window, compare_eval


@pytest.fixture(scope="module", autouse=True)
def _built():
    binding.build()
    yield


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECS)
def test_density_scale_moving_walls_and_a_shifted_inlet_profile(prec):
    """Parameters the other cases leave at their defaults: rho0 = 1000 (masses, pressures and
    p_b scaled with it) on the gated pulse channel whose inlet profile carries two modes
    measured from y0 = -0.15 over H = 0.8; and a Poiseuille channel between no-slip walls
    moving at (0.25, -0.1).  One evaluation and a window of steps against the oracle."""
    c = cases.channel(pulse_amp=1.0, pulse_xy=(0.8, 0.25))
    k = 1000.0
    c.params.rho0 *= k
    c.params.pb *= k
    c.m = c.m * k
    c.p = c.p * k
    c.params.inlet_modes = (0.03, -0.02)
    c.params.inlet_y0 = -0.15
    c.params.inlet_h = 0.8
    w = cases.poiseuille(n=12)
    w.params.wall_u = (0.25, 0.0)
    w.params.wall_v = (-0.1, 0.0)
    for case, n in ((c, 40), (w, 40)):
        ref = oracle.OracleSim(case)
        s = binding.Solver(case, precision=prec)
        compare_eval(s, ref, prec)
        ref.step(n)
        s.step(n)
        _compare_window(s, ref, prec)
        s.close()
