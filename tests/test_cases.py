"""The seeded input generators (`cases.py`) against the recipes the workloads state: particle
counts and zones, spacings, the initial fields, the cylinder's ring fill, the batched
workload's distributions, the time-step rule, and reproducibility from the seed."""
import math

import numpy as np
import pytest

from paper_1907_04034_gb300 import cases
from paper_1907_04034_gb300.cases import FLUID, INLET, OUTLET, SLIPWALL, WALL


def test_channel_workload():
    c = cases.channel()
    p = c.params
    assert (c.count(FLUID), c.count(INLET), c.count(OUTLET)) == (1250, 75, 125)
    assert p.dx == 0.02 and p.hdx == 1.2 and p.cs == 10.0 and p.nu == 0.01 and p.periodic_y
    assert p.dt == pytest.approx(min(0.25 * p.h / (p.cs + p.U), 0.125 * p.h ** 2 / p.nu))
    fl = c.tag == FLUID
    # fluid on the lattice (x, y) = ((i + 1/2) dx, (j + 1/2) dx) within +-0.01 dx
    for v in (c.x[fl], c.y[fl]):
        off = (v / p.dx - 0.5) - np.round(v / p.dx - 0.5)
        off = np.where(off > 0.5, off - 1.0, off)
        assert np.abs(off).max() <= 0.0100001 and np.abs(off).max() > 0.005
    assert np.all(c.x[c.tag == INLET] < p.x_in) and np.all(c.x[c.tag == OUTLET] > p.x_out)
    np.testing.assert_allclose(c.p, 0.1 * np.exp(-((c.x - 0.5) ** 2 + (c.y - 0.25) ** 2) / 0.005))
    assert np.all(c.u == 1.0) and np.all(c.v == 0.0) and np.all(c.m == p.rho0 * p.dx ** 2)
    assert np.array_equal(c.id, np.arange(c.n))
    d = cases.channel()
    assert np.array_equal(c.x, d.x) and np.array_equal(c.y, d.y)  # seeded


@pytest.mark.parametrize("dod", [25.0, 40.0])
def test_cylinder_workload(dod):
    dx = 1.0 / dod
    c = cases.cylinder(dx=dx)
    p = c.params
    assert p.nu == pytest.approx(1.0 / 200.0) and p.drag_length == 1.0
    xc, yc, R = 5.0, 5.0, 0.5
    fl = c.tag == FLUID
    r = np.hypot(c.x - xc, c.y - yc)
    assert r[fl].min() >= R + 0.5 * dx
    # three solid rings at R - k dx with round(2 pi r / dx) points each
    sol = c.tag == WALL
    radii = R - dx * np.arange(3)
    assert c.count(WALL) == sum(int(round(2 * math.pi * q / dx)) for q in radii)
    assert np.all(np.min(np.abs(r[sol][:, None] - radii[None, :]), axis=1) < 1e-12)
    # slip walls: 4 layers below y = 0 and above y = 10
    sw = c.tag == SLIPWALL
    assert np.all((c.y[sw] < 0.0) | (c.y[sw] > 10.0))
    assert len(np.unique(np.round(c.y[sw] / dx, 6))) == 8
    assert c.count(INLET) == 3 * round(10.0 / dx) and c.count(OUTLET) == 5 * round(10.0 / dx)
    assert np.all(c.u[fl] == 1.0) and np.all(c.u[sol | sw] == 0.0) and np.all(c.p == 0.0)


def test_batched_workload_distributions_and_seed():
    b = cases.batch_channels(n=64, seed=0)
    assert len(b) == 64
    n_fl = np.array([c.count(FLUID) for c in b])
    dxs = np.array([c.params.dx for c in b])
    re = np.array([c.params.U * (c.params.y_max - c.params.y_min) / c.params.nu for c in b])
    assert n_fl.min() >= 1500 and n_fl.max() <= 61000  # N ~ U[2k, 60k], rounded to whole rows
    assert dxs.min() >= 0.005 and dxs.max() <= 0.03
    assert re.min() >= 50.0 - 1e-9 and re.max() <= 500.0 + 1e-9
    for c in b:
        H = c.params.y_max - c.params.y_min
        L = c.params.x_out - c.params.x_in
        assert L == pytest.approx(2 * H, rel=0.05)
    b2 = cases.batch_channels(n=64, seed=0)
    assert all(np.array_equal(a.x, d.x) and a.params.nu == d.params.nu for a, d in zip(b, b2))
    b3 = cases.batch_channels(n=64, seed=1)
    assert any(a.n != d.n for a, d in zip(b, b3))


def test_outlet_problems_and_pressure_bump():
    for prob, W in (("pulse2d", 2.0), ("ramp", 2.0), ("vortex", 4.0)):
        c = cases.outlet_problem(prob)
        p = c.params
        assert p.nu == 0.0 and p.dx == 0.1 and p.x_out == 2.0 and p.inlet_h == W
        fl = c.tag == FLUID
        assert c.count(FLUID) == round(2.0 / 0.1) * round(W / 0.1)
        assert np.all(c.u[fl] == (0.0 if prob == "ramp" else 1.0))
        long = cases.outlet_problem(prob, long=True)
        assert long.params.x_out == pytest.approx(1.7 + 10.0 * 3.0)  # d + c t_end
    b = cases.pressure_bump()
    fl = b.tag == FLUID
    np.testing.assert_allclose(b.p[fl], 1e-3 * (1 - 0.2 * np.exp(-(b.x[fl] - 0.5) ** 2 / 0.001)))
    assert np.all(b.p[~fl] == 1e-3) and b.params.x_in == 0.0 and b.params.x_out == 1.0
    bl = cases.pressure_bump(long=True)
    assert bl.params.x_in <= -(10.0 - 1.0) * 0.3 and bl.params.x_out >= 1.0 + 11.0 * 0.3


def test_taylor_green_and_poiseuille():
    c = cases.taylor_green(n=20)
    k = 2 * math.pi
    np.testing.assert_allclose(c.u, -np.cos(k * c.x) * np.sin(k * c.y))
    np.testing.assert_allclose(c.v, np.sin(k * c.x) * np.cos(k * c.y))
    assert c.params.periodic_x and c.params.periodic_y and c.n == 400
    q = cases.poiseuille(n=10, nu=0.1, umax=1.0)
    assert q.params.gx == pytest.approx(8 * 0.1 * 1.0)  # g = 8 nu u_max / W^2, W = 1
    assert q.count(WALL) == 2 * 4 * 5 and q.count(FLUID) == 10 * 5
