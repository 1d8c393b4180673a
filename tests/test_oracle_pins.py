"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
hand-worked kernel values, integrals, symmetry/conservation invariants, exact
special cases (linear fields, uniform flow) and brute force.  A dropped term, a
wrong sign or index, or a transposed operand anywhere in the oracle fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1907_04034_gb300 import cases
from paper_1907_04034_gb300.cases import FLUID, INLET, OUTLET, WALL, SLIPWALL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- kernel (Eq. quintic-spline)
def test_quintic_values_match_hand_worked_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "quintic_w.txt"))
    for q, w, dw in rows:
        assert oracle.w(q) == w, q
        assert oracle.dw(q) == dw, q


def test_quintic_normalised_in_2d():
    # 2 pi int_0^{3h} W(r) r dr = 1 fixes alpha_2 = 7/(478 pi h^2)
    for h in (0.024, 1.0, 3.7):
        val, err = integrate.quad(lambda r: 2 * math.pi * r * oracle.W(r, h), 0.0, 3 * h,
                                  points=[h, 2 * h], epsabs=1e-14, epsrel=1e-13)
        assert abs(val - 1.0) < 1e-11


def test_quintic_derivative_is_dW_dr():
    h = 0.05
    for r in np.linspace(0.013, 0.149, 23):
        e = 1e-6
        fd = (oracle.W(r + e, h) - oracle.W(r - e, h)) / (2 * e)
        assert abs(fd - oracle.dWdr(r, h)) < 1e-6 * max(1.0, abs(fd))


def test_kernel_smooth_at_branch_points():
    for q in (1.0, 2.0, 3.0):
        e = 1e-9
        assert abs(oracle.w(q - e) - oracle.w(q + e)) < 1e-6
        assert abs(oracle.dw(q - e) - oracle.dw(q + e)) < 1e-6


# ---------------------------------------------------------------- neighbour search
def _brute_lists(case):
    p = case.params
    rc = 3.0 * (p.hdx * p.dx)
    rc2 = rc * rc
    x, y = case.x, case.y
    lists = []
    for i in range(case.n):
        dx = x[i] - x
        dy = y[i] - y
        if p.periodic_x:
            L = p.x_max - p.x_min
            dx = np.where(dx > 0.5 * L, dx - L, np.where(dx < -0.5 * L, dx + L, dx))
        if p.periodic_y:
            L = p.y_max - p.y_min
            dy = np.where(dy > 0.5 * L, dy - L, np.where(dy < -0.5 * L, dy + L, dy))
        lists.append(np.nonzero(dx * dx + dy * dy < rc2)[0])
    return lists


@pytest.mark.parametrize("maker", [lambda: cases.channel(),
                                   lambda: cases.random_box(n=400, seed=3),
                                   lambda: cases.random_box(n=300, seed=4, periodic_y=0),
                                   lambda: cases.taylor_green(n=16, jitter=0.3, seed=2)])
def test_neighbor_lists_are_the_definition(maker):
    c = maker()
    ref = _brute_lists(c)
    for mode in (0, 1):
        o = oracle.OracleSim(c, neighbor_mode=mode)
        start, idx = o.neighbors()
        for i in range(c.n):
            np.testing.assert_array_equal(idx[start[i]:start[i + 1]], ref[i])
        np.testing.assert_array_equal(o.field("nnb"), [len(r) for r in ref])


def test_binned_mode_matches_brute_force_over_a_window():
    c = cases.channel()
    a = oracle.OracleSim(c, neighbor_mode=0)
    b = oracle.OracleSim(c, neighbor_mode=1)
    a.step(40)
    b.step(40)
    for k in ("x", "y", "u", "v", "p", "rho", "au", "ap", "id", "tag"):
        np.testing.assert_array_equal(a.field(k), b.field(k))


# ----------------------------------------------------------- lattice / consistency
def test_partition_of_unity_on_lattice():
    # sum_j W_ij dx^2 approximates int W dA = 1; sum_j grad W_ij = 0 by symmetry
    c = cases.taylor_green(n=20)
    c.u[:] = 0.0
    c.v[:] = 0.0
    c.p[:] = 0.0
    o = oracle.OracleSim(c)
    dx = c.params.dx
    S = 1.0 / o.field("V")
    assert np.all(np.abs(S * dx * dx - 1.0) < 1e-4)
    # every particle of the periodic lattice sees the same value
    assert np.ptp(S) < 1e-9 * S.mean()
    np.testing.assert_allclose(o.field("rho"), S * c.params.rho0 * dx * dx, rtol=1e-14)
    # background-pressure acceleration vanishes on the symmetric lattice
    assert np.max(np.abs(o.field("abu"))) < 1e-9
    assert np.max(np.abs(o.field("abv"))) < 1e-9


def test_constant_fields_give_zero_rates():
    # constant p (a power of two) and constant u: p~_ij = 0 and u_ij = 0 exactly,
    # so the pressure, A and viscous terms and dp/dt vanish on a disordered box
    c = cases.taylor_green(n=16, jitter=0.3, seed=5)
    c.u[:] = 0.75
    c.v[:] = -0.25
    c.p[:] = 2.0
    o = oracle.OracleSim(c)
    assert np.all(o.field("au") == 0.0)
    assert np.all(o.field("av") == 0.0)
    assert np.all(o.field("ap") == 0.0)
    # ... while the background-pressure term does not vanish on disorder
    assert np.max(np.abs(o.field("abu"))) > 1.0


def _random_periodic(seed, use_pavg):
    c = cases.taylor_green(n=14, jitter=0.35, seed=seed)
    rng = np.random.default_rng(seed + 100)
    c.u[:] = rng.normal(0, 1, c.n)
    c.v[:] = rng.normal(0, 1, c.n)
    c.p[:] = rng.normal(0, 1, c.n)
    c.m[:] *= rng.uniform(0.8, 1.2, c.n)
    c.params.use_pavg = use_pavg
    return c


def test_momentum_antisymmetry_without_pavg():
    # with p_avg off, p~_ij = p~_ji and every pair term is antisymmetric: sum m a = 0
    c = _random_periodic(7, use_pavg=0)
    o = oracle.OracleSim(c)
    # make u~ != u so that the A-term is exercised
    o.a["ut"][: c.n] += np.random.default_rng(1).normal(0, 0.1, c.n)
    o.a["vt"][: c.n] += np.random.default_rng(2).normal(0, 0.1, c.n)
    o.evaluate()
    m = o.field("m")
    for k in ("au", "av"):
        f = m * o.field(k)
        assert abs(f.sum()) < 1e-12 * np.abs(f).sum()
    for k in ("abu", "abv"):
        f = m * o.field(k)
        assert abs(f.sum()) < 1e-12 * np.abs(f).sum()


def test_pavg_breaks_pair_symmetry_by_the_closed_form():
    # p~_ij - p~_ji = p_avg,j - p_avg,i, so sum_i m_i a_i = sum_{i<j} c_ij (pa_i - pa_j) gW_ij.
    # Check the sign and size with a field whose neighbour means differ strongly.
    c = _random_periodic(8, use_pavg=1)
    c.u[:] = 0.0
    c.v[:] = 0.0
    o = oracle.OracleSim(c)
    start, idx = o.neighbors()
    x, y, p = o.field("x"), o.field("y"), o.field("p")
    V = o.field("V")
    h = c.params.h
    L = 1.0
    pa = np.array([p[idx[start[i]:start[i + 1]]].mean() for i in range(c.n)])
    tot = np.zeros(2)
    for i in range(c.n):
        for j in idx[start[i]:start[i + 1]]:
            if j <= i:
                continue
            d = np.array([x[i] - x[j], y[i] - y[j]])
            d = np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d))
            r = np.hypot(*d)
            g = oracle.dWdr(r, h) * d / r
            tot += (V[i] ** 2 + V[j] ** 2) * (pa[i] - pa[j]) * g
    m = o.field("m")
    got = np.array([(m * o.field("au")).sum(), (m * o.field("av")).sum()])
    np.testing.assert_allclose(got, tot, rtol=1e-9, atol=1e-12 * np.abs(m * o.field("au")).sum())


def test_solid_force_balances_the_fluid_pressure_force():
    """Eq. tvf-momentum_solid read with the interpolated pressure pbar_ij (no p_avg shift on the
    solid's one-sided fluid sum).  Fluid at rest, random pressure, a solid block counted in the
    drag, p_avg on for the fluid: all pair terms are antisymmetric except the fluid's p_avg
    shift, so  sum_fluid m (a - g) + sum_solid F = sum_fluid p_avg,i G_i  with
    G_i = sum_j c_ij gW_ij = -m_i abg_i / p_b.  A p_avg shift on the solid side would add
    sum_solid p_avg,i sum_(j fluid) c_ij gW_ij to the left."""
    c = cases.taylor_green(n=16, jitter=0.3, seed=11)
    rng = np.random.default_rng(12)
    c.u[:] = 0.0
    c.v[:] = 0.0
    c.p[:] = rng.normal(0.0, 1.0, c.n)
    blk = (np.abs(c.x - 0.5) < 0.2) & (np.abs(c.y - 0.5) < 0.15)
    c.tag[blk] = cases.WALL
    c.params.use_pavg = 1
    c.params.wall_drag = (1, 0)
    o = oracle.OracleSim(c)
    start, idx = o.neighbors()
    tag, p, m = o.field("tag"), o.field("p"), o.field("m")
    fl = tag == cases.FLUID
    sol = tag == cases.WALL
    pa = np.array([p[idx[start[i]:start[i + 1]]].mean() for i in range(c.n)])
    lhs = np.zeros(2)
    rhs = np.zeros(2)
    for k, (a, ab, f) in enumerate((("au", "abu", "fx"), ("av", "abv", "fy"))):
        lhs[k] = np.sum(m[fl] * o.field(a)[fl]) + np.sum(o.field(f)[sol])
        G = -m * o.field(ab) / c.params.pb
        rhs[k] = np.sum(pa[fl] * G[fl])
    scale = np.sum(np.abs(m[fl] * o.field("au")[fl]))
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-10 * scale)
    # the solid force is not small: the identity is not met trivially
    assert np.abs(o.field("fx")[sol]).sum() > 1e-2 * scale


def _solid_block_case(seed, drag):
    c = cases.taylor_green(n=16, jitter=0.3, seed=seed)
    c.u[:] = 0.0
    c.v[:] = 0.0
    blk = (np.abs(c.x - 0.5) < 0.2) & (np.abs(c.y - 0.5) < 0.15)
    c.tag[blk] = cases.WALL
    c.params.use_pavg = 1
    c.params.wall_drag = (drag, 0)
    return c


def test_literal_solid_force_vanishes_for_uniform_pressure():
    """Eq. tvf-momentum_solid as printed (wall_drag 2): with p uniform (a power of two) on the
    fluid, hence on the walls, and everything at rest, p_avg,i = p and p~_ij = 0 for every
    pair, so the force is exactly zero on every solid particle; the fluid-only reading
    (wall_drag 1) leaves -p sum_(j fluid) c_ij gW_ij on the surface particles."""
    out = {}
    for drag in (1, 2):
        c = _solid_block_case(21, drag)
        c.p[:] = 2.0
        o = oracle.OracleSim(c)
        sol = o.field("tag") == cases.WALL
        np.testing.assert_array_equal(o.field("p")[sol], 2.0)
        out[drag] = np.hypot(o.field("fx"), o.field("fy"))[sol]
    assert np.all(out[2] == 0.0)
    # about p times the surface element dx on the block's faces
    assert out[1].max() > 0.5 * 2.0 * c.params.dx


def test_literal_solid_force_sums_every_neighbour_with_its_own_pavg():
    """wall_drag 2: F_i = sum over all j of c_ij [-p~_ij gW + viscous] with p~_ij of Eq.
    tvf-p-ij-basa (the solid particle's p_avg,i over all its neighbours).  Fluid at rest,
    random pressure, p_avg on: every pair term between fluid and solid particles is
    antisymmetric except the p_avg,i shift, so
        sum_fluid m (a - g) + sum_solid F = sum_(fluid and solid) p_avg,i G_i,
    G_i = sum_j c_ij gW_ij over all neighbours (brute force here for the solid particles).
    A fluid-only solid sum, or one without the shift, misses the solid part of the right."""
    c = _solid_block_case(11, 2)
    rng = np.random.default_rng(12)
    c.p[:] = rng.normal(0.0, 1.0, c.n)
    o = oracle.OracleSim(c)
    start, idx = o.neighbors()
    tag, p, m = o.field("tag"), o.field("p"), o.field("m")
    x, y, V = o.field("x"), o.field("y"), o.field("V")
    h = c.params.h
    fl = tag == cases.FLUID
    sol = tag == cases.WALL
    pa = np.array([p[idx[start[i]:start[i + 1]]].mean() for i in range(c.n)])
    Gs = np.zeros((c.n, 2))
    for i in np.nonzero(sol)[0]:
        for j in idx[start[i]:start[i + 1]]:
            d = np.array([x[i] - x[j], y[i] - y[j]])
            d = np.where(d > 0.5, d - 1.0, np.where(d < -0.5, d + 1.0, d))
            r = np.hypot(*d)
            if r > 0.0:
                Gs[i] += (V[i] ** 2 + V[j] ** 2) * oracle.dWdr(r, h) * d / r
    lhs = np.zeros(2)
    rhs = np.zeros(2)
    for k, (a, ab, f) in enumerate((("au", "abu", "fx"), ("av", "abv", "fy"))):
        lhs[k] = np.sum(m[fl] * o.field(a)[fl]) + np.sum(o.field(f)[sol])
        G = -m * o.field(ab) / c.params.pb
        rhs[k] = np.sum(pa[fl] * G[fl]) + np.sum(pa[sol] * Gs[sol, k])
    scale = np.sum(np.abs(m[fl] * o.field("au")[fl]))
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-10 * scale)
    # the solid part of the right side is far above the tolerance: a reading without the
    # shift or without the solid-solid pairs fails the identity
    assert np.abs(np.sum(pa[sol, None] * Gs[sol], axis=0)).max() > 1e-5 * scale


def _wall_and_one_fluid(r, dx=0.05):
    """A no-slip wall particle at the origin and one fluid particle at (r, 0)."""
    cs = 10.0
    prm = cases.Params(x_min=-1.0, x_max=1.0, y_min=-1.0, y_max=1.0, dx=dx, hdx=1.2,
                       nu=0.01, cs=cs, pb=cs * cs, dt=1e-4, wall_drag=(0, 0))
    x = np.array([0.0, r])
    y = np.zeros(2)
    return cases.Case("wall_pair", prm, x, y, np.array([0.0, 0.3]), np.array([0.0, -0.2]),
                      np.array([0.0, 0.7]), np.full(2, dx * dx),
                      np.array([cases.WALL, cases.FLUID], dtype=np.uint8),
                      np.arange(2, dtype=np.uint64), capacity=8)


def test_wall_shepard_with_one_fluid_neighbour_at_the_support_edge():
    """Shepard projection on a wall (Adami et al., cited in Sec. 2) over one fluid neighbour is
    that neighbour's value: near the support edge (W tiny) and at the edge itself, where W
    rounds to exactly 0 and the all-zero-weights rule (plain mean) takes over."""
    # a spacing at which the largest separation inside the support (one ulp below r_c, so
    # that r^2 < r_c^2) gives q = r/h = 3 exactly in fp64, hence W = 0
    dx = 0.01303
    h = 1.2 * dx
    rc = 3.0 * h
    r0 = math.nextafter(rc, 0.0)
    assert r0 * r0 < rc * rc and oracle.W(r0, h) == 0.0
    r1 = rc * (1.0 - 1e-9)  # W > 0 but tiny
    assert 0.0 < oracle.W(r1, h) < 1e-30
    for r in (r1, r0):
        o = oracle.OracleSim(_wall_and_one_fluid(r, dx))
        o.evaluate()
        start, idx = o.neighbors()
        assert list(idx[start[0]:start[1]]) == [0, 1]  # the fluid particle is a neighbour
        assert o.field("p")[0] == pytest.approx(0.7, rel=1e-15)
        assert o.field("u")[0] == pytest.approx(-0.3, rel=1e-15)  # 2 u_wall - u_f
        assert o.field("v")[0] == pytest.approx(0.2, rel=1e-15)


# ----------------------------------------------------------------- full scheme
def test_taylor_green_decay_rate():
    # velocity amplitude of the Taylor-Green vortex decays as exp(-8 pi^2 nu t)
    # (discretisation error at h = 1.2 dx, 40x40: about 3%, mostly the eta h^2 regulariser
    # of the viscous denominator, which is a fixed fraction of the nearest-pair r^2)
    nu = 0.05
    c = cases.taylor_green(n=40, nu=nu)
    o = oracle.OracleSim(c, neighbor_mode=1)
    dt = c.params.dt
    ke0 = 0.5 * np.sum(o.field("m") * (o.field("u") ** 2 + o.field("v") ** 2))
    nsteps = int(round(0.25 / dt))
    o.step(nsteps)
    t = nsteps * dt
    ke = 0.5 * np.sum(o.field("m") * (o.field("u") ** 2 + o.field("v") ** 2))
    rate = -math.log(ke / ke0) / (2 * t)
    exact = 8 * math.pi ** 2 * nu
    assert abs(rate - exact) / exact < 0.04, (rate, exact)


def test_viscous_term_is_nu_laplacian_of_shear():
    # u = sin(k y), p = 0, u~ = u: du/dt = nu d2u/dy2 = -nu k^2 sin(k y) up to the kernel's
    # smoothing error, which shrinks with dx
    ratios = []
    for n in (20, 40):
        c = cases.taylor_green(n=n, nu=0.05)
        k = 2 * math.pi
        c.u[:] = np.sin(k * c.y)
        c.v[:] = 0.0
        c.p[:] = 0.0
        o = oracle.OracleSim(c, neighbor_mode=1)
        ex = -0.05 * k * k * np.sin(k * o.field("y"))
        sel = np.abs(ex) > 0.5 * np.abs(ex).max()
        r = o.field("au")[sel] / ex[sel]
        assert np.ptp(r) < 1e-10
        ratios.append(r.mean())
        assert np.abs(o.field("av")).max() < 1e-12
    assert abs(ratios[0] - 1.0) < 0.03 and abs(ratios[1] - 1.0) < 0.015
    assert abs(ratios[1] - 1.0) < abs(ratios[0] - 1.0)


@pytest.mark.slow
def test_poiseuille_profile():
    # steady plane Poiseuille flow between no-slip walls: u(y) = g/(2 nu) y (W - y)
    c = cases.poiseuille(n=10, nu=0.25, umax=1.0)
    o = oracle.OracleSim(c, neighbor_mode=1)
    dt = c.params.dt
    o.step(int(round(2.0 / dt)))
    f = o.fields()
    fl = f["tag"] == FLUID
    y = f["y"][fl]
    g = c.params.gx
    exact = g / (2 * c.params.nu) * y * (1.0 - y)
    err = np.abs(f["u"][fl] - exact).max()
    assert err < 0.03, err
    assert np.abs(f["v"][fl]).max() < 0.01


# ---------------------------------------------------------------- inlet mirror
def test_mirror_recovers_linear_field_exactly():
    # first-order consistency of Eq. (matform): a linear field is reproduced with its gradient
    c = cases.taylor_green(n=30, jitter=0.2, seed=3)
    c.params.periodic_x = 0
    c.params.periodic_y = 0
    c.u[:] = 0
    c.v[:] = 0
    a, b, cc = 0.3, -1.7, 0.9
    c.p[:] = a + b * c.x + cc * c.y
    o = oracle.OracleSim(c)
    qx = np.array([0.5, 0.3, 0.62, 0.41])
    qy = np.array([0.5, 0.7, 0.33, 0.5])
    pk, gx, gy = o.mirror_points(qx, qy)
    np.testing.assert_allclose(pk, a + b * qx + cc * qy, rtol=0, atol=1e-11)
    np.testing.assert_allclose(gx, b, rtol=0, atol=1e-9)
    np.testing.assert_allclose(gy, cc, rtol=0, atol=1e-9)


def test_inlet_pressure_uses_minus_sign_taylor_extrapolation():
    # Eq. (taylor2): p_o = p_k - (r_o - r_k).grad p_k; for p = a + b x that is a + b (2 x_k - x_o)
    c = cases.channel(jitter=0.0)
    a, b = 0.2, 0.5
    c.p[:] = a + b * c.x
    c.u[:] = 1.0
    o = oracle.OracleSim(c)
    f = o.fields()
    inl = f["tag"] == INLET
    xo = f["x"][inl]
    xk = 2 * c.params.x_in - xo
    np.testing.assert_allclose(f["p"][inl], a + b * (2 * xk - xo), rtol=0, atol=1e-10)


# ---------------------------------------------------------------- walls
def test_wall_projection_of_uniform_fluid():
    c = cases.poiseuille(n=10)
    c.u[:] = np.where(c.tag == FLUID, 0.4, 0.0)
    c.p[:] = np.where(c.tag == FLUID, 0.125, 0.0)
    o = oracle.OracleSim(c)
    f = o.fields()
    wl = f["tag"] == WALL
    # wall rows within 3h = 3.6 dx of the first fluid row (y = dx/2) see fluid
    near = wl & (f["y"] > -3.1 * c.params.dx) & (f["y"] < 1 + 3.1 * c.params.dx)
    far = wl & ~near
    # no-slip: ghost velocity 2 u_w - <u_f> = -0.4; Shepard pressure of a constant field
    np.testing.assert_allclose(f["u"][near], -0.4, rtol=0, atol=1e-14)
    np.testing.assert_allclose(f["p"][near], 0.125, rtol=0, atol=1e-14)
    assert np.all(f["u"][far] == 0.0) and np.all(f["p"][far] == 0.0)


# ------------------------------------------------------- hybrid outlet and recycling
def test_uniform_flow_through_inlet_and_outlet_stays_uniform():
    # lattice with 8 inlet and 8 outlet layers (> 2 x 3h, so that every neighbour of a fluid
    # particle has full support), u = U, p = 0: J2 = 0 and the flow is unchanged to round-off;
    # every column that leaves is replaced by one spawned a lattice period upstream
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=8, n_out=8)
    o = oracle.OracleSim(c)
    n0 = o.n
    hist = o.step(150)
    f = o.fields()
    assert np.abs(f["u"] - 1.0).max() < 1e-12
    assert np.abs(f["v"]).max() < 1e-12
    assert np.abs(f["p"]).max() < 1e-12
    spawned = sum(h["n_spawn"] for h in hist)
    deleted = sum(h["n_delete"] for h in hist)
    assert spawned > 0 and deleted > 0
    assert o.n == n0 + spawned - deleted
    assert [h["n_active"] for h in hist][-1] == o.n
    ids = f["id"]
    assert len(np.unique(ids)) == len(ids)
    assert np.all(np.diff(ids.astype(np.int64)) > 0)
    # the spawned particles keep the lattice: x positions of inlet particles are a lattice
    xi = np.sort(np.unique(np.round(f["x"][f["tag"] == INLET] / c.params.dx, 6)))
    assert np.allclose(np.diff(xi), 1.0)


def test_recycling_counts_and_conversions():
    c = cases.channel()
    o = oracle.OracleSim(c)
    n0 = o.n
    nf0 = c.count(FLUID)
    hist = o.step(200)
    sp = sum(h["n_spawn"] for h in hist)
    dl = sum(h["n_delete"] for h in hist)
    to = sum(h["n_to_outlet"] for h in hist)
    f = o.fields()
    assert o.n == n0 + sp - dl
    # inlet count is conserved (each conversion spawns one), fluid count follows the flux
    assert np.count_nonzero(f["tag"] == INLET) == c.count(INLET)
    assert np.count_nonzero(f["tag"] == FLUID) == nf0 + sp - to
    # each record's particle count is the count after that step's recycling
    counts = n0 + np.cumsum([h["n_spawn"] - h["n_delete"] for h in hist])
    assert [h["n_active"] for h in hist] == counts.tolist() and counts[-1] == o.n
    # mass flux history equals the mass of the converted particles per unit time
    m = c.params.rho0 * c.params.dx ** 2
    for h in hist:
        assert abs(h["mass_flux"] * c.params.dt - h["n_to_outlet"] * m) < 1e-15
    # new ids follow ascending parent order and are contiguous
    ids = np.sort(f["id"])
    assert ids[-1] == n0 + sp - 1


def _events_from_states(a, b, step, L_in):
    """The recycling events of one step read off the states before (a) and after (b) it, by
    id: ids gone = deletions; FLUID -> OUTLET = conversions; new ids = spawns, each matched
    to the INLET -> FLUID particle at its x + L_in and its y.  Kinds in that order, each in
    ascending id."""
    ia = {int(i): k for k, i in enumerate(a["id"])}
    ib = {int(i): k for k, i in enumerate(b["id"])}
    gone = sorted(i for i in ia if i not in ib)
    conv = sorted(i for i in ia if i in ib and a["tag"][ia[i]] == FLUID and b["tag"][ib[i]] == OUTLET)
    parents = sorted(i for i in ia if i in ib and a["tag"][ia[i]] == INLET and b["tag"][ib[i]] == FLUID)
    new = sorted(i for i in ib if i not in ia)
    assert len(new) == len(parents)
    ev = [(step, 0, i, 0) for i in gone] + [(step, 1, i, 0) for i in conv]
    for p_id, n_id in zip(parents, new):
        kp, kn = ib[p_id], ib[n_id]
        assert b["tag"][kn] == INLET
        assert b["y"][kn] == b["y"][kp] and abs(b["x"][kn] - (b["x"][kp] - L_in)) < 1e-12
        ev.append((step, 2, n_id, p_id))
    return ev


def test_event_log_is_the_state_transitions_of_each_step():
    """The oracle's recycling event log (Sec. 3.4's transitions) against the events read off
    consecutive states: deletions, fluid->outlet conversions and spawns (new id, parent id)
    in that order, each in ascending id, with the step number; new ids ascend with the
    parent ids.  A small log drops whole steps and counts them."""
    c = cases.channel()
    o = oracle.OracleSim(c, max_events=10000)
    L_in = c.params.n_in_layers * c.params.dx
    want = []
    a = o.fields(("id", "tag", "x", "y"))
    for k in range(1, 161):
        o.step(1)
        b = o.fields(("id", "tag", "x", "y"))
        want += _events_from_states(a, b, k, L_in)
        a = b
    got = o.events()
    assert got["dropped"] == 0
    rows = list(zip(got["step"].tolist(), got["kind"].tolist(), got["id"].tolist(),
                    got["other"].tolist()))
    assert rows == want
    kinds = {kd: sum(1 for r in rows if r[1] == kd) for kd in (0, 1, 2)}
    assert min(kinds.values()) > 5, kinds  # every kind occurs
    # a log too small for one step's events keeps nothing of that step and counts it
    o2 = oracle.OracleSim(cases.channel(), max_events=1)
    o2.step(160)
    e2 = o2.events()
    assert all(np.count_nonzero(e2["step"] == s) == 1 for s in np.unique(e2["step"]))
    assert len(e2["step"]) + e2["dropped"] == len(rows)


def test_acoustic_gate_freezes_time_average():
    # with pulse amplitude 1 the intensity p^2/(2 rho c) exceeds I = (rho U^2/2)^2/(2 rho c)
    # near the pulse: those rings take no sample (write index stays 0); elsewhere one is taken
    c = cases.channel(pulse_amp=1.0)
    o = oracle.OracleSim(c)
    o.step(1)
    f = o.fields(("tag", "p", "rpos"))
    fl = f["tag"] == FLUID
    I = (0.5 * 1.0 * 1.0) ** 2 / (2 * 1.0 * 10.0)
    hot = fl & (f["p"] ** 2 / (2 * 1.0 * 10.0) > I)
    cold = fl & ~hot
    assert hot.sum() > 10 and cold.sum() > 100
    assert np.all(f["rpos"][hot] == 0)
    assert np.all(f["rpos"][cold] == 1)


def test_characteristic_inversion_round_trip():
    # Eq. (characteristic-vars) with J3 = 0: a fluid state with u' = J2/(2 rho c), p' = J2/2
    # relative to its time average must be reproduced at a red outlet particle sitting
    # among fluid particles that all carry the same J2.
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=4)
    o = oracle.OracleSim(c)
    # bump u and p of all fluid particles by an acoustic pair, leave the rings at the old values
    J2 = 0.02
    rho_c = c.params.rho0 * c.params.cs
    fl = o.a["tag"][: o.n] == FLUID
    o.a["u"][: o.n][fl] += J2 / (2 * rho_c)
    o.a["p"][: o.n][fl] += J2 / 2
    o.a["J2"][: o.n][fl] = rho_c * (J2 / (2 * rho_c)) + J2 / 2
    o.evaluate()
    # one step moves things a little; check the red outlet particles right after the update
    o.step(1)
    f = o.fields(("tag", "x", "u", "p", "J2p"))
    red = (f["tag"] == OUTLET) & (f["x"] < c.params.x_out + 2 * c.params.dx)
    assert red.sum() > 0
    # the outlet u and p equal average + acoustic part implied by the stored J2
    np.testing.assert_allclose(f["p"][red], 0.5 * f["J2p"][red], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(f["u"][red] - 1.0, f["J2p"][red] / (2 * rho_c), rtol=1e-12,
                               atol=1e-15)
    assert np.all(np.abs(f["J2p"][red]) > 0.3 * J2)


# --------------------------------------------------------- the other outlets (Sec. 3)
OUTLET_KINDS = {"donothing": 1, "mod_donothing": 2, "characteristic": 3, "mirror": 4}


@pytest.mark.parametrize("kind", list(OUTLET_KINDS))
def test_uniform_flow_stays_uniform_with_every_outlet(kind):
    # u = U, p = 0 on a lattice with 8 inlet and 8 outlet layers: frozen values (Sec. 3.1),
    # the Shepard advection velocity of a constant field (Sec. 3.1.1), J2 = 0 against the free
    # stream (Sec. 3.3) and the Taylor extrapolation of constant fields (Sec. 3.2) all keep it
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=8, n_out=8)
    c.params.outlet_kind = OUTLET_KINDS[kind]
    o = oracle.OracleSim(c)
    hist = o.step(120)
    f = o.fields()
    assert np.abs(f["u"] - 1.0).max() < 1e-12
    assert np.abs(f["v"]).max() < 1e-12
    assert np.abs(f["p"]).max() < 1e-12
    assert sum(h["n_delete"] for h in hist) > 0


def test_donothing_outlet_freezes_values_and_advects_with_them():
    # Sec. 3.1: an outlet particle keeps u, v, p and moves x by u dt per step, y fixed
    c = cases.channel(pulse_amp=0.3)
    c.params.outlet_kind = OUTLET_KINDS["donothing"]
    o = oracle.OracleSim(c)
    o.step(40)
    a = o.fields(("id", "tag", "x", "y", "u", "v", "p"))
    o.step(1)
    b = o.fields(("id", "tag", "x", "y", "u", "v", "p"))
    ia = {int(i): k for k, i in enumerate(a["id"])}
    kept = [(ia[int(i)], k) for k, i in enumerate(b["id"])
            if b["tag"][k] == OUTLET and int(i) in ia and a["tag"][ia[int(i)]] == OUTLET]
    assert len(kept) > 50
    ka, kb = np.array(kept).T
    for fld in ("u", "v", "p", "y"):
        np.testing.assert_array_equal(b[fld][kb], a[fld][ka])
    np.testing.assert_allclose(b["x"][kb], a["x"][ka] + c.params.dt * a["u"][ka], rtol=0,
                               atol=1e-15)
    assert np.ptp(a["p"][ka]) > 1e-4  # the frozen values are not all the same


def test_modified_donothing_advects_with_the_fluid_velocity():
    # Sec. 3.1.1: values frozen as in do-nothing, but a red outlet particle advects with the
    # Shepard average of its fluid neighbours' u (a convex combination, Eq. shepard0), not
    # with its own frozen u
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=4, n_out=8)
    c.params.outlet_kind = OUTLET_KINDS["mod_donothing"]
    c.u[c.tag == OUTLET] = 1.3
    o = oracle.OracleSim(c)
    o.step(1)
    f = o.fields(("id", "tag", "x", "u", "v", "p", "advp", "redp"))
    start, idx = o.neighbors()
    tag, u = f["tag"], f["u"]
    out = np.nonzero(tag == OUTLET)[0]
    red = [k for k in out if np.any(tag[idx[start[k]:start[k + 1]]] == FLUID)]
    assert len(red) > 20
    for k in red:
        nb = idx[start[k]:start[k + 1]]
        uf = u[nb[tag[nb] == FLUID]]
        assert uf.min() - 1e-14 <= f["advp"][k] <= uf.max() + 1e-14
        assert f["redp"][k] == 1
    assert np.all(u[out] == 1.3)  # the particles' own velocity stays frozen
    assert np.abs(f["advp"][red] - 1.3).min() > 0.2


def test_characteristic_outlet_passes_a_right_running_wave():
    # Sec. 3.3 with the free stream (U, p = 0) as reference: a fluid state u = U + a/(2 rho c),
    # p = a/2 has J2 = a and J3 = 0; the red outlet particles reproduce it (p = J2/2,
    # u = U + J2/(2 rho c)) and keep their transverse velocity
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=4)
    c.params.outlet_kind = OUTLET_KINDS["characteristic"]
    a = 0.02
    rho_c = c.params.rho0 * c.params.cs
    fl = c.tag == FLUID
    c.u[fl] += a / (2 * rho_c)
    c.p[fl] += a / 2
    c.v[c.tag == OUTLET] = 0.05
    o = oracle.OracleSim(c)
    o.step(1)
    f = o.fields(("tag", "x", "u", "v", "p", "J2p", "redp"))
    red = (f["tag"] == OUTLET) & (f["redp"] == 1)
    assert red.sum() > 20
    np.testing.assert_allclose(f["p"][red], 0.5 * f["J2p"][red], rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(f["u"][red] - 1.0, f["J2p"][red] / (2 * rho_c), rtol=1e-12,
                               atol=1e-16)
    np.testing.assert_allclose(f["J2p"][red], a, rtol=0.1)
    assert np.all(f["v"][f["tag"] == OUTLET] == 0.05)


def test_mirrored_outlet_is_exact_for_linear_fields():
    # Sec. 3.2 at the outlet: for linear f the first-order system returns f(x_k) and grad f
    # exactly, so Eq. taylor2 gives f_o = f(x_k) - (x_o - x_k) f_x = f(4 x_out - 3 x_o, y_o)
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=4, n_out=6)
    c.params.outlet_kind = OUTLET_KINDS["mirror"]
    o = oracle.OracleSim(c)
    n = o.n
    x, y = o.a["x"][:n], o.a["y"][:n]
    # linear in x only: the channel is periodic in y, where a linear field would jump
    lin = {"p": (0.3, -0.7, 0.0), "u": (1.0, 0.4, 0.0), "v": (-0.2, 0.1, 0.0)}
    for k, (c0, cx, cy) in lin.items():
        o.a[k][:n] = c0 + cx * x + cy * y
    o.outlet_mirror()
    tag = o.a["tag"][:n]
    out = tag == OUTLET
    xr = 4.0 * c.params.x_out - 3.0 * x[out]
    for k, (c0, cx, cy) in lin.items():
        want = c0 + cx * xr + cy * y[out]
        np.testing.assert_allclose(o.a[k][:n][out], want, rtol=0, atol=1e-11)
    np.testing.assert_allclose(o.a["advp"][:n][out], o.a["u"][:n][out], rtol=0, atol=0)


# ------------------------------------------------- inlet in time, probes (Sec. 4 problems)
def test_ramp_inlet_moves_particles_by_the_integral_of_the_ramp():
    # Sec. 4.3: u = U t / T for t < T, so an inlet particle moves by U t^2 / (2 T); the
    # integrator stage takes the inlet velocity at the end of each stage, which adds at most
    # U t dt / (2 T)
    c = cases.outlet_problem("ramp")
    o = oracle.OracleSim(c, neighbor_mode=1)
    x0 = {int(i): x for i, x, t in zip(o.field("id"), o.field("x"), o.field("tag")) if t == INLET}
    o.step(180)
    t = o.t
    T = c.params.inlet_prm[0]
    f = o.fields(("id", "x", "u", "v", "tag"))
    inl = [(x0[int(i)], x, u) for i, x, u, tg in zip(f["id"], f["x"], f["u"], f["tag"])
           if tg == INLET and int(i) in x0]
    assert len(inl) > 50 and t < T
    want = t * t / (2 * T)
    for a, b, u in inl:
        assert want <= b - a <= want + t * c.params.dt / (2 * T) + 1e-12
        assert u == pytest.approx(t / T, rel=1e-12)
    assert np.all(f["v"][f["tag"] == INLET] == 0.0)


def test_vortex_inlet_velocity_is_antisymmetric_about_the_centre_line():
    # Eqs. vortex, vortexx: u - U is odd and v even in y - y_c; on the centre line u = U and,
    # at t = 0 (centre d0 = 1 upstream), v = -G d0 / (d0^2 + c)
    c = cases.outlet_problem("vortex")
    G, core, d0, yc = c.params.inlet_prm
    o = oracle.OracleSim(c, neighbor_mode=1)
    o.step(1)
    f = o.fields(("x", "y", "u", "v", "tag"))
    inl = f["tag"] == INLET
    y, u, v = f["y"][inl], f["u"][inl], f["v"][inl]
    up = {round(a - yc, 9): (b, w) for a, b, w in zip(y, u, v)}
    pairs = [(up[k], up[-k]) for k in up if k > 0 and -k in up]
    assert len(pairs) > 10
    for (ua, va), (ub, vb) in pairs:
        assert ua - 1.0 == pytest.approx(-(ub - 1.0), rel=1e-12, abs=1e-15)
        assert va == pytest.approx(vb, rel=1e-12)
    t = c.params.dt
    xr = 1.0 * (d0 - t)
    ymin = np.min(np.abs(y - yc))
    k = np.argmin(np.abs(y - yc))
    assert v[k] == pytest.approx(-G * xr / (xr * xr + ymin * ymin + core), rel=1e-12)
    # the sense of rotation: with G > 0, u exceeds U above the centre line (u - U = G y_r / ...)
    top = np.argmax(y - yc)
    yr = y[top] - yc
    assert G > 0 and yr > 0
    assert u[top] - 1.0 == pytest.approx(G * yr / (xr * xr + yr * yr + core), rel=1e-12)


def test_pulse_inlet_is_quiet_outside_its_window():
    c = cases.outlet_problem("pulse2d")
    o = oracle.OracleSim(c, neighbor_mode=1)
    o.step(300)  # t = 0.82 < t0
    f = o.fields(("u", "tag"))
    assert np.all(f["u"][f["tag"] == INLET] == 1.0)
    o.step(70)   # t = 1.009: inside (1, 1.1), A cos(pi y/12) exp(-(t-1)^2/delta) added
    f = o.fields(("y", "u", "tag"))
    inl = f["tag"] == INLET
    A, t0, t1, dl = c.params.inlet_prm
    t = o.t
    want = 1.0 + A * np.cos(np.pi * f["y"][inl] / 12.0) * np.exp(-(t - t0) ** 2 / dl)
    np.testing.assert_allclose(f["u"][inl], want, rtol=1e-12)
    assert f["u"][inl].min() > 1.4


def test_probe_is_the_shepard_average_of_the_fluid():
    # on a lattice, the kernel weights around a lattice node are symmetric, so the Shepard
    # average of a linear field at the node is the field's value there; the count is the
    # number of lattice points within 3h (brute force)
    c = cases.taylor_green(n=30)
    c.params.periodic_x = c.params.periodic_y = 0
    c.u[:] = 0.5 - 2.0 * c.x + 0.25 * c.y
    c.v[:] = 0.0
    c.p[:] = 1.0 + 3.0 * c.x - 1.5 * c.y
    o = oracle.OracleSim(c)
    k = int(np.argmin((c.x - 0.5) ** 2 + (c.y - 0.5) ** 2))
    qx, qy = c.x[k], c.y[k]
    out = o.probe([qx], [qy])[0]
    assert out[0] == pytest.approx(1.0 + 3.0 * qx - 1.5 * qy, rel=1e-12)
    assert out[1] == pytest.approx(0.5 - 2.0 * qx + 0.25 * qy, rel=1e-12)
    rc = 3.0 * c.params.h
    assert out[3] == np.count_nonzero((c.x - qx) ** 2 + (c.y - qy) ** 2 < rc * rc)
    # far from every particle: zeros
    assert np.all(o.probe([5.0], [5.0])[0] == 0.0)


def test_inviscid_rates_are_finite():
    # nu = 0 (Sec. 4 test problems): the harmonic mean of two zero viscosities is zero
    c = cases.outlet_problem("vortex")
    o = oracle.OracleSim(c, neighbor_mode=1)
    o.step(3)
    for k in ("au", "av", "ap", "u", "p"):
        assert np.all(np.isfinite(o.field(k)))


def test_characteristic_outlet_with_a_reference_state():
    # Sec. 3.3 with (u_ref, p_ref) = (1.2, 0.3): a fluid state u = u_ref + a/(2 rho c),
    # p = p_ref + a/2 has J2 = a, J3 = 0 and reaches the red outlet particles unchanged
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=4)
    c.params.outlet_kind = OUTLET_KINDS["characteristic"]
    c.params.moc_ref = (1.2, 0.3)
    a = 0.02
    rho_c = c.params.rho0 * c.params.cs
    c.u[:] = 1.2 + a / (2 * rho_c)
    c.p[:] = 0.3 + a / 2
    o = oracle.OracleSim(c)
    o.step(1)
    f = o.fields(("tag", "u", "p", "J2p", "redp"))
    red = (f["tag"] == OUTLET) & (f["redp"] == 1)
    assert red.sum() > 20
    np.testing.assert_allclose(f["p"][red], 0.3 + 0.5 * f["J2p"][red], rtol=1e-13)
    np.testing.assert_allclose(f["u"][red], 1.2 + f["J2p"][red] / (2 * rho_c), rtol=1e-13)
    np.testing.assert_allclose(f["J2p"][red], a, rtol=0.1)


def _open_lattice(n=24):
    c = cases.taylor_green(n=n)
    c.params.periodic_x = 0
    c.params.periodic_y = 0
    c.u[:] = 0.0
    c.v[:] = 0.0
    c.p[:] = 0.0
    return c


def _interior(o, c, margin=3.6):
    x, y = o.field("x"), o.field("y")
    d = margin * c.params.dx
    return (x > d) & (x < 1 - d) & (y > d) & (y < 1 - d)


def test_pressure_gradient_of_linear_field():
    # Eq. (tvf-momentum) reduces to du/dt = -grad p / rho for u = 0 (continuous form, Eq. mom-newt)
    c = _open_lattice()
    c.p[:] = 0.3 * c.x - 0.2 * c.y + 1.5
    o = oracle.OracleSim(c)
    sel = _interior(o, c)
    rho = o.field("rho")[sel]
    np.testing.assert_allclose(o.field("au")[sel], -0.3 / rho, rtol=2e-3)
    np.testing.assert_allclose(o.field("av")[sel], 0.2 / rho, rtol=2e-3)


def test_edac_divergence_of_linear_velocity():
    # Eq. (p-edac) for a linear u and constant p reduces to dp/dt = -rho c^2 div u (Eq. p-evolve)
    c = _open_lattice()
    c.u[:] = 0.4 * c.x
    c.v[:] = -0.1 * c.y
    o = oracle.OracleSim(c)
    sel = _interior(o, c)
    rho = o.field("rho")[sel]
    np.testing.assert_allclose(o.field("ap")[sel], -rho * c.params.cs ** 2 * 0.3, rtol=2e-3)


def test_edac_pressure_diffusion_of_quadratic_field():
    # the damping term of Eq. (p-evolve) is nu_edac lap p with nu_edac = alpha h c / 8 (Eq. edac-nu);
    # for p = x^2 + y^2 and u = 0, dp/dt = 4 nu_edac (less the eta h^2 regulariser's ~1-2%)
    c = _open_lattice(n=30)
    c.p[:] = c.x ** 2 + c.y ** 2
    o = oracle.OracleSim(c)
    sel = _interior(o, c)
    nu_e = c.params.alpha * c.params.h * c.params.cs / 8
    r = o.field("ap")[sel] / (4 * nu_e)
    assert np.all(np.abs(r - 1.0) < 0.03), (r.min(), r.max())


def test_slip_wall_keeps_tangential_flow_and_no_slip_wall_brakes_it():
    out = {}
    for slip in (1, 0):
        c = cases.poiseuille(n=10, nu=0.1)
        c.params.gx = 0.0
        c.tag[c.tag == WALL] = SLIPWALL if slip else WALL
        c.params.wall_slip = (0, 1)
        c.u[:] = np.where(c.tag == FLUID, 0.5, 0.0)
        o = oracle.OracleSim(c, neighbor_mode=1)
        o.step(int(round(0.5 / c.params.dt)))
        f = o.fields()
        row = (f["tag"] == FLUID) & (f["y"] < 0.1)
        out[slip] = f["u"][row].mean()
        assert np.abs(f["v"][f["tag"] == FLUID]).max() < 5e-3
    assert abs(out[1] - 0.5) < 5e-3, out
    assert out[0] < 0.4, out


# ----------------------------------------- A-term, blue rule, time window, integrator order
def test_pressure_bump_splits_into_waves_at_the_sound_speed():
    """The 1D pressure bump of Sec. 4.1 (Eq. pressurebump) splits into two acoustic waves that,
    in the fluid moving at U, travel at -c and +c (the EDAC pressure equation with the
    momentum equation is the wave equation with speed c for small perturbations), each
    carrying about half the depth; the pattern stays symmetric about the advected centre.
    A wrong factor c^2 in dp/dt or a wrong sign of the pressure gradient fails."""
    c = cases.pressure_bump(outlet=0)
    o = oracle.OracleSim(c, neighbor_mode=1)
    p = c.params
    n = int(round(0.03 / p.dt))
    o.step(n)
    t = n * p.dt
    f = o.fields(("x", "p", "tag"))
    fl = f["tag"] == FLUID
    dx = p.dx
    nb = int(round(1.0 / dx))
    b = np.minimum((f["x"][fl] / dx).astype(int), nb - 1)
    prof = np.bincount(b, weights=f["p"][fl], minlength=nb) / np.maximum(np.bincount(b, minlength=nb), 1)
    xs = (np.arange(nb) + 0.5) * dx
    dev = (prof - 1e-3) / 0.2e-3  # in units of the bump's depth
    centre = 0.5 + p.U * t
    left, right = xs < centre, xs >= centre
    xl = xs[left][np.argmin(dev[left])]
    xr = xs[right][np.argmin(dev[right])]
    # wave speeds relative to the fluid within 4% of c
    assert abs((centre - xl) / t - p.cs) < 0.04 * p.cs, (xl, xr, t)
    assert abs((xr - centre) / t - p.cs) < 0.04 * p.cs, (xl, xr, t)
    # symmetric about the advected centre, each wave about half the depth
    assert abs((centre - xl) - (xr - centre)) <= 1.01 * dx
    dl, dr = dev[left].min(), dev[right].min()
    assert abs(dl - dr) < 0.02 * abs(dl)
    assert -0.55 < dl < -0.35 and -0.55 < dr < -0.35
    # and the centre has relaxed toward the undisturbed pressure
    assert abs(dev[np.argmin(abs(xs - centre))]) < 0.1


def test_A_term_is_the_divergence_of_rho_u_times_the_shift():
    """The A-term of Eq. tvf-momentum, 1/2 (A_i + A_j).gW with A = rho u (x) (u~ - u), is the
    SPH form of div(A)/rho.  With u = (U, 0), p = 0 and u~ - u = (0, gamma y) that is
    d/dy(rho U gamma y)/rho = U gamma in x and 0 in y (interior of an open lattice).  The
    transposed tensor rho (u~ - u) (x) u gives 0 in x, a flipped sign -U gamma; the viscous and
    pressure terms vanish (uniform u, p = 0), so the A-term alone is measured."""
    c = _open_lattice(n=30)
    U, gamma = 0.8, 0.35
    c.u[:] = U
    o = oracle.OracleSim(c)
    n = o.n
    o.a["vt"][:n] = o.a["v"][:n] + gamma * o.a["y"][:n]
    o.evaluate()
    sel = _interior(o, c)
    au, av = o.field("au")[sel], o.field("av")[sel]
    np.testing.assert_allclose(au, U * gamma, rtol=2e-3)
    assert np.abs(av).max() < 1e-10 * U * gamma
    # with u~ = u the same state has no A-term: the rate above is the A-term's alone
    o.a["vt"][:n] = o.a["v"][:n]
    o.evaluate()
    assert np.abs(o.field("au")[sel]).max() < 1e-10 * U * gamma


def test_A_term_shift_along_the_flow():
    """Second orientation check of A = rho u (x) (u~ - u): u = (0, V), u~ - u = (gamma x, 0) gives
    div(A)_y / rho = d/dx(rho V gamma x)/rho = V gamma in y and 0 in x."""
    c = _open_lattice(n=30)
    V, gamma = -0.6, 0.45
    c.v[:] = V
    o = oracle.OracleSim(c)
    n = o.n
    o.a["ut"][:n] = o.a["u"][:n] + gamma * o.a["x"][:n]
    o.evaluate()
    sel = _interior(o, c)
    np.testing.assert_allclose(o.field("av")[sel], V * gamma, rtol=2e-3)
    assert np.abs(o.field("au")[sel]).max() < 1e-10 * abs(V * gamma)


def test_blue_outlet_particles_take_the_previous_red_mean():
    """Eq. average_old (Sec. 3.4): an outlet particle without fluid in reach ("blue") takes J2
    as the mean of the previous step's J2 over the outlet particles within 3h that were red in
    the previous step (self included), 0 if there are none, and the mean of their previous
    advection velocities (else its frozen u average).  The stored previous-step values and red
    flags are planted at random (blue particles among the flagged ones, so that the flag and
    not the current class decides), one step is taken, and every blue particle's p - p_bar,
    u - u_bar, stored J2 and advection velocity are checked against a numpy evaluation over
    the brute-force neighbour lists."""
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=4, n_out=8)
    o = oracle.OracleSim(c)
    n = o.n
    rng = np.random.default_rng(21)
    tag = o.a["tag"][:n]
    out = tag == OUTLET
    J2p0 = np.where(out, rng.normal(0.0, 0.02, n), 0.0)
    adv0 = np.where(out, rng.uniform(0.8, 1.2, n), o.a["advp"][:n])
    red0 = np.where(out, rng.integers(0, 2, n), 0).astype(np.int32)
    o.a["J2p"][:n] = J2p0
    o.a["advp"][:n] = adv0
    o.a["redp"][:n] = red0
    hist = o.step(1)
    assert hist[0]["n_delete"] == hist[0]["n_to_outlet"] == hist[0]["n_spawn"] == 0
    assert o.n == n
    f = o.fields(("tag", "p", "u", "J2p", "advp", "redp", "ubar", "pbar"))
    start, idx = o.neighbors()
    rho_c = c.params.rho0 * c.params.cs
    nblue = nmix = 0
    for k in np.nonzero(f["tag"] == OUTLET)[0]:
        nb = idx[start[k]:start[k + 1]]
        if np.any(f["tag"][nb] == FLUID):
            continue
        nblue += 1
        assert f["redp"][k] == 0
        prev = nb[(f["tag"][nb] == OUTLET) & (red0[nb] == 1)]
        J2 = J2p0[prev].mean() if len(prev) else 0.0
        adv = adv0[prev].mean() if len(prev) else f["ubar"][k]
        nmix += len(prev) > 0 and len(prev) < np.count_nonzero(f["tag"][nb] == OUTLET)
        assert f["J2p"][k] == pytest.approx(J2, rel=1e-13, abs=1e-16)
        assert f["p"][k] - f["pbar"][k] == pytest.approx(0.5 * J2, rel=1e-12, abs=1e-16)
        assert f["u"][k] - f["ubar"][k] == pytest.approx(J2 / (2 * rho_c), rel=1e-9, abs=1e-16)
        assert f["advp"][k] == pytest.approx(adv, rel=1e-13)
    assert nblue > 50 and nmix > 50


def test_time_average_is_a_moving_window_of_n_avg_samples():
    """Eq. timeevg with N = n_avg = 6: after an ungated update, the average is the mean of the
    last six samples, i.e. the ring with its oldest entry (at the write index) replaced by the
    current value; the write index advances by one modulo 6 and J2 = rho0 c (u - u_bar) +
    (p - p_bar) (Eq. characteristic-vars against the average).  Rings and write indices are
    planted at random on every fluid particle."""
    c = cases.channel()
    o = oracle.OracleSim(c)
    n = o.n
    navg = c.params.n_avg
    assert navg == 6
    rng = np.random.default_rng(5)
    fl = o.a["tag"][:n] == FLUID
    ring = o.a["ring"].reshape(-1, oracle.NAVG_MAX, 3)
    planted = rng.normal(0.0, 0.3, (n, navg, 3)) + np.array([1.0, 0.0, 0.0])
    ring[:n, :navg][fl] = planted[fl]
    rpos0 = rng.integers(0, navg, n).astype(np.int32)
    o.a["rpos"][:n] = np.where(fl, rpos0, o.a["rpos"][:n])
    o.step(1)
    assert o.n == n
    f = o.fields(("tag", "u", "v", "p", "ubar", "vbar", "pbar", "J2", "rpos"))
    assert np.array_equal(f["tag"] == FLUID, fl)
    rho_c = c.params.rho0 * c.params.cs
    I = (0.5 * c.params.rho0 * c.params.U ** 2) ** 2 / (2 * c.params.rho0 * c.params.cs)
    assert np.all(f["p"][fl] ** 2 / (2 * c.params.rho0 * c.params.cs) <= I)  # ungated
    for i in np.nonzero(fl)[0]:
        win = planted[i].copy()
        win[rpos0[i]] = (f["u"][i], f["v"][i], f["p"][i])
        for comp, key in enumerate(("ubar", "vbar", "pbar")):
            assert f[key][i] == pytest.approx(win[:, comp].sum() / navg, rel=1e-13, abs=1e-15)
        assert f["rpos"][i] == (rpos0[i] + 1) % navg
        assert f["J2"][i] == pytest.approx(rho_c * (f["u"][i] - f["ubar"][i])
                                           + (f["p"][i] - f["pbar"][i]), rel=1e-9, abs=1e-13)


def test_integrator_stages_local_error():
    """The integrator (the paper defers it to the EDAC paper; read as the midpoint
    predictor-corrector whose stages update u, then u~ = u + tau a_bg, then x = x^n + tau u~,
    then p): velocity and pressure take the rates at the midpoint state, so their one-step
    error is O(h^3) (falling 8 times per halving of h; forward Euler, or a predictor of length
    h, gives O(h^2), a factor 4); the position takes the transport velocity at the end of the
    stage, x^(n+1) = x^n + h u^(n+1) = x^n + h u^n + h^2 a^(n+1/2), whose one-step error is
    +h^2 a / 2 (a position update with the midpoint velocity would give 0, one with u^n
    -h^2 a / 2).  Reference: the same state after 64 steps of h / 64.  p_b = 0 (no transport
    shift, itself proportional to h) and p_avg off (its neighbour count is not smooth in the
    positions) keep the map smooth; the seeded jitter makes the lattice disordered."""
    def make(h):
        c = cases.taylor_green(n=16, nu=0.05, jitter=0.2, seed=9)
        c.params.pb = 0.0
        c.params.use_pavg = 0
        c.params.dt = h
        return c

    dt = cases.taylor_green(n=16, nu=0.05).params.dt
    o0 = oracle.OracleSim(make(dt))
    a0 = np.concatenate([o0.field("au"), o0.field("av")])
    err_u, err_p, coef = {}, {}, {}
    for h in (dt, dt / 2, dt / 4):
        o = oracle.OracleSim(make(h))
        o.step(1)
        r = oracle.OracleSim(make(h / 64))
        r.step(64)
        err_u[h] = np.abs(o.field("u") - r.field("u")).max()
        err_p[h] = np.abs(o.field("p") - r.field("p")).max()
        dxy = np.concatenate([o.field("x") - r.field("x"), o.field("y") - r.field("y")])
        coef[h] = dxy / (0.5 * h * h * a0)
    for e in (err_u, err_p):
        assert 7.0 < e[dt] / e[dt / 2] < 9.0, e
        assert 7.0 < e[dt / 2] / e[dt / 4] < 9.0, e
    sel = np.abs(a0) > 0.3 * np.abs(a0).max()
    c4 = coef[dt / 4][sel]
    assert np.all(np.abs(c4 - 1.0) < 0.07), (c4.min(), c4.max())


# ------------------------------------------ unequal masses, walls, outlet state, recycling
def test_density_sums_the_neighbours_masses_and_the_volume_ignores_them():
    """Eq. summation-density sums m_j W_ij over the neighbours j, and the volume of Sec. 2 is the
    number-density one, V_i = 1 / sum_j W_ij: raising one particle's mass by dm raises the
    density of every particle within 3h of it by dm W(r) (itself by dm W(0)) and leaves every
    volume unchanged.  (With equal masses a sum of m_i W_ij, or V = m/rho, is indistinguishable
    from the definitions.)"""
    k = 137
    base = cases.taylor_green(n=16)
    o0 = oracle.OracleSim(base)
    heavy = cases.taylor_green(n=16)
    heavy.m = heavy.m.copy()
    dm = 2.0 * heavy.m[k]
    heavy.m[k] += dm
    o1 = oracle.OracleSim(heavy)
    p = base.params
    L = p.x_max - p.x_min
    dx = base.x - base.x[k]
    dy = base.y - base.y[k]
    dx = np.where(dx > 0.5 * L, dx - L, np.where(dx < -0.5 * L, dx + L, dx))
    dy = np.where(dy > 0.5 * L, dy - L, np.where(dy < -0.5 * L, dy + L, dy))
    r = np.hypot(dx, dy)
    want = dm * np.array([oracle.W(ri, p.h) for ri in r])
    assert np.count_nonzero(want) > 30
    np.testing.assert_allclose(o1.field("rho") - o0.field("rho"), want, rtol=0,
                               atol=1e-12 * o0.field("rho").max())
    assert np.array_equal(o1.field("V"), o0.field("V"))


def _pair(m=(1.0, 1.0), p=(0.0, 0.0), u=(0.0, 0.0), eta_reg=0.01, r_over_h=1.5):
    """Two fluid particles on the x axis of an open box, r = r_over_h h apart; masses in units
    of dx^2; p_avg off, no background pressure."""
    dx = 0.05
    h = 1.2 * dx
    prm = cases.Params(x_min=-1.0, x_max=1.0, y_min=-1.0, y_max=1.0, dx=dx, hdx=1.2, nu=0.01,
                       cs=10.0, pb=0.0, eta_reg=eta_reg, dt=1e-4, use_pavg=0, wall_drag=(0, 0))
    c = cases.Case("pair", prm, np.array([0.0, r_over_h * h]), np.zeros(2),
                   np.array(u, dtype=float), np.zeros(2), np.array(p, dtype=float),
                   np.array(m, dtype=float) * dx * dx, np.array([FLUID, FLUID], dtype=np.uint8),
                   np.arange(2, dtype=np.uint64), capacity=8)
    return oracle.OracleSim(c)


def test_interparticle_pressure_weights_each_pressure_by_the_other_density():
    """Eq. tvf-p-ij-basa: p~_ij = (rho_j p_i + rho_i p_j) / (rho_i + rho_j).  For two particles
    of unequal mass (so rho_i != rho_j), the pressure force on i with (p_i, p_j) = (1, 0) over
    the one with (0, 1) is p~(1, 0) / p~(0, 1) = rho_j / rho_i; the weights the other way
    round give rho_i / rho_j."""
    a = _pair(m=(1.0, 3.0), p=(1.0, 0.0))
    b = _pair(m=(1.0, 3.0), p=(0.0, 1.0))
    rho = a.field("rho")
    assert rho[1] > 1.5 * rho[0]
    assert a.field("au")[0] != 0.0
    assert a.field("au")[0] / b.field("au")[0] == pytest.approx(rho[1] / rho[0], rel=1e-12)


def test_viscous_coefficient_is_the_harmonic_mean_of_the_dynamic_viscosities():
    """Eq. tvf-momentum's eta~_ij = 2 eta_i eta_j / (eta_i + eta_j), eta = rho nu: with p = 0 and
    u~ = u the force on particle i of a moving pair is the viscous term alone, and neither
    c_ij (number-density volumes) nor the kernel depends on the masses, so the force with
    masses (1, 3) over the one with (1, 1) is eta~(rho_i, rho_j) / (rho_e nu), rho_e the density
    of the equal pair (the arithmetic mean would give (rho_i + rho_j) / (2 rho_e))."""
    e = _pair(m=(1.0, 1.0), u=(1.0, 0.0))
    q = _pair(m=(1.0, 3.0), u=(1.0, 0.0))
    rho_e = e.field("rho")
    assert rho_e[0] == rho_e[1]
    ri, rj = q.field("rho")
    want = (2.0 * ri * rj / (ri + rj)) / rho_e[0]
    assert q.field("au")[0] / e.field("au")[0] == pytest.approx(want, rel=1e-12)
    assert abs(want - 0.5 * (ri + rj) / rho_e[0]) > 0.05


def test_viscous_term_is_regularised_by_eta_h2():
    """The denominator of the viscous term of Eq. tvf-momentum is r^2 + eta h^2: the viscous force
    of a moving pair with eta = 0.01 over the one with eta = 0.5 is (r^2 + 0.5 h^2) / (r^2 +
    0.01 h^2), at r = 1.5 h 2.75 / 2.26."""
    a = _pair(u=(1.0, 0.0), eta_reg=0.01)
    b = _pair(u=(1.0, 0.0), eta_reg=0.5)
    assert a.field("au")[0] / b.field("au")[0] == pytest.approx(2.75 / 2.26, rel=1e-12)


def test_edac_divergence_term_carries_the_neighbour_mass_and_the_density_ratio():
    """Eq. p-edac's first term is sum_j (m_j rho_i / rho_j) c^2 u_ij . grad W_ij: for a moving pair
    at p = 0 (no diffusion term), dp_i/dt with masses (1, 3) over the one with (1, 1) is
    3 rho_i / rho_j."""
    e = _pair(m=(1.0, 1.0), u=(1.0, 0.0))
    q = _pair(m=(1.0, 3.0), u=(1.0, 0.0))
    ri, rj = q.field("rho")
    assert e.field("ap")[0] != 0.0
    assert q.field("ap")[0] / e.field("ap")[0] == pytest.approx(3.0 * ri / rj, rel=1e-12)


def test_body_force_is_added_to_the_acceleration():
    """Eq. tvf-momentum ends with + g: a fluid at rest at p = 0 on the periodic lattice feels
    exactly g."""
    c = cases.taylor_green(n=16)
    c.u[:] = 0.0
    c.v[:] = 0.0
    c.p[:] = 0.0
    c.params.gx, c.params.gy = 0.3, -0.2
    o = oracle.OracleSim(c)
    assert np.all(o.field("au") == 0.3) and np.all(o.field("av") == -0.2)


def test_wall_ghost_velocities_and_the_wall_velocity_without_fluid():
    """Walls (Adami et al., cited in Sec. 2, as read here): a slip wall whose normal is y takes
    (u_f, -v_f), a no-slip wall 2 u_w - u_f, Shepard averages of the fluid; a wall particle with
    no fluid in reach takes the wall velocity itself."""
    for slip in (1, 0):
        c = cases.poiseuille(n=10)
        c.tag[c.tag == WALL] = SLIPWALL if slip else WALL
        c.u[:] = np.where(c.tag == FLUID, 0.4, 0.0)
        c.v[:] = np.where(c.tag == FLUID, 0.3, 0.0)
        c.params.wall_u = (0.25, 0.25)
        c.params.wall_v = (-0.1, -0.1)
        o = oracle.OracleSim(c)
        f = o.fields()
        wl = f["tag"] != FLUID
        near = wl & (f["y"] > -3.1 * c.params.dx) & (f["y"] < 1 + 3.1 * c.params.dx)
        far = wl & ~near
        assert np.count_nonzero(near) > 10 and np.count_nonzero(far) > 5
        want = (0.4, -0.3) if slip else (2 * 0.25 - 0.4, 2 * -0.1 - 0.3)
        np.testing.assert_allclose(f["u"][near], want[0], rtol=0, atol=1e-14)
        np.testing.assert_allclose(f["v"][near], want[1], rtol=0, atol=1e-14)
        assert np.all(f["u"][far] == 0.25) and np.all(f["v"][far] == -0.1)


def test_wall_pressure_is_kernel_weighted():
    """The wall pressure is the Shepard average sum p_f W / sum W of the fluid: with a fluid
    particle at 0.5 h (p = 1) and one at 2.5 h (p = 0) the nearer one dominates, where a plain
    mean gives 1/2."""
    dx = 0.05
    h = 1.2 * dx
    prm = cases.Params(x_min=-1.0, x_max=1.0, y_min=-1.0, y_max=1.0, dx=dx, hdx=1.2, nu=0.01,
                       cs=10.0, pb=0.0, dt=1e-4, wall_drag=(0, 0))
    c = cases.Case("wall3", prm, np.array([0.0, 0.5 * h, -2.5 * h]), np.zeros(3), np.zeros(3),
                   np.zeros(3), np.array([0.0, 1.0, 0.0]), np.full(3, dx * dx),
                   np.array([WALL, FLUID, FLUID], dtype=np.uint8), np.arange(3, dtype=np.uint64),
                   capacity=8)
    o = oracle.OracleSim(c)
    w1, w2 = oracle.W(0.5 * h, h), oracle.W(2.5 * h, h)
    assert o.field("p")[0] == pytest.approx(w1 / (w1 + w2), rel=1e-14)
    assert o.field("p")[0] > 0.9


def test_solid_force_of_a_shear_flow_is_viscous_and_proportional_to_nu():
    """Eq. tvf-momentum_solid at p = 0 is its viscous term alone: fluid sliding at u past a no-slip
    wall at rest drags the wall in +x, and the force doubles exactly with nu (the ghost
    velocities do not depend on nu)."""
    fx = {}
    for nu in (0.05, 0.1):
        c = cases.poiseuille(n=10, nu=nu)
        c.params.gx = 0.0
        c.params.wall_drag = (1, 0)
        c.u[:] = np.where(c.tag == FLUID, 0.5, 0.0)
        c.p[:] = 0.0
        o = oracle.OracleSim(c)
        f = o.fields()
        bottom = (f["tag"] == WALL) & (f["y"] < 0.0)
        fx[nu] = f["fx"][bottom].sum()
        assert np.all(f["fy"][bottom] == 0.0) or np.abs(f["fy"][bottom]).max() < 1e-12 * abs(fx[nu])
    assert fx[0.05] > 0.0
    assert fx[0.1] / fx[0.05] == pytest.approx(2.0, rel=1e-12)


def _channel_with_events(outlet_kind=0, seed=31):
    c = cases.channel(jitter=0.02, n_in=4, n_out=8)
    c.params.outlet_kind = outlet_kind
    rng = np.random.default_rng(seed)
    fl = c.tag == FLUID
    c.u[:] = np.where(fl, 1.0 + 0.05 * rng.standard_normal(c.n), c.u)
    c.v[:] = np.where(fl, 0.05 * rng.standard_normal(c.n), c.v)
    c.p[:] = np.where(fl, c.p + 0.05, c.p)
    return c


def test_hybrid_outlet_keeps_the_average_transverse_velocity():
    """Sec. 3.4: the hybrid outlet sets an outlet particle's value to its frozen average plus the
    acoustic part carried by J2 (Eq. acou); the transverse velocity has no acoustic part and
    stays at its average.  The outlet particles' v is disturbed after set-up; one step later
    every outlet particle has v = v_bar again."""
    c = _channel_with_events()
    o = oracle.OracleSim(c)
    n = o.n
    out = o.a["tag"][:n] == OUTLET
    o.a["v"][:n] = np.where(out, o.a["v"][:n] + 0.07, o.a["v"][:n])
    o.step(1)
    f = o.fields(("tag", "v", "vbar"))
    out = f["tag"] == OUTLET
    assert np.count_nonzero(out) > 100
    assert np.array_equal(f["v"][out], f["vbar"][out])


def test_red_outlet_value_is_the_shepard_average_of_the_fluid():
    """Eqs. shepard0 and shepard (Secs. 3.1.1 and 3.4): an outlet particle with fluid in reach
    takes the kernel-weighted (Shepard) average of the fluid value; with the modified
    do-nothing outlet that is its advection velocity, the Shepard average of the fluid u.
    Checked against the probe at the particle's position (the Shepard average of the fluid,
    itself pinned), over a fluid u rising towards the outlet, where the plain mean of the
    fluid neighbours differs; particles near a fluid particle that converted in the step are
    left out (the probe sees it as outlet)."""
    c = _channel_with_events(outlet_kind=2)
    c.u[:] = np.where(c.tag == FLUID, 1.0 + 2.0 * (c.x - c.params.x_out), c.u)
    o = oracle.OracleSim(c, max_events=100000)
    o.step(1)
    ev = o.events()
    f = o.fields(("x", "y", "u", "tag", "id", "advp", "redp"))
    conv = np.isin(f["id"], ev["id"][ev["kind"] == 1])
    rc = 3.0 * c.params.h
    red = np.nonzero((f["tag"] == OUTLET) & (f["redp"] == 1))[0]
    keep = [k for k in red
            if not np.any(np.hypot(f["x"][conv] - f["x"][k], f["y"][conv] - f["y"][k]) < rc)]
    assert len(keep) > 20
    keep = np.array(keep)
    pr = o.probe(f["x"][keep], f["y"][keep])
    np.testing.assert_allclose(f["advp"][keep], pr[:, 1], rtol=1e-13)
    start, idx = o.neighbors()
    plain = np.array([f["u"][nb[f["tag"][nb] == FLUID]].mean()
                      for nb in (idx[start[k]:start[k + 1]] for k in keep)])
    assert np.abs(f["advp"][keep] - plain).max() > 1e-2


def test_outlet_particles_move_with_their_advection_velocity():
    """Sec. 3.4 (as read, like the do-nothing update of Sec. 3.1): an outlet particle moves in x
    with the advection velocity the previous outlet update chose for it, not with its u, and
    its y stays fixed: x^(n+1) = x^n + dt adv^n.  With the modified do-nothing outlet (Sec.
    3.1.1) the two differ: u stays frozen, adv is the Shepard average of the fluid u."""
    c = _channel_with_events(outlet_kind=2)
    o = oracle.OracleSim(c)
    o.step(3)
    f0 = o.fields(("x", "y", "u", "tag", "id", "advp"))
    o.step(1)
    f1 = o.fields(("x", "y", "tag", "id"))
    dt = c.params.dt
    out0 = f0["tag"] == OUTLET
    pos = {int(i): k for k, i in enumerate(f1["id"])}
    idx0 = [k for k in np.nonzero(out0)[0] if int(f0["id"][k]) in pos]
    idx1 = [pos[int(f0["id"][k])] for k in idx0]
    np.testing.assert_allclose(f1["x"][idx1], f0["x"][idx0] + dt * f0["advp"][idx0], rtol=0, atol=1e-14)
    np.testing.assert_array_equal(f1["y"][idx1], f0["y"][idx0])
    assert np.abs(f0["advp"][idx0] - f0["u"][idx0]).max() > 1e-4


def test_crossing_and_spawned_particles_take_their_stated_values():
    """End of Sec. 3.4 (as read): a fluid particle entering the hybrid outlet takes its time
    averages (u, v, p) = (u_bar, v_bar, p_bar) and advects with u_bar; a particle spawned at the
    inlet when its parent becomes fluid starts one inlet length behind the parent with the
    parent's pressure and mass and the prescribed inlet velocity, and the parent, now fluid,
    starts its time window (Eq. timeevg) from its current values.  No particle is left on the
    wrong side of its line after a step."""
    c = _channel_with_events()
    o = oracle.OracleSim(c, max_events=100000)
    nconv = nspawn = 0
    spread = 0.0
    navg = c.params.n_avg
    L_in = c.params.n_in_layers * c.params.dx
    for _ in range(45):
        o.step(1)
        ev = o.events()
        f = o.fields(("x", "y", "u", "v", "p", "m", "tag", "id", "ubar", "vbar", "pbar", "advp",
                      "rpos", "J2"))
        pos = {int(i): k for k, i in enumerate(f["id"])}
        ring = o.a["ring"].reshape(-1, oracle.NAVG_MAX, 3)[:, :navg]
        for i in ev["id"][ev["kind"] == 1]:
            k = pos[int(i)]
            assert f["tag"][k] == OUTLET
            for a, b in (("u", "ubar"), ("v", "vbar"), ("p", "pbar"), ("advp", "ubar")):
                assert f[a][k] == f[b][k]
            # the averages are the window's (Eq. timeevg), not the values at the crossing
            for comp, b in enumerate(("ubar", "vbar", "pbar")):
                assert f[b][k] == pytest.approx(ring[k, :, comp].sum() / navg, rel=1e-13, abs=1e-15)
            spread = max(spread, np.ptp(ring[k, :, 0]))
            nconv += 1
        for i, par in zip(ev["id"][ev["kind"] == 2], ev["other"][ev["kind"] == 2]):
            k, q = pos[int(i)], pos[int(par)]
            assert f["tag"][k] == INLET and f["tag"][q] == FLUID
            assert f["p"][k] == f["p"][q] and f["m"][k] == f["m"][q] and f["y"][k] == f["y"][q]
            assert f["x"][k] == pytest.approx(f["x"][q] - L_in, abs=1e-15)
            assert f["u"][k] == c.params.U and f["v"][k] == 0.0
            # the parent, fluid from now on, starts its time window from its current values
            assert f["rpos"][q] == 0 and f["J2"][q] == 0.0
            for a, b in (("u", "ubar"), ("v", "vbar"), ("p", "pbar")):
                assert f[a][q] == f[b][q]
            assert np.all(ring[q, :, 0] == f["u"][q]) and np.all(ring[q, :, 2] == f["p"][q])
            nspawn += 1
        # every crossing is taken in the step it happens (the lines are x_in, x_out and
        # x_out + L_out)
        assert np.all(f["x"][f["tag"] == INLET] < c.params.x_in)
        fl = f["tag"] == FLUID
        assert np.all((f["x"][fl] >= c.params.x_in) & (f["x"][fl] < c.params.x_out))
        L_out = c.params.n_out_layers * c.params.dx
        assert np.all(f["x"][f["tag"] == OUTLET] < c.params.x_out + L_out)
    assert nconv > 20 and nspawn > 20
    assert spread > 1e-3  # the window's samples differ: its mean is not the crossing value


def _half_refined_block(refine, dx=0.05, n=16):
    """Fluid on [-n dx, n dx]^2; for refine, the half x > 0 at half the spacing in x and half
    the mass (the same density).  p is a quadratic field."""
    xs, ys, ms = [], [], []
    for j in range(-n, n):
        for i in range(-n, 0):
            xs.append((i + 0.5) * dx); ys.append((j + 0.5) * dx); ms.append(dx * dx)
        k = 2 if refine else 1
        for i in range(0, k * n):
            xs.append((i + 0.5) * dx / k); ys.append((j + 0.5) * dx); ms.append(dx * dx / k)
    x, y, m = np.array(xs), np.array(ys), np.array(ms)
    prm = cases.Params(x_min=-2.0, x_max=2.0, y_min=-2.0, y_max=2.0, dx=dx, hdx=1.2, nu=0.01,
                       cs=10.0, pb=0.0, dt=1e-4, use_pavg=0, wall_drag=(0, 0))
    p = (x - 0.013) ** 2 + 0.5 * (y + 0.02) ** 2
    c = cases.Case("half_refined", prm, x, y, np.zeros_like(x), np.zeros_like(x), p, m,
                   np.full(len(x), FLUID, dtype=np.uint8), np.arange(len(x), dtype=np.uint64),
                   capacity=len(x) + 8)
    return oracle.OracleSim(c)


def test_mirror_sums_are_quadratures_with_the_particle_volumes():
    """The sums of Eq. matform weight each fluid particle by its volume V_l = m_l / rho_l, so that
    they approximate integrals over the support whatever the particle spacing: with half of
    the support refined (half the spacing and half the mass, so V halves) the extrapolated
    value and gradient of a quadratic field move by the discretisation error only (a few %
    of the gradient), where unit weights would count the refined half twice (~45%)."""
    qx = np.array([0.0, 0.011, -0.017, 0.03])
    qy = np.array([0.0, 0.021, -0.013, 0.0])
    a = _half_refined_block(False).mirror_points(qx, qy)
    b = _half_refined_block(True).mirror_points(qx, qy)
    gscale = 0.03  # |grad p| near the origin
    assert np.abs(a[1] - b[1]).max() < 0.1 * gscale
    assert np.abs(a[2] - b[2]).max() < 0.1 * gscale
    assert np.abs(a[0] - b[0]).max() < 0.03 * np.abs(a[0]).max()


def test_the_scheme_is_invariant_under_a_change_of_density_scale():
    """The equations hold in any unit of mass: with rho0, the masses, the pressures and p_b all
    multiplied by 1000 (the same fluid in other units: p/rho, nu, c and the geometry unchanged),
    every velocity, position, gate decision and recycling event stays the same and the
    pressures and densities scale by 1000.  This pins each place a density multiplies a term:
    the dynamic viscosities of both diffusion terms, rho_i/rho_j, the A-term's densities,
    the acoustic intensity and its threshold (Eq. acouinten), rho0 c in J2 (Eq.
    characteristic-vars) and in its inversion (Eq. acou).  The pulse is strong enough for the
    gate to close near it."""
    runs = {}
    for k in (1.0, 1000.0):
        c = cases.channel(pulse_amp=1.0, jitter=0.05, seed=3)
        c.params.rho0 *= k
        c.params.pb *= k
        c.m = c.m * k
        c.p = c.p * k
        o = oracle.OracleSim(c)
        o.step(25)
        runs[k] = o.fields(("x", "y", "u", "v", "ut", "vt", "p", "rho", "V", "tag", "id", "rpos",
                            "ubar", "pbar", "J2", "au", "ap"))
    a, b = runs[1.0], runs[1000.0]
    for key in ("tag", "id", "rpos"):
        assert np.array_equal(a[key], b[key]), key
    assert len(np.unique(a["rpos"][a["tag"] == FLUID])) > 1  # some rings were gated
    for key in ("x", "y"):
        np.testing.assert_allclose(b[key], a[key], rtol=0, atol=1e-13)
    for key in ("u", "v", "ut", "vt", "ubar", "V", "au"):
        np.testing.assert_allclose(b[key], a[key], rtol=0, atol=1e-10 * np.abs(a[key]).max())
    for key in ("p", "rho", "pbar", "J2", "ap"):
        np.testing.assert_allclose(b[key], 1000.0 * a[key], rtol=0,
                                   atol=1e-10 * 1000.0 * np.abs(a[key]).max())
    assert np.abs(a["J2"]).max() > 1e-4


def _fluid_row(p0=0.7, dx=0.05):
    n = 21
    x = (np.arange(n) - 10) * dx
    prm = cases.Params(x_min=-2.0, x_max=2.0, y_min=-2.0, y_max=2.0, dx=dx, hdx=1.2, nu=0.01,
                       cs=10.0, pb=0.0, dt=1e-4, use_pavg=0, wall_drag=(0, 0))
    c = cases.Case("row", prm, x, np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, p0),
                   np.full(n, dx * dx), np.full(n, FLUID, dtype=np.uint8),
                   np.arange(n, dtype=np.uint64), capacity=n + 8)
    return oracle.OracleSim(c)


def test_mirror_without_fluid_or_with_a_singular_system():
    """Readings of Sec. 3.2's mirror: a point with no fluid in reach gets p = 0 and no gradient;
    a point whose fluid neighbours lie on one line (the 3x3 system of Eq. matform is
    singular: no y moments) gets the Shepard value sum p W V / sum W V and no gradient, which
    for a constant field is that constant."""
    o = _fluid_row()
    pk, gx, gy = o.mirror_points(np.array([0.013, 0.0]), np.array([0.0, 1.5]))
    assert pk[0] == pytest.approx(0.7, rel=1e-14) and gx[0] == 0.0 and gy[0] == 0.0
    assert pk[1] == 0.0 and gx[1] == 0.0 and gy[1] == 0.0


def test_inlet_profile_modes_at_their_special_heights():
    """Sec. 3's inlet profile u(y) = U + sum_k a_k sin(k pi (y - y0) / H) with y0 = -0.15 and
    H = 0.8 on the channel's inlet: mode 1 adds a_1 at mid-height y0 + H/2 = 0.25 and
    a_1 / sqrt(2) at the quarter heights 0.05 and 0.45; mode 2 adds nothing at mid-height,
    +a_2 at 0.05 and -a_2 at 0.45; v = 0."""
    for modes, want in (((0.3,), {0.25: 0.3, 0.05: 0.3 / math.sqrt(2), 0.45: 0.3 / math.sqrt(2)}),
                        ((0.0, 0.2), {0.25: 0.0, 0.05: 0.2, 0.45: -0.2})):
        c = cases.channel(jitter=0.0, pulse_amp=0.0)
        c.params.inlet_modes = modes
        c.params.inlet_y0 = -0.15
        c.params.inlet_h = 0.8
        o = oracle.OracleSim(c)
        o.step(1)
        f = o.fields(("y", "u", "v", "tag"))
        inl = f["tag"] == INLET
        assert np.all(f["v"][inl] == 0.0)
        for y, du in want.items():
            at = inl & (np.abs(f["y"] - y) < 1e-9)
            assert np.count_nonzero(at) >= 3
            np.testing.assert_allclose(f["u"][at], c.params.U + du, rtol=0, atol=1e-12)


def test_ramp_inlet_holds_the_free_stream_after_the_ramp():
    """Sec. 4.3's ramp u = U min(t / T, 1): after t = T the inlet velocity stays at U."""
    c = cases.outlet_problem("ramp")
    T = 5 * c.params.dt
    c.params.inlet_prm = (T,)
    o = oracle.OracleSim(c, neighbor_mode=1)
    o.step(20)
    f = o.fields(("u", "tag"))
    assert o.t > 3 * T
    assert np.all(f["u"][f["tag"] == INLET] == c.params.U)


def test_new_ids_continue_from_the_largest_id_in_ascending_parent_order():
    """Recycling hands out ids after the largest id in use, one per spawn, in ascending order of
    the parents' ids (the canonical order that makes runs comparable); with input ids that
    are neither contiguous nor in array order, the array order would give another
    assignment."""
    c = cases.channel()
    rng = np.random.default_rng(8)
    c.id = (10 * rng.permutation(c.n) + 7).astype(np.uint64)
    nxt = int(c.id.max()) + 1
    o = oracle.OracleSim(c, max_events=100000)
    nsp = 0
    for _ in range(60):
        o.step(1)
        ev = o.events()
        sp = ev["kind"] == 2
        new, par = ev["id"][sp].astype(np.int64), ev["other"][sp].astype(np.int64)
        np.testing.assert_array_equal(new, nxt + np.arange(len(new)))
        assert np.all(np.diff(par) > 0)
        nxt += len(new)
        nsp += len(new)
    assert nsp > 20


def test_force_history_is_the_sum_over_the_counted_solids():
    """The drag/lift record of a step (Sec. 4.6's c_d, c_l) sums fx and fy of the solid
    particles counted in the drag, as evaluated at the end of the step."""
    c = cases.cylinder(dx=1.0 / 8.0, Lx=6.0, H=4.0, xc=2.0)
    o = oracle.OracleSim(c, neighbor_mode=1)
    o.step(3)
    h = o.history[-1]
    f = o.fields(("fx", "fy", "tag"))
    counted = f["tag"] == WALL  # the cylinder; the slip walls are not counted
    assert np.abs(f["fy"][counted]).max() > 0.0
    assert h["fx"] == pytest.approx(f["fx"][counted].sum(), rel=1e-12)
    assert h["fy"] == pytest.approx(f["fy"][counted].sum(), rel=1e-12, abs=1e-15)
    assert np.all(f["fx"][f["tag"] == SLIPWALL] == 0.0)


def test_rates_are_computed_for_fluid_and_inlet_particles_only():
    """Eq. tvf-momentum and Eq. p-edac hold for the fluid and for the inlet particles (an inlet
    particle that becomes fluid starts from the rates computed for it): the inlet particles'
    rates, with the pressure the mirror gave them, are those they get as fluid particles of
    the same state.  Outlet and wall particles carry no rates, and a wall's transport
    velocity is its ghost velocity (no A-term from it)."""
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=6)
    c.p[:] = np.where(c.tag == FLUID, 0.1 * (1.0 - c.x), 0.0)
    o = oracle.OracleSim(c)
    f = o.fields(("tag", "x", "y", "au", "av", "ap", "u", "v", "p"))
    inl = f["tag"] == INLET
    assert np.abs(f["au"][inl]).max() > 0.01 and np.abs(f["ap"][inl]).max() > 0.01
    as_fluid = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=6)
    assert np.array_equal(as_fluid.x, f["x"]) and np.array_equal(as_fluid.y, f["y"])
    as_fluid.tag = np.where(as_fluid.tag == INLET, FLUID, as_fluid.tag).astype(np.uint8)
    as_fluid.p, as_fluid.u, as_fluid.v = f["p"].copy(), f["u"].copy(), f["v"].copy()
    g = oracle.OracleSim(as_fluid).fields(("au", "av", "ap"))
    for key in ("au", "av", "ap"):
        np.testing.assert_array_equal(g[key][inl], f[key][inl])
    for t in (OUTLET, WALL, SLIPWALL):
        sel = f["tag"] == t
        assert np.all(f["au"][sel] == 0.0) and np.all(f["ap"][sel] == 0.0)
    cy = cases.poiseuille(n=10)
    cy.u[:] = np.where(cy.tag == FLUID, 0.4, 0.0)
    w = oracle.OracleSim(cy).fields(("tag", "u", "v", "ut", "vt"))
    wl = w["tag"] == WALL
    assert np.array_equal(w["ut"][wl], w["u"][wl]) and np.array_equal(w["vt"][wl], w["v"][wl])
    assert np.abs(w["u"][wl]).max() > 0.1
    sw = cases.poiseuille(n=10)
    sw.u[:] = np.where(sw.tag == FLUID, 0.4, 0.0)
    sw.params.wall_drag = (0, 0)
    ow = oracle.OracleSim(sw).fields(("tag", "au", "ap"))
    assert np.all(ow["au"][ow["tag"] == WALL] == 0.0)


@pytest.mark.parametrize("kind", ["mod_donothing", "characteristic", "mirror"])
def test_blue_rules_of_the_other_outlets(kind):
    """Where the Shepard interpolation of the fluid does not reach (Sec. 3.4's blue particles):
    the modified do-nothing outlet (Sec. 3.1.1) advects a blue particle with the mean previous
    advection velocity of its previously red neighbours, else with its frozen u average; the
    characteristic outlet (Sec. 3.3) takes J2 as their mean previous J2 and advects with that
    mean velocity, else (J2 = 0) with its own u = u_ref; the mirrored outlet (Sec. 3.2) keeps
    no red flags or J2.  Previous values, flags and frozen averages are planted at random."""
    c = cases.channel(jitter=0.0, pulse_amp=0.0, n_in=4, n_out=12)
    c.params.outlet_kind = OUTLET_KINDS[kind]
    o = oracle.OracleSim(c)
    n = o.n
    rng = np.random.default_rng(33)
    out = o.a["tag"][:n] == OUTLET
    J2p0 = np.where(out, rng.normal(0.0, 0.02, n), 0.0)
    adv0 = np.where(out, rng.uniform(0.8, 1.2, n), o.a["advp"][:n])
    # red flags in the first outlet layers only, so that the deepest blue particles have none
    front = o.a["x"][:n] < c.params.x_out + 5 * c.params.dx
    red0 = np.where(out & front, rng.integers(0, 2, n), 0).astype(np.int32)
    o.a["ubar"][:n] = np.where(out, rng.uniform(0.9, 1.1, n), o.a["ubar"][:n])
    o.a["J2p"][:n] = J2p0
    o.a["advp"][:n] = adv0
    o.a["redp"][:n] = red0
    o.step(1)
    f = o.fields(("tag", "u", "J2p", "advp", "redp", "ubar"))
    out = f["tag"] == OUTLET
    if kind == "mirror":
        assert np.all(f["redp"][out] == 0) and np.all(f["J2p"][out] == 0.0)
        return
    start, idx = o.neighbors()
    rho_c = c.params.rho0 * c.params.cs
    nblue = nnone = 0
    for k in np.nonzero(out)[0]:
        nb = idx[start[k]:start[k + 1]]
        if np.any(f["tag"][nb] == FLUID):
            continue
        nblue += 1
        prev = nb[(f["tag"][nb] == OUTLET) & (red0[nb] == 1)]
        nnone += len(prev) == 0
        if kind == "mod_donothing":
            want = adv0[prev].mean() if len(prev) else f["ubar"][k]
            assert f["advp"][k] == pytest.approx(want, rel=1e-13)
        else:
            J2 = J2p0[prev].mean() if len(prev) else 0.0
            assert f["J2p"][k] == pytest.approx(J2, rel=1e-13, abs=1e-16)
            assert f["u"][k] == pytest.approx(c.params.U + J2 / (2 * rho_c), rel=1e-13)
            want = adv0[prev].mean() if len(prev) else f["u"][k]
            assert f["advp"][k] == pytest.approx(want, rel=1e-13)
    assert nblue > 50 and nnone > 5


@pytest.mark.parametrize("other", [INLET, OUTLET, WALL])
def test_wall_values_come_from_the_fluid_alone(other):
    """A wall's Shepard projection runs over its fluid neighbours only: a neighbour of another
    kind, whatever its pressure and velocity, changes nothing."""
    dx = 0.05
    h = 1.2 * dx
    prm = cases.Params(x_min=-1.0, x_max=1.0, y_min=-1.0, y_max=1.0, dx=dx, hdx=1.2, nu=0.01,
                       cs=10.0, pb=0.0, dt=1e-4, wall_drag=(0, 0), has_inlet=1, x_in=-0.5,
                       has_outlet=1, x_out=-0.5)
    c = cases.Case("wall_other", prm, np.array([0.0, 0.5 * h, -0.5 * h]), np.zeros(3),
                   np.array([0.0, 0.3, 2.0]), np.array([0.0, 0.1, -1.0]),
                   np.array([0.0, 1.0, 5.0]), np.full(3, dx * dx),
                   np.array([WALL, FLUID, other], dtype=np.uint8), np.arange(3, dtype=np.uint64),
                   capacity=8)
    o = oracle.OracleSim(c)
    f = o.fields(("p", "u", "v"))
    assert f["p"][0] == 1.0 and f["u"][0] == -0.3 and f["v"][0] == -0.1


def test_outlet_particles_are_red_only_through_fluid_and_keep_their_frozen_averages():
    """An outlet particle is red when fluid is in reach (Sec. 3.4): a wall in reach does not make
    it red.  And the outlet's time averages are frozen at the crossing: the outlet particles'
    u_bar, v_bar, p_bar do not change from step to step while their u and p do."""
    c = cases.channel(jitter=0.02, n_in=4, n_out=8)
    c.p[:] = np.where(c.tag == FLUID, c.p + 0.02 * np.sin(7.0 * c.y), c.p)
    far = (c.tag == OUTLET) & (c.x > c.params.x_out + 6.5 * c.params.dx)
    c.tag = np.where(far & (c.y < 0.1), WALL, c.tag).astype(np.uint8)  # walls among blue ones
    c.params.wall_drag = (0, 0)
    o = oracle.OracleSim(c)
    o.step(2)
    f0 = o.fields(("id", "tag", "x", "ubar", "vbar", "pbar", "u", "p", "redp"))
    start, idx = o.neighbors()
    walled = 0
    for k in np.nonzero(f0["tag"] == OUTLET)[0]:
        nb = idx[start[k]:start[k + 1]]
        if not np.any(f0["tag"][nb] == FLUID) and np.any(f0["tag"][nb] == WALL):
            assert f0["redp"][k] == 0
            walled += 1
    assert walled > 5
    o.step(3)
    f1 = o.fields(("id", "tag", "ubar", "vbar", "pbar", "u", "p"))
    pos = {int(i): k for k, i in enumerate(f1["id"])}
    both = [(k, pos[int(i)]) for k, i in enumerate(f0["id"])
            if f0["tag"][k] == OUTLET and int(i) in pos]
    assert len(both) > 100
    a, b = np.array([q[0] for q in both]), np.array([q[1] for q in both])
    for key in ("ubar", "vbar", "pbar"):
        assert np.array_equal(f0[key][a], f1[key][b]), key
    assert np.abs(f0["p"][a] - f1["p"][b]).max() > 1e-6


def test_a_zero_intensity_threshold_closes_the_gate_for_any_pressure():
    """edac_set_outlet's i_thresh >= 0 replaces Eq. acouinten's threshold; 0 admits only samples
    of exactly zero pressure: every fluid particle of the pulse channel keeps its window."""
    c = cases.channel()
    c.params.i_thresh = 0.0
    o = oracle.OracleSim(c)
    o.step(1)
    f = o.fields(("tag", "p", "rpos"))
    fl = f["tag"] == FLUID
    assert np.all(f["p"][fl] != 0.0)
    assert np.all(f["rpos"][fl] == 0)


def test_spawned_inlet_particles_take_the_inlet_velocity_at_the_end_of_the_step():
    """A particle spawned at the end of a step takes the inlet velocity at the new time level
    t^(n+1): during the ramp of Sec. 4.3, u = U t^(n+1) / T."""
    c = cases.outlet_problem("ramp")
    o = oracle.OracleSim(c, neighbor_mode=1, max_events=100000)
    T = c.params.inlet_prm[0]
    nsp = 0
    while nsp < 20 and o.t < 0.9 * T:
        o.step(1)
        ev = o.events()
        f = o.fields(("id", "u"))
        pos = {int(i): k for k, i in enumerate(f["id"])}
        for i in ev["id"][ev["kind"] == 2]:
            assert f["u"][pos[int(i)]] == pytest.approx(c.params.U * o.t / T, rel=1e-13)
            nsp += 1
    assert nsp >= 20


def test_mirror_solves_ill_conditioned_systems_that_are_not_singular():
    """The Shepard fallback of the mirror is for singular systems only: with the fluid in two rows
    at one and two smoothing lengths from the mirror point (a one-sided support: the system
    of Eq. matform is ill-conditioned, |det M| / |M00 M11 M22| ~ 0.05, but regular), the
    Taylor solve still returns a linear field's value and gradient exactly."""
    dx = 0.05
    h = 1.2 * dx
    xs = (np.arange(21) - 10) * dx
    x = np.r_[xs, xs]
    y = np.r_[np.full(21, h), np.full(21, 2 * h)]
    n = len(x)
    p = 0.3 + 2.0 * x - 1.5 * y
    prm = cases.Params(x_min=-2.0, x_max=2.0, y_min=-2.0, y_max=2.0, dx=dx, hdx=1.2, nu=0.01,
                       cs=10.0, pb=0.0, dt=1e-4, use_pavg=0, wall_drag=(0, 0))
    c = cases.Case("two_rows", prm, x, y, np.zeros(n), np.zeros(n), p, np.full(n, dx * dx),
                   np.full(n, FLUID, dtype=np.uint8), np.arange(n, dtype=np.uint64), capacity=n + 8)
    o = oracle.OracleSim(c)
    qx = np.array([0.013, -0.021])
    pk, gx, gy = o.mirror_points(qx, np.zeros(2))
    np.testing.assert_allclose(pk, 0.3 + 2.0 * qx, rtol=0, atol=1e-9)
    np.testing.assert_allclose(gx, 2.0, rtol=0, atol=1e-7)
    np.testing.assert_allclose(gy, -1.5, rtol=0, atol=1e-7)
