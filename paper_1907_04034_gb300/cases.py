"""Seeded synthetic problem generators (particle lattices, rings, initial fields).

This module is the only code shared by the CUDA path and the CPU oracle. It holds
no arithmetic of the SPH method itself: it places particles, draws the seeded
jitter, fills the initial velocity/pressure fields the workload prescribes, and
collects the run parameters. Both sides receive its output as plain arrays.

Workloads (all 2D, rho0 = 1, U = 1, c_s = 10 U, h = 1.2 dx, support 3h):

* ``channel``   -- the pulse channel: [0,1]x[0,0.5], periodic in y, dx = 0.02,
  3 inlet layers at x<0, 5 hybrid-outlet layers at x>1, nu = 0.01, Gaussian
  pressure pulse p = 0.1 exp(-((x-0.5)^2+(y-0.25)^2)/0.005), fluid jitter of
  +-0.01 dx (uniform, seeded).
* ``cylinder``  -- flow past a circular cylinder D = 1 centred 5D behind the
  inlet of a 15D x 10D channel, slip walls top and bottom (4 layers), 3 solid
  rings in the cylinder (the paper's ring fill, Sec. 4.6), uniform inlet U = 1,
  hybrid outlet; dx = D/40 (~245k particles), D/100 (~1.5M), D/25 (~95k).
* ``taylor_green`` -- doubly periodic unit box (used to pin the scheme).
* ``poiseuille``   -- x-periodic channel between no-slip walls, body force g.
* ``random_box``   -- small seeded boxes with random tags (property tests).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict

import numpy as np

FLUID, INLET, OUTLET, WALL, SLIPWALL = 0, 1, 2, 3, 4
TAG_NAMES = {FLUID: "fluid", INLET: "inlet", OUTLET: "outlet", WALL: "wall", SLIPWALL: "slipwall"}


@dataclasses.dataclass
class Params:
    """Run parameters (SI units, all floating point fp64)."""
    x_min: float
    x_max: float
    y_min: float
    y_max: float
    periodic_x: int = 0
    periodic_y: int = 0
    dx: float = 0.02
    hdx: float = 1.2
    rho0: float = 1.0
    U: float = 1.0
    nu: float = 0.01
    cs: float = 10.0
    alpha: float = 0.5
    pb: float = 100.0          # background pressure; rho0 * cs^2 by default
    eta_reg: float = 0.01
    gx: float = 0.0
    gy: float = 0.0
    dt: float = 0.0
    use_pavg: int = 1
    # inlet
    has_inlet: int = 0
    x_in: float = 0.0
    n_in_layers: int = 3
    inlet_modes: tuple = ()    # a_k of u(y) = U + sum a_k sin(k pi (y - inlet_y0) / inlet_h)
    inlet_y0: float = 0.0
    inlet_h: float = 1.0
    # inlet velocity in time: 0 steady modes, 1 2D pulse (A, t0, t1, delta), 2 ramp (T),
    # 3 passing vortex (Gamma, core, d0, y_c) of the Sec. 4 test problems
    inlet_kind: int = 0
    inlet_prm: tuple = ()
    # outlet (hybrid)
    has_outlet: int = 0
    x_out: float = 1.0
    n_out_layers: int = 5
    n_avg: int = 6
    i_thresh: float = -1.0     # < 0: use the acoustic-intensity formula
    # outlet treatment: 0 hybrid (Sec. 3.4), 1 do-nothing (Sec. 3.1), 2 modified do-nothing
    # (Sec. 3.1.1), 3 method of characteristics (Sec. 3.3), 4 mirroring (Sec. 3.2)
    outlet_kind: int = 0
    moc_ref: tuple = ()        # (u_ref, p_ref) of the characteristic outlet; () = (U, 0)
    # walls: per wall tag (WALL, SLIPWALL): slip flag, wall velocity, counted in drag (0 no;
    # 1 fluid neighbours with the interpolated pressure; 2 Eq. tvf-momentum_solid as printed:
    # every neighbour, p~_ij with the solid particle's p_avg)
    wall_slip: tuple = (0, 1)
    wall_u: tuple = (0.0, 0.0)
    wall_v: tuple = (0.0, 0.0)
    wall_drag: tuple = (1, 0)
    drag_length: float = 1.0   # reference length D of c_d = F / (0.5 rho U^2 D)

    @property
    def h(self) -> float:
        return self.hdx * self.dx


@dataclasses.dataclass
class Case:
    name: str
    params: Params
    x: np.ndarray
    y: np.ndarray
    u: np.ndarray
    v: np.ndarray
    p: np.ndarray
    m: np.ndarray
    tag: np.ndarray
    id: np.ndarray
    capacity: int

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def arrays(self) -> Dict[str, np.ndarray]:
        return dict(x=self.x, y=self.y, u=self.u, v=self.v, p=self.p, m=self.m,
                    tag=self.tag, id=self.id)

    def count(self, tag: int) -> int:
        return int(np.count_nonzero(self.tag == tag))


def default_dt(dx: float, hdx: float, cs: float, U: float, nu: float) -> float:
    """Time step recipe of the channel workload: min(0.25 h/(c+U), 0.125 h^2/nu)."""
    h = hdx * dx
    return min(0.25 * h / (cs + U), 0.125 * h * h / nu if nu > 0 else math.inf)


def _lattice(x0: float, nx: int, y0: float, ny: int, dx: float):
    """Cell-centred square lattice: x0 + (i+1/2) dx, y0 + (j+1/2) dx."""
    xs = x0 + (np.arange(nx, dtype=np.float64) + 0.5) * dx
    ys = y0 + (np.arange(ny, dtype=np.float64) + 0.5) * dx
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return X.ravel().copy(), Y.ravel().copy()


def _assemble(name, params, parts, capacity_extra, seed_ids=0):
    x = np.concatenate([q[0] for q in parts])
    y = np.concatenate([q[1] for q in parts])
    tag = np.concatenate([np.full(q[0].shape, q[2], dtype=np.uint8) for q in parts])
    n = x.shape[0]
    u = np.zeros(n)
    v = np.zeros(n)
    p = np.zeros(n)
    m = np.full(n, params.rho0 * params.dx * params.dx)
    ids = np.arange(seed_ids, seed_ids + n, dtype=np.uint64)
    return Case(name, params, x, y, u, v, p, m, tag, ids, n + capacity_extra)


def channel(dx: float = 0.02, nu: float = 0.01, seed: int = 0, jitter: float = 0.01,
            pulse_amp: float = 0.1, pulse_xy=(0.5, 0.25), pulse_w: float = 0.005,
            n_in: int = 3, n_out: int = 5, L: float = 1.0, H: float = 0.5,
            U: float = 1.0) -> Case:
    """The 2D pulse channel (periodic in y) with inlet at x=0 and hybrid outlet at x=L."""
    cs = 10.0 * U
    hdx = 1.2
    rc = 3.0 * hdx * dx
    nx, ny = int(round(L / dx)), int(round(H / dx))
    params = Params(x_min=-n_in * dx - rc, x_max=L + n_out * dx + rc, y_min=0.0, y_max=H,
                    periodic_y=1, dx=dx, hdx=hdx, rho0=1.0, U=U, nu=nu, cs=cs,
                    pb=1.0 * cs * cs, dt=default_dt(dx, hdx, cs, U, nu),
                    has_inlet=1, x_in=0.0, n_in_layers=n_in, inlet_y0=0.0, inlet_h=H,
                    has_outlet=1, x_out=L, n_out_layers=n_out)
    fx, fy = _lattice(0.0, nx, 0.0, ny, dx)
    ix, iy = _lattice(-n_in * dx, n_in, 0.0, ny, dx)
    ox, oy = _lattice(L, n_out, 0.0, ny, dx)
    rng = np.random.default_rng(seed)
    fx = fx + rng.uniform(-jitter * dx, jitter * dx, fx.shape)
    fy = fy + rng.uniform(-jitter * dx, jitter * dx, fy.shape)
    # the jitter may push a bottom-row particle below y=0: wrap into the periodic box
    fy = np.where(fy < 0.0, fy + H, np.where(fy >= H, fy - H, fy))
    c = _assemble("channel", params, [(fx, fy, FLUID), (ix, iy, INLET), (ox, oy, OUTLET)],
                  capacity_extra=4 * ny + 64)
    c.u[:] = U
    c.p[:] = pulse_amp * np.exp(-((c.x - pulse_xy[0]) ** 2 + (c.y - pulse_xy[1]) ** 2) / pulse_w)
    return c


def outlet_problem(problem: str = "pulse2d", outlet: int = 0, long: bool = False,
                   dx: float = 0.1, t_end: float = 3.0, probe_d: float = 1.7,
                   delta: float = 1e-3) -> Case:
    """The outlet test problems of Sec. 4: a channel of length 2 and width 2 (4 for the
    vortex) between inviscid (slip) walls, inviscid fluid, U = 1, c = 10 U, six layers of
    inlet, outlet and wall particles, spacing 0.1, the probe at d = 1.7 on the centre line.
    The long-domain reference has length d + c t_end, so that nothing the outlet reflects
    reaches the probe before t_end.
      pulse2d (Sec. 4.2): fluid at u = U; the inlet adds A cos(pi y / 12) exp(-(t-1)^2/delta)
        for 1 < t < 1.1, A = 0.5 (delta is not given; 1e-3 is the reading);
      ramp (Sec. 4.3): fluid at rest; the inlet ramps from 0 to U over 1 s;
      vortex (Sec. 4.4): fluid at u = U; the inlet carries a vortex of strength 0.1 and core
        0.2 whose centre starts 1 upstream of the inlet and moves at U.
    The characteristic outlet's reference is (1 m/s, 1 Pa) at rho = 1000 (Sec. 4.1), i.e.
    (U, 0.001) at rho0 = 1."""
    U, cs, n_lay = 1.0, 10.0, 6
    W = 4.0 if problem == "vortex" else 2.0
    L = probe_d + cs * t_end if long else 2.0
    hdx = 1.2
    rc = 3.0 * hdx * dx
    nx, ny = int(round(L / dx)), int(round(W / dx))
    if problem == "pulse2d":
        kind, prm, u0 = 1, (0.5, 1.0, 1.1, delta), U
    elif problem == "ramp":
        kind, prm, u0 = 2, (1.0,), 0.0
    elif problem == "vortex":
        kind, prm, u0 = 3, (0.1, 0.2, 1.0, 0.5 * W), U
    else:
        raise ValueError(f"unknown problem {problem!r}")
    params = Params(x_min=-n_lay * dx - rc, x_max=L + n_lay * dx + rc,
                    y_min=-n_lay * dx - rc, y_max=W + n_lay * dx + rc, periodic_y=0,
                    dx=dx, hdx=hdx, rho0=1.0, U=U, nu=0.0, cs=cs, pb=cs * cs,
                    dt=default_dt(dx, hdx, cs, U, 0.0),
                    has_inlet=1, x_in=0.0, n_in_layers=n_lay, inlet_y0=0.0, inlet_h=W,
                    inlet_kind=kind, inlet_prm=prm,
                    has_outlet=1, x_out=L, n_out_layers=n_lay, outlet_kind=int(outlet),
                    moc_ref=(1.0, 1e-3), wall_slip=(0, 1), wall_drag=(0, 0))
    fx, fy = _lattice(0.0, nx, 0.0, ny, dx)
    ix, iy = _lattice(-n_lay * dx, n_lay, 0.0, ny, dx)
    ox, oy = _lattice(L, n_lay, 0.0, ny, dx)
    nxw = 2 * n_lay + nx
    bx, by = _lattice(-n_lay * dx, nxw, -n_lay * dx, n_lay, dx)
    tx, ty = _lattice(-n_lay * dx, nxw, W, n_lay, dx)
    # headroom for the inflow over t_end: the outlet may not remove as much as enters (a
    # frozen outlet at rest, or a long domain whose outlet the flow does not reach)
    c = _assemble(problem + ("_long" if long else ""), params,
                  [(fx, fy, FLUID), (ix, iy, INLET), (ox, oy, OUTLET),
                   (np.concatenate([bx, tx]), np.concatenate([by, ty]), SLIPWALL)],
                  capacity_extra=int((2.0 * U * t_end / dx + 2) * ny) + 64)
    c.u[:] = np.where(c.tag == SLIPWALL, 0.0, u0)
    c.p[:] = 0.0
    return c


def pressure_bump(outlet: int = 0, long: bool = False, dx: float = 0.005, t_end: float = 0.3,
                  n_rows: int = 12, n_lay: int = 6, av_alpha: float = 0.1) -> Case:
    """The 1D pressure bump of Sec. 4.1 (Eq. pressurebump): a fluid strip of length 1, periodic
    across (n_rows particle rows), moving at U = 1 with the inlet at x = 0 and the outlet at
    x = 1 (six layers each), initial p = 1 - 0.2 exp(-(x - 0.5)^2 / 0.001) Pa in the fluid and
    1 Pa in the inlet and outlet, rho = 1000 kg/m^3; here rho0 = 1 and p in units of 1000 Pa
    (so the characteristic outlet's reference (1 m/s, 1 Pa) is (U, 0.001)).  Readings: c = 10 U;
    the artificial viscosity alpha = 0.1 the paper takes from its source is the kinematic
    viscosity nu = alpha h c / 8 (the viscosity of Monaghan's term, the form of Eq. edac-nu);
    the spacing is not given (dx = 0.005: the bump's width sqrt(0.001) spans ~6 particles).
    The long-domain reference extends the fluid by (c + U) t_end downstream and (c - U) t_end
    upstream, so that neither acoustic wave reaches an end before t_end."""
    U, cs, hdx = 1.0, 10.0, 1.2
    h = hdx * dx
    rc = 3.0 * h
    nu = av_alpha * h * cs / 8.0
    W = n_rows * dx
    x0 = -(cs - U) * t_end if long else 0.0
    x1 = 1.0 + (cs + U) * t_end if long else 1.0
    x0 = dx * math.floor(x0 / dx)
    x1 = dx * math.ceil(x1 / dx)
    nx = int(round((x1 - x0) / dx))
    params = Params(x_min=x0 - n_lay * dx - rc, x_max=x1 + n_lay * dx + rc, y_min=0.0, y_max=W,
                    periodic_y=1, dx=dx, hdx=hdx, rho0=1.0, U=U, nu=nu, cs=cs, pb=cs * cs,
                    dt=default_dt(dx, hdx, cs, U, nu),
                    has_inlet=1, x_in=x0, n_in_layers=n_lay, inlet_y0=0.0, inlet_h=W,
                    has_outlet=1, x_out=x1, n_out_layers=n_lay, outlet_kind=int(outlet),
                    moc_ref=(1.0, 1e-3), wall_drag=(0, 0))
    fx, fy = _lattice(x0, nx, 0.0, n_rows, dx)
    ix, iy = _lattice(x0 - n_lay * dx, n_lay, 0.0, n_rows, dx)
    ox, oy = _lattice(x1, n_lay, 0.0, n_rows, dx)
    c = _assemble("pressure_bump" + ("_long" if long else ""), params,
                  [(fx, fy, FLUID), (ix, iy, INLET), (ox, oy, OUTLET)],
                  capacity_extra=int((2.0 * U * t_end / dx + 4) * n_rows) + 64)
    c.u[:] = U
    c.p[:] = 1e-3
    fl = c.tag == FLUID
    c.p[fl] = 1e-3 * (1.0 - 0.2 * np.exp(-(c.x[fl] - 0.5) ** 2 / 0.001))
    return c


def batch_channels(n: int = 64, seed: int = 0, n_min: int = 2000, n_max: int = 60000,
                   dx_min: float = 0.005, dx_max: float = 0.03, re_min: float = 50.0,
                   re_max: float = 500.0, U: float = 1.0) -> list:
    """Independent pulse channels of uneven size (the batched workload).  Per channel, from
    one seeded generator: a fluid count N ~ U[n_min, n_max], a spacing dx ~ U[dx_min, dx_max],
    Re = U H / nu ~ U[re_min, re_max] and a pulse centre uniform in the channel.  Each channel
    is L x H = L x L/2 with L = dx sqrt(2 N) rounded to whole spacings (so it holds about N
    fluid particles), periodic in y, with the pulse of the channel workload scaled to L
    (amplitude 0.1, exp(-r^2 / (0.005 L^2)))."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.integers(n_min, n_max + 1))
        dx = float(rng.uniform(dx_min, dx_max))
        Re = float(rng.uniform(re_min, re_max))
        nx = max(32, int(round(math.sqrt(2.0 * N))))
        ny = max(16, int(round(0.5 * nx)))
        L, H = nx * dx, ny * dx
        px, py = float(rng.uniform(0.0, L)), float(rng.uniform(0.0, H))
        c = channel(dx=dx, nu=U * H / Re, seed=seed * 1000 + i, L=L, H=H, U=U,
                    pulse_xy=(px, py), pulse_w=0.005 * L * L)
        c.name = f"channel{i}"
        out.append(c)
    return out


def cylinder(dx: float = 1.0 / 40.0, D: float = 1.0, Re: float = 200.0, Lx: float = 15.0,
             H: float = 10.0, xc: float = 5.0, n_solid: int = 3, n_in: int = 3, n_out: int = 5,
             n_wall: int = 4, U: float = 1.0, inlet_modes=()) -> Case:
    """Flow past a cylinder: 15D x 10D channel, slip walls, hybrid outlet (Sec. 4.6)."""
    cs = 10.0 * U
    hdx = 1.2
    rc = 3.0 * hdx * dx
    nu = U * D / Re
    R = 0.5 * D
    yc = 0.5 * H
    nx, ny = int(round(Lx / dx)), int(round(H / dx))
    params = Params(x_min=-n_in * dx - rc, x_max=Lx + n_out * dx + rc,
                    y_min=-n_wall * dx - rc, y_max=H + n_wall * dx + rc,
                    periodic_y=0, dx=dx, hdx=hdx, rho0=1.0, U=U, nu=nu, cs=cs,
                    pb=1.0 * cs * cs, dt=default_dt(dx, hdx, cs, U, nu),
                    has_inlet=1, x_in=0.0, n_in_layers=n_in, inlet_y0=0.0, inlet_h=H,
                    has_outlet=1, x_out=Lx, n_out_layers=n_out,
                    inlet_modes=tuple(inlet_modes), drag_length=D)
    fx, fy = _lattice(0.0, nx, 0.0, ny, dx)
    keep = (fx - xc) ** 2 + (fy - yc) ** 2 >= (R + 0.5 * dx) ** 2
    fx, fy = fx[keep], fy[keep]
    ix, iy = _lattice(-n_in * dx, n_in, 0.0, ny, dx)
    ox, oy = _lattice(Lx, n_out, 0.0, ny, dx)
    # slip walls below and above, spanning inlet + fluid + outlet
    nxw = n_in + nx + n_out
    bx, by = _lattice(-n_in * dx, nxw, -n_wall * dx, n_wall, dx)
    tx, ty = _lattice(-n_in * dx, nxw, H, n_wall, dx)
    # solid rings: first on the circumference, then dx further in each time
    sx, sy = [], []
    for k in range(n_solid):
        r = R - k * dx
        if r <= 0.0:
            break
        npt = max(1, int(round(2.0 * math.pi * r / dx)))
        th = 2.0 * math.pi * np.arange(npt) / npt
        sx.append(xc + r * np.cos(th))
        sy.append(yc + r * np.sin(th))
    sx = np.concatenate(sx)
    sy = np.concatenate(sy)
    c = _assemble("cylinder", params,
                  [(fx, fy, FLUID), (ix, iy, INLET), (ox, oy, OUTLET),
                   (np.concatenate([bx, tx]), np.concatenate([by, ty]), SLIPWALL),
                   (sx, sy, WALL)],
                  capacity_extra=4 * ny + 1024)
    c.u[:] = np.where((c.tag == WALL) | (c.tag == SLIPWALL), 0.0, U)
    if inlet_modes:
        sel = c.tag == INLET
        c.u[sel] = inlet_profile(c.y[sel], U, inlet_modes, 0.0, H)
    return c


def inlet_profile(y, U, modes, y0, H):
    """u(y) = U + sum_k a_k sin(k pi (y - y0)/H): the inlet-profile family of the workload."""
    out = np.full(np.shape(y), U, dtype=np.float64)
    for k, a in enumerate(modes, start=1):
        out = out + a * np.sin(k * math.pi * (np.asarray(y) - y0) / H)
    return out


def taylor_green(n: int = 20, nu: float = 0.01, U: float = 1.0, L: float = 1.0,
                 jitter: float = 0.0, seed: int = 0) -> Case:
    """Doubly periodic box with the Taylor-Green vortex u=-U cos(2pi x) sin(2pi y), ..."""
    dx = L / n
    cs = 10.0 * U
    params = Params(x_min=0.0, x_max=L, y_min=0.0, y_max=L, periodic_x=1, periodic_y=1,
                    dx=dx, hdx=1.2, rho0=1.0, U=U, nu=nu, cs=cs, pb=cs * cs,
                    dt=default_dt(dx, 1.2, cs, U, nu))
    x, y = _lattice(0.0, n, 0.0, n, dx)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        x = np.mod(x + rng.uniform(-jitter * dx, jitter * dx, x.shape), L)
        y = np.mod(y + rng.uniform(-jitter * dx, jitter * dx, y.shape), L)
    c = _assemble("taylor_green", params, [(x, y, FLUID)], capacity_extra=0)
    k = 2.0 * math.pi / L
    c.u[:] = -U * np.cos(k * c.x) * np.sin(k * c.y)
    c.v[:] = U * np.sin(k * c.x) * np.cos(k * c.y)
    c.p[:] = -0.25 * U * U * (np.cos(2 * k * c.x) + np.cos(2 * k * c.y))
    return c


def poiseuille(n: int = 10, nu: float = 0.1, umax: float = 1.0, Lx: float = 0.5,
               n_wall: int = 4) -> Case:
    """x-periodic channel of width 1 between no-slip walls driven by g = 8 nu umax / W^2."""
    W = 1.0
    dx = W / n
    cs = 10.0 * umax
    g = 8.0 * nu * umax / (W * W)
    nx = int(round(Lx / dx))
    rc = 3.6 * dx
    params = Params(x_min=0.0, x_max=Lx, y_min=-n_wall * dx - rc, y_max=W + n_wall * dx + rc,
                    periodic_x=1, dx=dx, hdx=1.2, rho0=1.0, U=umax, nu=nu, cs=cs,
                    pb=cs * cs, gx=g, dt=default_dt(dx, 1.2, cs, umax, nu),
                    wall_slip=(0, 1), wall_drag=(0, 0))
    fx, fy = _lattice(0.0, nx, 0.0, n, dx)
    bx, by = _lattice(0.0, nx, -n_wall * dx, n_wall, dx)
    tx, ty = _lattice(0.0, nx, W, n_wall, dx)
    return _assemble("poiseuille", params,
                     [(fx, fy, FLUID), (np.concatenate([bx, tx]), np.concatenate([by, ty]), WALL)],
                     capacity_extra=0)


def random_box(n: int = 300, seed: int = 0, periodic_y: int = 1, dx: float = 0.05,
               tags=(FLUID, INLET, OUTLET, WALL, SLIPWALL), L: float = 1.0, H: float = 0.6) -> Case:
    """Seeded random particles in [0,L]x[0,H] with random tags and fields (property tests).

    Inlet/outlet particles are placed left of x_in = 0.2 / right of x_out = 0.8 so
    that the zone semantics hold; walls and fluid are placed anywhere in between.
    """
    rng = np.random.default_rng(seed)
    cs = 10.0
    params = Params(x_min=-0.2, x_max=L + 0.2, y_min=0.0, y_max=H, periodic_y=periodic_y,
                    dx=dx, hdx=1.2, rho0=1.0, U=1.0, nu=0.01, cs=cs, pb=cs * cs,
                    dt=default_dt(dx, 1.2, cs, 1.0, 0.01),
                    has_inlet=int(INLET in tags), x_in=0.2, n_in_layers=3, inlet_y0=0.0, inlet_h=H,
                    has_outlet=int(OUTLET in tags), x_out=0.8, n_out_layers=3)
    tag = rng.choice(np.array(tags, dtype=np.uint8), size=n)
    x = rng.uniform(0.0, L, n)
    x = np.where(tag == INLET, rng.uniform(0.2 - 3 * dx, 0.2, n), x)
    x = np.where(tag == OUTLET, rng.uniform(0.8, 0.8 + 3 * dx, n), x)
    x = np.where(tag == FLUID, rng.uniform(0.2, 0.8, n), x)
    y = rng.uniform(0.0, H, n)
    c = Case("random_box", params, x, y, rng.normal(1.0, 0.1, n), rng.normal(0.0, 0.1, n),
             rng.normal(0.0, 0.2, n), rng.uniform(0.8, 1.2, n) * dx * dx, tag,
             np.arange(n, dtype=np.uint64), capacity=2 * n + 64)
    return c


def by_name(name: str, **kw) -> Case:
    """Named workloads: channel, cyl40 (dx=D/40), cyl100 (D/100), cyl25 (D/25)."""
    if name == "channel":
        return channel(**kw)
    if name == "cyl40":
        return cylinder(dx=1.0 / 40.0, **kw)
    if name == "cyl100":
        return cylinder(dx=1.0 / 100.0, **kw)
    if name == "cyl25":
        return cylinder(dx=1.0 / 25.0, **kw)
    raise ValueError(f"unknown workload {name!r}")
