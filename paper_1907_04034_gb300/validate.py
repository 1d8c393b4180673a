"""Long-run physics (Sec. 4): the flow past a cylinder (Sec. 4.6), drag and lift coefficients
and the Strouhal number from the library's force history, for comparison with Table clcd
(Re = 200) and Table hybridconv (Re = 20); and the outlet test problems (2D pulse, ramp,
passing vortex; Secs. 4.2-4.4), L2 errors at a probe against a long domain (Eq. l2norm).

The paper's setup: cylinder of diameter D, channel 15D x 15D with the cylinder 5D behind the
inlet interface, slip walls, uniform inlet velocity U, hybrid outlet, six layers of inlet,
outlet and wall particles, h = 1.2 dx, Re = U D / nu, the cylinder filled with rings of solid
particles spaced dx down to its centre, run to t = 150 s with D = 2 m and U = 1 m/s, i.e. 75
convective times D / U.  Coefficients: c_d = F_x / (rho0 U^2 D / 2), c_l = F_y / (rho0 U^2 D
/ 2) (per unit length, so that they match the literature values the paper compares with),
filtered with a five-point moving average; St = f D / U with f the shedding frequency.

    python -m paper_1907_04034_gb300.validate --dx-over-d 30 --t-end 75

prints one JSON line.  Everything runs on the GPU through the C ABI (`binding.Solver`).
"""
import argparse
import json
import math
import time

import numpy as np

from . import binding, cases


OUTLETS = {"hybrid": 0, "donothing": 1, "mod_donothing": 2, "characteristic": 3, "mirror": 4}


def paper_cylinder(dx_over_d: float = 30.0, Re: float = 200.0, D: float = 1.0,
                   layers: int = 6, outlet: str = "hybrid") -> cases.Case:
    """The Sec. 4.6 geometry at spacing D / dx_over_d (D = 1 instead of 2 m: only D/dx, Re and
    the convective time matter for the coefficients), with one of the outlets of Sec. 3."""
    dx = D / dx_over_d
    c = cases.cylinder(dx=dx, D=D, Re=Re, Lx=15.0 * D, H=15.0 * D, xc=5.0 * D,
                       n_solid=int(0.5 * D / dx) + 1, n_in=layers, n_out=layers, n_wall=layers)
    c.params.outlet_kind = OUTLETS[outlet]
    return c


def moving_average(a: np.ndarray, k: int = 5) -> np.ndarray:
    """k-point centred moving average (the ends average the available points)."""
    if len(a) < k:
        return a.copy()
    c = np.convolve(a, np.ones(k), mode="same")
    n = np.convolve(np.ones_like(a), np.ones(k), mode="same")
    return c / n


def coefficients(fx, fy, dt: float, D: float, U: float, rho0: float, t_from: float) -> dict:
    """c_d mean and range, c_l amplitude and St over t >= t_from (forces per step)."""
    q = 0.5 * rho0 * U * U * D
    cd = moving_average(np.asarray(fx) / q)
    cl = moving_average(np.asarray(fy) / q)
    t = (np.arange(len(cd)) + 1) * dt
    sel = t >= t_from
    if sel.sum() < 16:
        raise ValueError("averaging window too short")
    cdw, clw, tw = cd[sel], cl[sel], t[sel]
    # shedding frequency: peak of the lift spectrum (Hann window, zero-padded x8)
    x = (clw - clw.mean()) * np.hanning(len(clw))
    nfft = 8 * len(x)
    spec = np.abs(np.fft.rfft(x, nfft))
    freq = np.fft.rfftfreq(nfft, dt)
    lo = np.searchsorted(freq, 0.02 * U / D)  # ignore the slow drift
    f = float(freq[lo + int(np.argmax(spec[lo:]))])
    # lift amplitude: least-squares sinusoid at f (robust to the SPH force noise)
    A = np.stack([np.sin(2 * math.pi * f * tw), np.cos(2 * math.pi * f * tw), np.ones_like(tw)], 1)
    coef, *_ = np.linalg.lstsq(A, clw, rcond=None)
    # smoothed extremes over one-twentieth of a shedding period
    w = max(5, int(round(1.0 / (20.0 * max(f, 1e-9) * dt))))
    cls = moving_average(clw, w)
    return {"cd_mean": float(cdw.mean()), "cd_std": float(cdw.std()),
            "cl_amp_fit": float(math.hypot(coef[0], coef[1])),
            "cl_amp_smoothed": float(0.5 * (cls.max() - cls.min())),
            "cl_mean": float(clw.mean()), "St": f * D / U, "window": [float(tw[0]), float(tw[-1])]}


def run(dx_over_d: float = 30.0, Re: float = 200.0, t_end: float = 75.0, t_from: float = None,
        precision: str = "mixed", chunk: int = 5000, device: str = "cuda:0",
        diagnose: bool = False, outlet: str = "hybrid", drag_reading: int = 2) -> dict:
    """drag_reading: 1 the solid force over fluid neighbours with the interpolated pressure,
    2 Eq. tvf-momentum_solid as printed (every neighbour, p~_ij with the solid's p_avg)."""
    import torch

    case = paper_cylinder(dx_over_d, Re, outlet=outlet)
    case.params.wall_drag = (drag_reading, 0)
    p = case.params
    D, U = p.drag_length, p.U
    nsteps = int(math.ceil(t_end * U / D / p.dt)) if D > 0 else 0
    solver = binding.Solver(case, precision=precision, use_graphs=True, device=device,
                            max_history=nsteps + 16)
    torch.cuda.synchronize(torch.device(device))
    out = {"case": f"cylinder Re={Re:g}, 15D x 15D, dx=D/{dx_over_d:g}", "outlet": outlet,
           "precision": precision, "drag_reading": drag_reading,
           "particles": case.n, "fluid": int(np.sum(case.tag == cases.FLUID)), "dt": p.dt}
    t0 = time.perf_counter()
    done = 0
    last = None
    trace = []  # [step, max |u - U e_x| of fluid, its x, y, min p, max p]
    try:
        while done < nsteps:
            k = min(chunk, nsteps - done)
            solver.step(k)
            done += k
            if diagnose:  # per chunk: the fastest fluid particle and the field ranges per tag
                st = solver.state(("x", "y", "u", "v", "p"))
                last = {int(t): {f: [float(st[f][st["tag"] == t].min()), float(st[f][st["tag"] == t].max())]
                                 for f in ("x", "y", "u", "v", "p")}
                        for t in np.unique(st["tag"])}
                last["step"] = done
                fl = st["tag"] == cases.FLUID
                sp = np.hypot(st["u"][fl] - U, st["v"][fl])
                k = int(np.argmax(sp))
                trace.append([done, float(sp[k]), float(st["x"][fl][k]), float(st["y"][fl][k]),
                              float(st["p"][fl].min()), float(st["p"][fl].max())])
    except binding.EdacError as e:
        out.update({"error": str(e), "failed_in_chunk_after_step": done, "last_good": last,
                    "trace": trace})
        solver.close()
        return out
    h = solver.history(nsteps)
    t1 = time.perf_counter()
    n_final = solver.count()
    solver.close()
    if t_from is None:
        t_from = 0.6 * t_end
    out.update({"particles_final": n_final, "steps": nsteps, "t_end": nsteps * p.dt,
                "wall_s": t1 - t0})
    if diagnose:
        out["trace"] = trace
    out.update(coefficients(h["fx"], h["fy"], p.dt, D, U, p.rho0, t_from))
    return out


# --------------------------------------------------------- outlet test problems (Sec. 4)
def l2_error(f, f_long) -> float:
    """Eq. l2norm: (sum_n (f^n - f_l^n)^2 / sum_n (f_l^n)^2)^(1/2) over the time steps."""
    f, f_long = np.asarray(f), np.asarray(f_long)
    return float(np.sqrt(np.sum((f - f_long) ** 2) / np.sum(f_long ** 2)))


def probe_history(case, t_end: float, probe_d: float = 1.7, precision: str = "mixed",
                  device: str = "cuda:0") -> np.ndarray:
    """Step the case to t_end; after every step the probe (p, u, v) at (d, W/2)."""
    p = case.params
    n = int(round(t_end / p.dt))
    s = binding.Solver(case, precision=precision, use_graphs=True, device=device,
                       max_history=n + 16)
    qx, qy = np.array([probe_d]), np.array([0.5 * p.inlet_h])
    out = np.zeros((n, 3))
    for k in range(n):
        s.step(1)
        out[k] = s.probe(qx, qy)[0, :3]
    s.close()
    return out


def outlet_problem_errors(problem: str, t_end: float = None, precision: str = "mixed",
                          outlets=("characteristic", "donothing", "hybrid", "mirror",
                                   "mod_donothing")) -> dict:
    """e(p*), e(u*) (and e(v*)) at the probe for each outlet, against the long domain, with
    p* = 2 p / (rho u_ref^2), u* = u / u_ref, v* = v / u_ref and u_ref = U (Sec. 4.2)."""
    if t_end is None:
        t_end = 4.0 if problem == "vortex" else 3.0
    ref_case = cases.outlet_problem(problem, outlet=OUTLETS["hybrid"], long=True, t_end=t_end)
    rho0, U = ref_case.params.rho0, ref_case.params.U
    scale = np.array([2.0 / (rho0 * U * U), 1.0 / U, 1.0 / U])
    ref = probe_history(ref_case, t_end, precision=precision) * scale
    out = {"problem": problem, "t_end": t_end, "precision": precision, "errors": {}}
    for name in outlets:
        c = cases.outlet_problem(problem, outlet=OUTLETS[name], t_end=t_end)
        try:
            h = probe_history(c, t_end, precision=precision) * scale
        except binding.EdacError as e:
            out["errors"][name] = {"error": str(e)}
            continue
        e = {"p": l2_error(h[:, 0], ref[:, 0]), "u": l2_error(h[:, 1], ref[:, 1])}
        if problem == "vortex":
            e["v"] = l2_error(h[:, 2], ref[:, 2])
        out["errors"][name] = e
    return out


def bump_profiles(case, times, precision: str = "mixed", device: str = "cuda:0") -> np.ndarray:
    """The pressure of the 1D bump (Sec. 4.1) along x in [0, 1] at each of the times: the mean
    over the fluid particles in each of the bins [k dx, (k + 1) dx) (all rows of the strip),
    array (len(times), nbins); an empty bin holds NaN."""
    p = case.params
    dx = p.dx
    nb = int(round(1.0 / dx))
    steps = [int(round(t / p.dt)) for t in times]
    s = binding.Solver(case, precision=precision, use_graphs=True, device=device,
                       max_history=max(steps) + 16)
    out = np.full((len(times), nb), np.nan)
    done = 0
    for i, n in enumerate(steps):
        s.step(n - done)
        done = n
        st = s.state(("x", "p"))
        fl = (st["tag"] == cases.FLUID) & (st["x"] >= 0.0) & (st["x"] < 1.0)
        b = np.minimum((st["x"][fl] / dx).astype(np.int64), nb - 1)
        cnt = np.bincount(b, minlength=nb)
        tot = np.bincount(b, weights=st["p"][fl], minlength=nb)
        out[i] = np.where(cnt > 0, tot / np.maximum(cnt, 1), np.nan)
    s.close()
    return out


def pressure_bump_errors(times=(0.05, 0.1, 0.15, 0.2, 0.25, 0.3), precision: str = "mixed",
                         outlets=("characteristic", "donothing", "hybrid", "mirror",
                                  "mod_donothing")) -> dict:
    """The 1D pressure bump (Sec. 4.1) with each outlet against the long domain: per outlet the
    L2 error of the pressure profile over x in [0, 1], relative to the bump's depth
    (0.2 Pa), at each time and over all, and the mean pressure excess over the long domain's
    at the last time, over the domain and over its last tenth (same relative unit)."""
    t_end = max(times)
    depth = 0.2e-3
    ref = bump_profiles(cases.pressure_bump(outlet=OUTLETS["hybrid"], long=True, t_end=t_end),
                        times, precision)
    out = {"times": list(times), "precision": precision, "errors": {}}
    for name in outlets:
        c = cases.pressure_bump(outlet=OUTLETS[name], t_end=t_end)
        try:
            h = bump_profiles(c, times, precision)
        except binding.EdacError as e:
            out["errors"][name] = {"error": str(e)}
            continue
        per_t = np.sqrt(np.nanmean((h - ref) ** 2, axis=1)) / depth
        end = h.shape[1] - h.shape[1] // 10  # the last tenth, x in [0.9, 1)
        out["errors"][name] = {"per_time": [float(v) for v in per_t],
                               "all": float(np.sqrt(np.nanmean((h - ref) ** 2)) / depth),
                               "mean_excess_last": float((np.nanmean(h[-1]) - np.nanmean(ref[-1])) / depth),
                               "end_excess_last": float(np.nanmean(h[-1, end:] - ref[-1, end:]) / depth)}
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--dx-over-d", type=float, default=30.0)
    ap.add_argument("--re", type=float, default=200.0)
    ap.add_argument("--t-end", type=float, default=75.0, help="in convective times D/U")
    ap.add_argument("--t-from", type=float, default=None, help="start of the averaging window")
    ap.add_argument("--precision", default="mixed", choices=("mixed", "fp64"))
    ap.add_argument("--chunk", type=int, default=5000, help="steps per edac_step call")
    ap.add_argument("--diagnose", action="store_true",
                    help="record the per-tag field ranges after every chunk")
    ap.add_argument("--outlet", default="hybrid", choices=tuple(OUTLETS))
    ap.add_argument("--drag-reading", type=int, default=2, choices=(1, 2),
                    help="1: solid force over fluid neighbours with the interpolated pressure; "
                         "2: Eq. tvf-momentum_solid as printed (every neighbour, with p_avg)")
    ap.add_argument("--problem", default=None, choices=("pulse2d", "ramp", "vortex", "bump1d"),
                    help="an outlet test problem of Sec. 4 instead of the cylinder: L2 errors "
                         "at the probe for every outlet against the long domain")
    a = ap.parse_args()
    if a.problem == "bump1d":
        print(json.dumps(pressure_bump_errors(precision=a.precision)))
        return
    if a.problem:
        print(json.dumps(outlet_problem_errors(a.problem, precision=a.precision)))
        return
    print(json.dumps(run(a.dx_over_d, a.re, a.t_end, a.t_from, a.precision, a.chunk,
                         diagnose=a.diagnose, outlet=a.outlet, drag_reading=a.drag_reading)))


if __name__ == "__main__":
    main()
