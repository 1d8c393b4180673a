"""Gradients of losses of the step history with respect to the inlet-profile modes.

The inlet profile is u(y) = U + sum_k a_k sin(k pi (y - y0) / H), k = 1..8.  Losses:
  mean drag:        L = mean_n F_x^n / (rho0 U^2 D / 2) over a window of steps;
  pressure energy:  L = mean_n sum_fluid omega(x) p^2 at the end of each step with the
                    window weight omega = sin^2(pi (x - x0) / (x1 - x0)) on [x0, x1): the
                    energy of the pressure waves in a layer (the one in front of the outlet
                    holds what the outlet reflects); the weight vanishes smoothly at both
                    edges, so particles entering or leaving the layer change L continuously.
Two derivatives of the fp64 step, with neighbour sets and recycling events held fixed:
  reverse mode (edac_adjoint_run): the adjoint of every operation of the step, taken
    backwards with checkpoint-every-K recompute; its cost does not grow with the number
    of parameters (``drag_gradient_adjoint``, ``pressure_energy_gradient``);
  forward mode (edac_step_tangent): the tangent-linear model, 8 directions carried next to
    the values (``drag_gradient``).
``MeanDrag`` puts the mean drag behind ``torch.autograd.Function`` (the adjoint by default).
``central_differences`` is the check: two fp64 runs per mode at a_k +- eps, with the
recycling event counts of the two runs compared step by step (a run whose events differ is
not the same discrete map).
"""
import dataclasses

import numpy as np

from . import binding

N_MODES = 8


def _with_modes(case, a):
    """A copy of the case whose inlet carries the modes a (the inlet particles' velocities too)."""
    import copy

    c = copy.deepcopy(case)
    c.params = dataclasses.replace(case.params, inlet_modes=tuple(float(v) for v in a))
    from .cases import INLET, inlet_profile

    sel = c.tag == INLET
    c.u[sel] = inlet_profile(c.y[sel], c.params.U, c.params.inlet_modes, c.params.inlet_y0,
                             c.params.inlet_h)
    return c


def _scale(case):
    p = case.params
    return 0.5 * p.rho0 * p.U * p.U * p.drag_length


def drag_loss(case, a, nsteps: int, device: str = "cuda:0"):
    """L(a) and the step histories of an fp64 run (no tangents)."""
    c = _with_modes(case, a)
    s = binding.Solver(c, precision="fp64", use_graphs=True, device=device,
                       max_history=nsteps + 16)
    s.step(nsteps)
    h = s.history(nsteps)
    s.close()
    return float(np.mean(h["fx"])) / _scale(c), h


def drag_gradient(case, a, nsteps: int, device: str = "cuda:0"):
    """(L, dL/da [8], timings): one fp64 run with the tangents of the 8 modes."""
    import time

    import torch

    c = _with_modes(case, a)
    s = binding.Solver(c, precision="fp64", use_graphs=False, device=device,
                       max_history=nsteps + 16)
    s.tangent_enable()
    torch.cuda.synchronize(s.device)
    t0 = time.perf_counter()
    s.step_tangent(nsteps)
    torch.cuda.synchronize(s.device)
    t1 = time.perf_counter()
    h = s.history(nsteps)
    dfx, _ = s.tangent_history(nsteps)
    s.close()
    q = _scale(c)
    return float(np.mean(h["fx"])) / q, dfx.mean(axis=0)[:N_MODES] / q, {"tangent_s": t1 - t0}


def drag_gradient_adjoint(case, a, nsteps: int, checkpoint_every: int = 50,
                          device: str = "cuda:0"):
    """(L, dL/da [8], timings) of the mean drag by the reverse-mode adjoint."""
    import time

    import torch

    c = _with_modes(case, a)
    s = binding.Solver(c, precision="fp64", use_graphs=False, device=device,
                       max_history=nsteps + 16)
    q = _scale(c)
    w = np.full(nsteps, 1.0 / (nsteps * q))
    torch.cuda.synchronize(s.device)
    t0 = time.perf_counter()
    L, g = s.adjoint(nsteps, checkpoint_every, w_fx=w)
    torch.cuda.synchronize(s.device)
    t1 = time.perf_counter()
    s.close()
    return L, g[:N_MODES], {"adjoint_s": t1 - t0}


def pressure_energy_window(case, width: float = None):
    """The layer in front of the outlet, [x_out - width, x_out) (default: 2 support radii)."""
    p = case.params
    if width is None:
        width = 6.0 * p.hdx * p.dx
    return (p.x_out - width, p.x_out)


def window_weight(x, x0: float, x1: float):
    """omega(x) = sin^2(pi (x - x0) / (x1 - x0)) on [x0, x1), 0 elsewhere."""
    x = np.asarray(x, dtype=np.float64)
    inside = (x >= x0) & (x < x1)
    return np.where(inside, np.sin(np.pi * (x - x0) / (x1 - x0)) ** 2, 0.0)


def pressure_energy_loss(case, a, nsteps: int, window=None, device: str = "cuda:0"):
    """L = mean_n sum_fluid omega(x) p^2 of an fp64 run (the state read after every step)."""
    c = _with_modes(case, a)
    x0, x1 = window if window is not None else pressure_energy_window(c)
    s = binding.Solver(c, precision="fp64", use_graphs=True, device=device,
                       max_history=nsteps + 16)
    tot = 0.0
    for _ in range(nsteps):
        s.step(1)
        st = s.state(("x", "p"))
        fl = st["tag"] == 0
        tot += float(np.sum(window_weight(st["x"][fl], x0, x1) * st["p"][fl] ** 2))
    s.close()
    return tot / nsteps


def pressure_energy_gradient(case, a, nsteps: int, window=None, checkpoint_every: int = 50,
                             device: str = "cuda:0"):
    """(L, dL/da [8]) of the windowed pressure energy by the reverse-mode adjoint."""
    c = _with_modes(case, a)
    x0, x1 = window if window is not None else pressure_energy_window(c)
    s = binding.Solver(c, precision="fp64", use_graphs=False, device=device,
                       max_history=nsteps + 16)
    L, g = s.adjoint(nsteps, checkpoint_every, w_pe=np.full(nsteps, 1.0 / nsteps),
                     pe_window=(x0, x1))
    s.close()
    return L, g[:N_MODES]


def central_differences(case, a, nsteps: int, eps: float = 1e-6, modes=None,
                        device: str = "cuda:0"):
    """dL/da_k by central differences of fp64 runs; also whether each pair of runs took the
    same recycling events (n_spawn, n_delete, n_to_outlet per step)."""
    a = np.asarray(a, dtype=np.float64)
    modes = range(N_MODES) if modes is None else modes
    g = np.zeros(N_MODES)
    same = {}
    for k in modes:
        ap, am = a.copy(), a.copy()
        ap[k] += eps
        am[k] -= eps
        lp, hp = drag_loss(case, ap, nsteps, device)
        lm, hm = drag_loss(case, am, nsteps, device)
        g[k] = (lp - lm) / (2.0 * eps)
        same[k] = all(np.array_equal(hp[f], hm[f]) for f in ("n_spawn", "n_delete", "n_to_outlet"))
    return g, same


def _function():
    import torch

    class MeanDrag(torch.autograd.Function):
        """L = mean drag coefficient over `nsteps` steps of `case` with inlet modes a (a torch
        tensor of 8 values); backward returns grad_output * dL/da from the reverse-mode
        adjoint (checkpoints every `checkpoint_every` steps) or, with method="tangent", the
        tangent-linear run."""

        @staticmethod
        def forward(ctx, a, case, nsteps, method, checkpoint_every):
            av = a.detach().cpu().double().numpy()
            dev = str(a.device) if a.is_cuda else "cuda:0"
            if method == "tangent":
                L, g, _ = drag_gradient(case, av, int(nsteps), device=dev)
            else:
                L, g, _ = drag_gradient_adjoint(case, av, int(nsteps), int(checkpoint_every),
                                                device=dev)
            ctx.save_for_backward(torch.as_tensor(g, dtype=a.dtype, device=a.device))
            return torch.as_tensor(L, dtype=a.dtype, device=a.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None, None, None

    return MeanDrag


def mean_drag(a, case, nsteps: int, method: str = "adjoint", checkpoint_every: int = 50):
    """Autograd entry: L(a) with its gradient through the reverse-mode adjoint (or the
    tangent-linear model)."""
    return _function().apply(a, case, nsteps, method, checkpoint_every)
