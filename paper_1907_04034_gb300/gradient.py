"""Gradient of the time-averaged drag with respect to the inlet-profile modes.

The inlet profile is u(y) = U + sum_k a_k sin(k pi (y - y0) / H), k = 1..8; the loss is the
drag coefficient averaged over a window of steps, L = mean_n F_x^n / (rho0 U^2 D / 2).  The
library carries the derivatives of the fp64 step with respect to a_1..a_8 forward next to the
values (edac_step_tangent: the tangent-linear model of the discrete step, neighbour sets and
recycling events held fixed), so dL/da_k = mean_n dF_x^n/da_k / (rho0 U^2 D / 2) comes out of
one run.  ``MeanDrag`` puts that behind ``torch.autograd.Function``.  ``central_differences``
is the check: two fp64 runs per mode at a_k +- eps, with the recycling event counts of the
two runs compared step by step (a run whose events differ is not the same discrete map).
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
        tensor of 8 values); backward returns grad_output * dL/da from the tangent run."""

        @staticmethod
        def forward(ctx, a, case, nsteps):
            av = a.detach().cpu().double().numpy()
            L, g, _ = drag_gradient(case, av, int(nsteps), device=str(a.device) if a.is_cuda
                                    else "cuda:0")
            ctx.save_for_backward(torch.as_tensor(g, dtype=a.dtype, device=a.device))
            return torch.as_tensor(L, dtype=a.dtype, device=a.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None

    return MeanDrag


def mean_drag(a, case, nsteps: int):
    """Autograd entry: L(a) with its gradient through the tangent-linear model."""
    return _function().apply(a, case, nsteps)
