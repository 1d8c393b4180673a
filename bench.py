#!/usr/bin/env python
"""Benchmark: EDAC particle-steps/s on the 1.5M-particle cylinder (Re = 200, dx = D/100).

One step = the whole per-step particle pass (two cell builds, two evaluations of pass A,
the boundary kernel and pass B, two integrator stages, the hybrid-outlet update,
recycling, the drag reduction) on device-resident state.  The headline value is the
mixed-precision path (fp32 pair sums on cell-relative coordinates, fp64 integration and
reductions); the fp64 path and the drag difference between the two are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one rank per GPU) runs N independent replicas of the workload: the path
does not shard (one GPU per system), so value = particle-steps of all ranks / max time.
--impl reference times the CPU oracle (the plain fp64 statement of the method) on the
host cores on the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EDAC particle-steps/s (1.5M cyl), mixed vs FP64 at stated err; adjoint/fwd time"
UNIT = "particle-steps/s"
WORKLOAD = "cylinder Re=200, 15D x 10D channel, dx=D/100 (~1.5M particles), hybrid outlet"

# Algorithmic flops per neighbour pair of the two pair passes, counted from the paper's
# formulas (each add, subtract, multiply, divide or square root is one flop; the branch
# terms of the quintic spline are averaged over the pair distribution of the support).
FLOPS_PER_PAIR_A = 20
FLOPS_PER_PAIR_B = 90


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the pair kernels,
# measured with ncu on the 1.51M-particle workload itself.
TRAFFIC = {"pass_a": 109.4e6, "pass_b": 148.6e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--dx", type=float, default=0.01)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--batch-channels", type=int, default=64,
                    help="uneven channels of the batched measurement (0: skip it)")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--tangent-steps", type=int, default=400,
                    help="steps of the gradient workload (0: skip it)")
    ap.add_argument("--force-steps", type=int, default=2000,
                    help="steps over which the mixed path's drag and lift are compared with "
                         "the fp64 path's")
    ap.add_argument("--developed-steps", type=int, default=400,
                    help="steps timed after --force-steps steps (a flow past its start)")
    return ap.parse_args()


# ------------------------------------------------------------------------------ ranks
def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("BENCH_BACKEND", "nccl")
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local, dist


def reduce_max_sum(dist, t, n, device=None):
    """(max over ranks of t, sum over ranks of n); identity without a process group."""
    if dist is None:
        return float(t), float(n)
    import torch
    a = torch.tensor([float(t)], dtype=torch.float64, device=device)
    b = torch.tensor([float(n)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ peaks
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count, max_mhz):
    """FP32 FMA pipe: 128 lanes per SM, 2 flops per FMA, at the maximum SM clock."""
    return sm_count * 128 * 2 * max_mhz * 1e6 / 1e12


# ------------------------------------------------------------------------------ batched
def run_batched(n_chan, steps, dev):
    """The batched workload: uneven pulse channels (seeded sizes, spacings, Re and pulse
    centres), mixed path, all advanced by one graph launch per step, in the two forms of the
    library: graph branches (each member's own kernels, tiling picked per member by the
    autotuner) and fused (each kernel launched once over all members; the members' common
    tiling picked by timing a few).  Also timed: the members stepped one after the other."""
    import torch
    from paper_1907_04034_gb300 import binding, cases

    chans = cases.batch_channels(n=n_chan, seed=0)
    hist = 3 * steps + 400
    sol = [binding.Solver(c, precision="mixed", use_graphs=True, device=str(dev),
                          max_history=hist) for c in chans]
    done = 0

    def timed(b, k):
        nonlocal done
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.step(k)
        e1.record(b.stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        ps = sum(float(np.sum(s.history(done + k)["n_active"][done:done + k])) for s in sol)
        done += k
        return ms, ps

    def warm(b, k):
        nonlocal done
        b.step(k)
        torch.cuda.synchronize(dev)
        done += k

    out = {}
    # graph branches, per-member autotuned tilings
    tilings = [s.autotune(trials=2)[:2] for s in sol]
    b = binding.Batch(sol)
    warm(b, 5)
    ms, ps = timed(b, steps)
    kps = b.kernels_per_step()
    b.close()
    from collections import Counter
    out["branches"] = {"value": ps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                       "steps": steps, "kernels_per_graph_launch": kps,
                       "tilings": {f"{tx}x{tpb}": k for (tx, tpb), k in Counter(tilings).items()}}
    # fused: one common tiling, the fastest of a few over 20 steps each
    best = None
    trial = {}
    for tx, tpb in ((8, 128), (11, 160), (6, 128), (16, 256)):
        for s in sol:
            s.set_tiling(tx, tpb)
        b = binding.Batch(sol, fused=True)
        warm(b, 2)
        tms, _ = timed(b, 20)
        b.close()
        trial[f"{tx}x{tpb}"] = tms / 20
        if best is None or tms < best[0]:
            best = (tms, tx, tpb)
    for s in sol:
        s.set_tiling(best[1], best[2])
    b = binding.Batch(sol, fused=True)
    warm(b, 5)
    ms, ps = timed(b, steps)
    kps = b.kernels_per_step()
    b.close()
    out["fused"] = {"value": ps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                    "steps": steps, "kernels_per_graph_launch": kps,
                    "tiling": f"{best[1]}x{best[2]}", "tiling_trials_ms_per_step": trial}
    # the same members one after the other (each its own graph, one host thread)
    seq_steps = max(1, steps // 10)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for s in sol:
        s.step(seq_steps)
    torch.cuda.synchronize(dev)
    seq = time.perf_counter() - t0
    seq_ps = sum(float(np.sum(s.history(done + seq_steps)["n_active"][done:done + seq_steps]))
                 for s in sol)
    for s in sol:
        s.close()
    sizes = [c.n for c in chans]
    form = max(("branches", "fused"), key=lambda k: out[k]["value"])
    res = dict(out[form])
    res.update({"form": form, "channels": n_chan, "particles": int(sum(sizes)),
                "particles_min_max": [int(min(sizes)), int(max(sizes))],
                "branches": out["branches"], "fused": out["fused"],
                "members_one_after_another": {"value": seq_ps / seq, "unit": UNIT,
                                              "steps": seq_steps,
                                              "note": "host wall clock, each member its own graph"},
                "workload": "uneven pulse channels: N ~ U[2k, 60k], dx ~ U[0.005, 0.03], "
                            "Re ~ U[50, 500], pulse centre uniform (seed 0); mixed path"})
    return res


# ------------------------------------------------------------------------------ gradient
def run_tangent(steps, dev, checkpoint_every=50):
    """The gradient workload: cylinder at dx = D/25, inlet modes a_k ~ N(0, 0.02) (seed 0),
    mean drag over `steps` steps; the gradient with respect to the 8 modes by the reverse-mode
    adjoint (checkpoints every `checkpoint_every` steps, each segment recomputed once) and by
    the tangent-linear model, their times against the fp64 forward run of the same steps, and
    one central difference (mode 1, eps = 1e-8, see the tests) as a check."""
    import torch
    from paper_1907_04034_gb300 import binding, cases, gradient

    c = cases.cylinder(dx=1.0 / 25.0)
    a = np.random.default_rng(0).normal(0.0, 0.02, 8)
    # forward: fp64 steps on graphs, timed with events
    cc = gradient._with_modes(c, a)
    s = binding.Solver(cc, precision="fp64", use_graphs=True, device=str(dev),
                       max_history=steps + 16)
    s.step(2)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    torch.cuda.synchronize(dev)
    fwd_ms = e0.elapsed_time(e1)
    s.close()
    La, ga, ta = gradient.drag_gradient_adjoint(c, a, steps, checkpoint_every, device=str(dev))
    L, g, tm = gradient.drag_gradient(c, a, steps, device=str(dev))
    gf, same = gradient.central_differences(c, a, steps, eps=1e-8, modes=[0], device=str(dev))
    fwd_s = fwd_ms / 1e3
    return {"workload": f"cylinder Re=200, dx=D/25 ({c.n} particles), 8 inlet modes "
                        f"a_k ~ N(0, 0.02) seed 0, mean c_d over {steps} steps",
            "method": "reverse-mode adjoint of the fp64 step (checkpoints every "
                      f"{checkpoint_every} steps, segments recomputed once; fp32 pair-pass "
                      "adjoints, fp64 boundary adjoints), beside the tangent-linear model "
                      "(forward mode, 8 directions)",
            "loss": La, "dL_da": [float(v) for v in ga],
            "adjoint_s": ta["adjoint_s"], "tangent_s": tm["tangent_s"], "forward_s": fwd_s,
            "adjoint_over_forward": ta["adjoint_s"] / fwd_s,
            "tangent_over_forward": tm["tangent_s"] / fwd_s,
            "adjoint_vs_tangent_max_rel": float(np.abs(ga - g).max() / np.abs(g).max()),
            "fd_check_mode1": {"fd": float(gf[0]), "adjoint": float(ga[0]),
                               "rel_diff": float(abs(ga[0] - gf[0]) / max(abs(gf[0]), 1e-300)),
                               "eps": 1e-8, "same_events": bool(same[0])}}


# -------------------------------------------------------------------------- reference
def cpu_oracle_rate(case, steps):
    """The oracle as it stands (binned neighbour mode, OpenMP on all host cores); also its
    force history over those steps."""
    import oracle
    t0 = time.perf_counter()
    sim = oracle.OracleSim(case, neighbor_mode=1)
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = sim.step(steps)
    dt = time.perf_counter() - t0
    ps = float(sum(h["n_active"] for h in hist))
    fx = np.array([h["fx"] for h in hist])
    fy = np.array([h["fy"] for h in hist])
    return ps / dt, dt, t_init, fx, fy


def run_reference(args, rank, world, dist):
    from paper_1907_04034_gb300 import cases
    if rank != 0:
        return
    case = cases.cylinder(dx=args.dx)
    k = max(1, min(args.steps, args.cpu_steps))
    w = min(args.warmup, 3)  # an oracle step of the workload takes ~0.5 s on 16 cores
    import oracle
    sim = oracle.OracleSim(case, neighbor_mode=1)
    if w:
        sim.step(w)
    t0 = time.perf_counter()
    hist = sim.step(k)
    el = time.perf_counter() - t0
    ps = float(sum(h["n_active"] for h in hist))
    val = ps / el
    cores = os.cpu_count()
    sample = (f"{k} full oracle steps of the workload ({case.n} particles) after {w} warm-up "
              f"step(s); oracle in its binned-neighbour mode, fp64, OpenMP")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": k, "warmup": w, "ms_per_step": el / k * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": case.n, "dx": args.dx},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------------------- ours
def main():
    args = parse()
    rank, world, local, dist = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world, dist)
        if dist is not None:
            dist.destroy_process_group()
        return

    import torch
    from paper_1907_04034_gb300 import binding, cases

    binding.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    case = cases.cylinder(dx=args.dx)
    K, W = args.steps, args.warmup
    F = max(args.force_steps, 0)
    hist_cap = max(4096, K + W + 200 + F + args.developed_steps)

    # ---------------------------------------------------------------- mixed (headline)
    sm = binding.Solver(case, precision="mixed", use_graphs=True, device=str(dev),
                        max_history=hist_cap)
    stream = sm.stream
    sm.step(W)
    torch.cuda.synchronize(dev)
    l0 = sm.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier(dist, dev if dist else None)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        sm.step(K)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(dist, dev if dist else None)
    ms = ev0.elapsed_time(ev1)
    launches = sm.launch_count() - l0
    h = sm.history(K)
    ps_local = float(np.sum(h["n_active"]))
    t_max, ps_all = reduce_max_sum(dist, ms / 1e3, ps_local, dev if dist else None)
    value = ps_all / t_max

    # --------------------------------------------- roofline of the dominant kernel (pass B)
    nb = sm.state(("nnb",))
    # pass B's pairs exclude the particle itself (its terms vanish and are not computed)
    pair_b = int(np.sum(nb["nnb"][(nb["tag"] == cases.FLUID) | (nb["tag"] == cases.INLET)] - 1))
    pair_a = int(np.sum(nb["nnb"]))
    kp = min(K, 100)
    for kname in ("pass_b", "pass_a", "rebuild", "boundary", "stage", "recycle"):
        sm.profile(kname, True)
    sm.step(kp)
    prof = {}
    for kname in ("pass_b", "pass_a", "rebuild", "boundary", "stage", "recycle"):
        t, n = sm.read_profile(kname)
        prof[kname] = {"ms_total": t, "launches": n, "ms_per_launch": t / max(n, 1)}
        sm.profile(kname, False)
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_src = load_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_nominal = fp32_peak_tflops(props.multi_processor_count, max_mhz)
    # measured FMA-pipe peaks (FMA chains filling every SM), the roofline denominators
    peak = binding.fma_peak(binding.EDAC_PEAK_FP32, str(dev))
    peak64 = binding.fma_peak(binding.EDAC_PEAK_FP64, str(dev))
    step_ms_eager = sum(p["ms_total"] for p in prof.values()) / kp
    # the roofline of the dominant (largest total time) of the two arithmetic kernels
    cand = {"pass_b": (pair_b, FLOPS_PER_PAIR_B), "pass_a": (pair_a, FLOPS_PER_PAIR_A)}
    dom = max(cand, key=lambda k: prof[k]["ms_total"])
    pairs, fpp = cand[dom]
    k_ms = prof[dom]["ms_per_launch"]
    achieved = pairs * fpp / (k_ms * 1e-3) / 1e12 if k_ms > 0 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": TRAFFIC.get(dom),
                "kernel": dom + " (mixed)",
                "peak_note": "of measured: fp32 FMA pipe, FMA chains on every SM (edac_fma_peak); "
                             f"nominal {props.multi_processor_count} SMs x 128 lanes x 2 x "
                             f"{max_mhz:.0f} MHz = {peak_nominal:.1f}",
                "pairs_per_launch": pairs, "flops_per_pair": fpp, "ms_per_launch": k_ms}
    kernels = {k: round(v["ms_per_launch"], 5) for k, v in prof.items()}
    for k, (pp, f) in cand.items():
        kernels[k + "_tflops"] = pp * f / (prof[k]["ms_per_launch"] * 1e-3) / 1e12
    # the same run past its start: to F steps, then Kd steps timed (graph replay, events)
    developed = None
    done = W + K + kp
    Kd = args.developed_steps
    if Kd > 0:
        if F > done:
            sm.step(F - done)
            done = F
        torch.cuda.synchronize(dev)
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        sm.step(Kd)
        d1.record(stream)
        torch.cuda.synchronize(dev)
        dms = d0.elapsed_time(d1)
        hd = sm.history(Kd)
        nbd = sm.state(("nnb",))
        developed = {"value": float(np.sum(hd["n_active"])) / (dms * 1e-3) * world, "unit": UNIT,
                     "ms_per_step": dms / Kd, "steps_timed": Kd, "steps_before": done,
                     "mean_neighbours": float(np.mean(nbd["nnb"])),
                     "mean_neighbours_at_headline": float(np.mean(nb["nnb"])),
                     "note": "the headline's run continued past the impulsive start (t = "
                             f"{done * case.params.dt:.3f} D/U), same graph, CUDA events"}
        done += Kd
    fx_mixed = sm.history(done)["fx"]
    fy_mixed = sm.history(done)["fy"]
    sm.close()
    del sm
    torch.cuda.empty_cache()

    # ----------------------------------------------------------------- fp64 path + drag
    K64 = max(1, min(args.fp64_steps, K))
    s64 = binding.Solver(case, precision="fp64", use_graphs=True, device=str(dev),
                         max_history=hist_cap)
    s64.step(W)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s64.stream)
    s64.step(K64)
    e1.record(s64.stream)
    torch.cuda.synchronize(dev)
    ms64 = e0.elapsed_time(e1)
    h64 = s64.history(K64)
    v64 = float(np.sum(h64["n_active"])) / (ms64 / 1e3) * world
    if F > W + K64:
        s64.step(F - W - K64)
    h64all = s64.history(max(F, W + K64))
    fx64, fy64 = h64all["fx"], h64all["fy"]
    # fp64 pair passes against the measured fp64 FMA peak
    kp64 = 2
    for kname in ("pass_b", "pass_a"):
        s64.profile(kname, True)
    s64.step(kp64)
    roof64 = {}
    for kname, (pp, f) in (("pass_b", (pair_b, FLOPS_PER_PAIR_B)), ("pass_a", (pair_a, FLOPS_PER_PAIR_A))):
        t, n = s64.read_profile(kname)
        s64.profile(kname, False)
        kms = t / max(n, 1)
        ach = pp * f / (kms * 1e-3) / 1e12 if kms > 0 else None
        roof64[kname] = {"ms_per_launch": kms, "achieved_tflops": ach,
                         "frac": ach / peak64 if ach and peak64 else None}
    nc = min(len(fx64), len(fx_mixed))
    scale = max(float(np.abs(fx64[:nc]).max()), 1e-12)
    drag_err = float(np.abs(fx_mixed[:nc] - fx64[:nc]).max()) / scale
    forces = {"steps": nc,
              "drag_max_rel": drag_err,
              "lift_max_rel_to_drag": float(np.abs(fy_mixed[:nc] - fy64[:nc]).max()) / scale,
              "mean_drag_rel": float(abs(fx_mixed[:nc].mean() - fx64[:nc].mean())
                                     / max(abs(fx64[:nc].mean()), 1e-300)),
              "fp64_lift_max": float(np.abs(fy64[:nc]).max()),
              "note": "mixed vs fp64 GPU path, per step from the impulsive start; the lift is "
                      "round-off this early (symmetric flow), so it is scaled by the drag"}
    s64.close()
    del s64
    torch.cuda.empty_cache()

    # -------------------------------------------------------------- end to end (C ABI)
    e2e = None
    K2 = min(K, 200)
    se = binding.Solver(case, precision="mixed", use_graphs=True, device=str(dev),
                        max_history=hist_cap)
    se.step(2)  # graph capture outside the timed region
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    se.upload(case)
    se.step(K2)
    he = se.history(K2)
    st = se.state(("x", "y", "u", "v", "p"))
    t1 = time.perf_counter()
    ps_e = float(np.sum(he["n_active"]))
    h2d = case.n * (6 * 8 + 1 + 8)
    d2h = int(st["x"].size) * (5 * 8 + 1 + 8) + K2 * (3 * 8 + 4 * 4)
    e2e = {"value": ps_e / (t1 - t0) * world, "unit": UNIT,
           "h2d_bytes_per_step": h2d / K2, "d2h_bytes_per_step": d2h / K2,
           "steps": K2, "note": "upload from host arrays + K steps + history and field read-back"}
    se.close()
    del se

    # ------------------------------------------- batched uneven channels (one graph launch)
    batched = None
    if args.batch_channels > 0:
        batched = run_batched(args.batch_channels, args.batch_steps, dev)

    # ------------------------------------ gradient workload: tangent-linear model vs forward
    tangent = None
    if args.tangent_steps > 0:
        tangent = run_tangent(args.tangent_steps, dev)

    # ---------------------------------------------------------------------- CPU baseline
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, el, t_init, fxo, fyo = cpu_oracle_rate(case, args.cpu_steps)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{args.cpu_steps} full oracle steps of the workload ({case.n} particles), "
                         f"binned-neighbour mode, fp64, OpenMP, {el:.1f} s"}
        no = min(len(fxo), len(fx_mixed), len(fx64))
        if no:
            so = max(float(np.abs(fxo[:no]).max()), 1e-300)
            forces["vs_oracle"] = {
                "steps": no,
                "mixed_drag_max_rel": float(np.abs(fx_mixed[:no] - fxo[:no]).max()) / so,
                "mixed_lift_max_rel_to_drag": float(np.abs(fy_mixed[:no] - fyo[:no]).max()) / so,
                "fp64_drag_max_rel": float(np.abs(fx64[:no] - fxo[:no]).max()) / so,
                "fp64_lift_max_rel_to_drag": float(np.abs(fy64[:no] - fyo[:no]).max()) / so}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": t_max * 1e3 / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "particles": case.n, "dx": args.dx,
                           "precision": "mixed (fp32 pair sums, fp64 integration/reductions)",
                           "parallelism": f"replicas x{world}",
                           "l2": "no flush: the per-step state (~0.7 GB) is larger than L2"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(),
                "fp64_path": {"value": v64, "unit": UNIT, "steps": K64,
                              "ms_per_step": ms64 / K64, "fp64_peak_tflops": peak64,
                              "pair_kernels": roof64},
                "mixed_over_fp64": value / v64 if v64 else None,
                "drag_rel_err_mixed_vs_fp64": drag_err, "drag_steps_compared": nc,
                "forces_mixed_vs_fp64": forces, "developed": developed,
                "batched": batched,
                "gradient": tangent,
                "kernel_ms_per_launch": kernels, "eager_step_ms": step_ms_eager}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
