"""Benchmark: cell-direction update rate and time to converge of GSIS against
plain source iteration on one GB300, with the roofline of the dominant kernel.

Headline workload: the time-dependent gray radiation-material problem
(Sec. 2.1, Eqs. (RTE_g), (Tm_g); backward Euler, Sec. 4.1), 1024 x 1024
cells on the unit square, S16 (144 directions), a thin bent channel
(sigma_t 0.2, 32 cells wide) in a thick medium (sigma_t 2000), scattering
ratio 0.999, unit isotropic intensity through the left wall, vacuum
elsewhere, a = c = C_v = 1, cold start T = 0.1, 100 backward-Euler steps of
dt = 1e-3; GSIS with FP64 sweeps, moments and synthetic solve, every step
iterated to Err(rho) < 1e-8.

One step of this benchmark = one complete gsis_td_solve call (all 100 time
steps: every kinetic sweep with its moments, adaptive least-squares
gradients, high-order terms, the rho-T synthetic solve, the material update)
from the initial state, inputs resident in HBM.  value = (inner iterations x
cells x directions) / time, summed over steps and ranks.  The two FP64
intensity arrays of a time step (1.2 GB each) exceed L2, and L2 is also
flushed (512 MiB write) before every run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm) on bounded
samples of the same workload on the host cores.  Under torchrun every rank
runs an independent replica (no collective in the data path); rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "cell-direction updates/s and time-to-converge (GSIS vs SI) on 1 GB300; HBM roofline %"
UNIT = "cell-direction updates/s"
TOL = 1e-8
BETA = 10.0        # local pseudo-time control (Sec. 4.3) the steady 2000/0.2 opacity jump needs
SYNTH_CAP = 2      # inner iterations of the synthetic solve per GSIS iteration, steady channel (Sec. 4.2)
TD_SYNTH_CAP = 6   # the cap on the time-dependent workload, with the quadratic predictor (measured: 4 -> 776, 5 -> 598, 6 -> 560, 7 -> 549, 8 -> 547 GSIS iterations; 1.84, 1.78, 1.79, 1.84 s at 5-8)
TD_CHECK_EVERY = 5   # status read every 5 iterations (measured, 100-step run: 3 -> 1.752, 4 -> 1.760, 5 -> 1.749, 6 -> 1.753, 8 -> 1.760 s)
# first iterate of every time step: quadratic extrapolation in time of the last
# three steps' (rho, T) (gsis_time_params::predictor; 0 would start from the
# previous step, as the paper's loop does)
TD_PREDICTOR = 2
FP32_STALL = (2, 5)   # check_every, stall_window: an FP32 step ends after 10 iterations without a new minimum


# ----------------------------------------------------------------- helpers
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_totals(dist, units, ms, device):
    """Whole-job totals of independent replicas: the units every rank
    processed (sum) and the slowest rank's timed milliseconds (max); with no
    process group, the local values."""
    if dist is None:
        return float(units), float(ms)
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


CLOCK_FIELDS = ("uuid,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def _clock_sampler():
    """nvidia-smi clocks/throttle sampling during the timed region."""
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                 "-lms", "20"], stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        return None, f
    # nvidia-smi takes a moment to start: begin the timed region only once it
    # is sampling (at most 3 s), so that the samples cover it
    t0 = time.time()
    while time.time() - t0 < 3.0 and proc.poll() is None:
        if os.path.getsize(f.name) > 0:
            break
        time.sleep(0.01)
    return proc, f


def device_uuid(torch, dev) -> str | None:
    """The CUDA device's UUID as nvidia-smi prints it (without the GPU- prefix),
    or None: nvidia-smi numbers GPUs physically, while CUDA_VISIBLE_DEVICES
    renumbers them for the process, so the clock samples are matched by UUID."""
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:   # noqa: BLE001
        return None
    return u[4:] if u.startswith("GPU-") else u


def parse_clock_samples(lines, uuid=None, index=None):
    """Median SM clock, max clock and active throttle reasons of the samples
    of one GPU (matched by UUID, else by nvidia-smi index)."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        u = parts[0][4:] if parts[0].startswith("GPU-") else parts[0]
        if uuid is not None:
            if u != uuid:
                continue
        elif index is not None and parts[1] != str(index):
            continue
        try:
            sm.append(float(parts[2]))
            smax = float(parts[3])
        except ValueError:
            continue
        for n, v in zip(names, parts[6:10]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm),
            "matched_by": "uuid" if uuid is not None else "index"}


def _clock_summary(proc, f, uuid, index):
    if proc is None:
        f.close()
        os.unlink(f.name)
        return None
    proc.terminate()
    try:
        proc.wait(5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.flush()
    f.seek(0)
    lines = f.read().splitlines()
    os.unlink(f.name)
    return parse_clock_samples(lines, uuid=uuid, index=None if uuid else index)


# DRAM bytes per launch from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum, one capture each, summarised in profiles/), valid
# while the sources that define the sweep launch (kernel, arguments, grid,
# workspace layout) are the captured ones.
SWEEP_SOURCES = ("sweep.cu", "gsis_internal.cuh", "host.h", "api.cu", "timedep.cu", "batch.cu")
SWEEP_TRAFFIC = {   # {workload: (sources digest, bytes per launch)}
    "timedep_fp64": ("a03f3ba1fdf55726", 3_812_679_040),   # profiles/sweep_kernel_wide_td1024_fp64.md
    "channel": ("a03f3ba1fdf55726", 106_284_800),          # profiles/sweep_kernel_channel256.md
    "batch": ("a03f3ba1fdf55726", 932_232_448),            # profiles/sweep_kernel_batch64.md
}


def sweep_sources_digest() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2507_03975_gb300", "csrc")
    for name in SWEEP_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def _sweep_traffic(workload):
    """ncu DRAM bytes of one sweep launch of `workload`, or None once the
    sweep-launch sources differ from the captured ones."""
    ent = SWEEP_TRAFFIC.get(workload)
    if ent is None or ent[0] != sweep_sources_digest():
        return None
    return ent[1]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _events(torch, n=2):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _rel(a, b):
    a = a.double().cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
    b = b.double().cpu().numpy() if hasattr(b, "cpu") else np.asarray(b)
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


# ------------------------------------------------ headline: time-dependent
class TdWorkload:
    """Inputs of the time-dependent workload on the device (and pinned on the
    host for the end-to-end pass)."""

    def __init__(self, torch, dev):
        self.p = p = W.config_timedep()
        self.tp = tp = W.TIMEDEP
        self.host = [np.ascontiguousarray(a, dtype=np.float64) for a in
                     (p.sigma_a, p.sigma_s, p.q, p.inflow.reshape(-1), np.full(p.N, tp["T0"]),
                      np.full(p.N, tp["a"] * tp["c"] * tp["T0"] ** 4))]
        t = lambda a: torch.from_numpy(a).to(dev)
        self.sa, self.ss, self.q, self.inflow, self.T0, self.rho0 = (t(a) for a in self.host)
        self.upd = p.N * p.K

    def run(self, gsis, opt, nsteps=None, workspace=None, stream=None, inputs=None, predictor=TD_PREDICTOR):
        p, tp = self.p, self.tp
        sa, ss, q, inflow, T0, rho0 = inputs or (self.sa, self.ss, self.q, self.inflow, self.T0, self.rho0)
        return gsis.td_solve(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, q, rho0, T0, tp["dt"],
                             nsteps or tp["nsteps"], c=tp["c"], a=tp["a"], cv=tp["cv"], inflow=inflow,
                             options=opt, workspace=workspace, stream=stream, predictor=predictor)


def td_options(gsis, scheme=None, precision=None, tol=TOL, **kw):
    base = dict(scheme=gsis.SCHEME_GSIS if scheme is None else scheme,
                precision=gsis.FP64 if precision is None else precision, tol=tol, max_iter=2000,
                check_every=TD_CHECK_EVERY, synth_rtol=1e-12, synth_max_iter=TD_SYNTH_CAP)
    base.update(kw)
    return gsis.default_options(**base)


def _td_config(p, tp):
    return dict(workload="channel_td_1024x1024_S16", nx=p.nx, ny=p.ny, K=p.K, nsteps=tp["nsteps"], dt=tp["dt"],
                scheme="gsis", precision="fp64", tol=TOL, tol_applies_to="Err(rho) of every time step",
                synthetic=f"rho-T system with T eliminated (Newton about T^m); FP64 iterative refinement, FP32 "
                          f"multigrid-CG inner iterations capped at {TD_SYNTH_CAP} per GSIS iteration",
                predictor="each step starts from the quadratic extrapolation in time of the last three steps' "
                          "(rho, T) (linear at step 1, the previous step at step 0); every step still iterates "
                          "to the tolerance" if TD_PREDICTOR == 2 else f"order {TD_PREDICTOR}",
                l2="inputs larger than L2 (two FP64 K x N intensity arrays of 1.2 GB per time step); L2 also "
                   "flushed (512 MiB write) before every run",
                step="one complete 100-time-step gsis_td_solve call from the cold start",
                kernel_timing="a separate instrumented run with CUDA events around every kernel class on the "
                              "launching stream (roofline, shares); value and ms_per_step from uninstrumented runs")


def td_class_model(cls, prof, iters, upd, N, fp64_peak, hbm, fp64=True):
    """Roofline entry of one kernel class of the time-dependent run, per
    working launch (one launch group per inner iteration; launches after a
    step converged inside a check_every batch return at once, their few
    microseconds stay in the total, so this slightly overstates the time).
    Algorithmic work (what the method must do, not what this implementation
    adds):
      sweep:   the upwind update I = (X + a I_W + b I_S) / d over the
               time step's source X = S + I^n/(c dt): 2 FMA + 1 MUL per
               update (5 FLOP; the FMA that forms X is the update class's;
               FP64 binds: 5 FLOP at 1.25 TFLOP/s take 3x longer than the
               HBM bytes at peak); bytes: read I^n once per update (8 B
               FP64, 4 B FP32) plus 64 B per cell (sigma_t, source in, six
               moments out);
      moments: rho, F_x, F_y: over x-reflection pairs of one weight, 2 adds
               + 3 FMA per two updates (4 FLOP per update; an add takes a
               full FMA slot of the FP64 pipe, so the fraction is a lower
               bound);
      synth:   36 B per cell from HBM per call (level coefficients, r0,
               guess, x) -- bound by barriers and latency;
      hot_rhs / update: 15 / 10 doubles per cell."""
    g = max(int(iters), 1)
    avg_ms = prof[cls]["total_ms"] / g
    ib = 8.0 if fp64 else 4.0
    hbm_bytes = None
    if cls == "sweep":
        work, bound, peak, unit = 5.0 * upd, ("alu" if fp64 else "hbm"), (fp64_peak if fp64 else hbm), \
            ("GFLOP/s" if fp64 else "GB/s")
        hbm_bytes = ib * upd + 64.0 * N
        if not fp64:
            work = hbm_bytes
    elif cls == "moments":
        work, bound, peak, unit = 4.0 * upd, ("alu" if fp64 else "hbm"), (fp64_peak if fp64 else hbm), \
            ("GFLOP/s" if fp64 else "GB/s")
        if not fp64:
            work = ib * upd + 48.0 * N
    elif cls == "synth":
        work, bound, peak, unit = 36.0 * N, "latency", hbm, "GB/s"
    elif cls == "hot_rhs":
        work, bound, peak, unit = 15 * 8.0 * N, "hbm", hbm, "GB/s"
    else:
        work, bound, peak, unit = 10 * 8.0 * N, "hbm", hbm, "GB/s"
    ach = work / (avg_ms * 1e-3) / 1e9
    out = {"bound": bound, "kernel": cls, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
           "avg_launch_ms": avg_ms, "launch_groups": g, "launches_timed": prof[cls]["timed"],
           "algorithmic_work_per_launch": work}
    if hbm_bytes is not None:
        gbs = hbm_bytes / (avg_ms * 1e-3) / 1e9
        out["hbm_view"] = {"algorithmic_bytes": hbm_bytes, "achieved_gbs": gbs, "peak_gbs": hbm,
                           "frac": gbs / hbm}
    return out


def td_fp32_measure(gsis, torch, stream, wl, ref64, ws=None):
    """The same 100 steps with FP32 sweeps (FP64 moments accumulate FP32
    intensities; synthetic solve, material update and Err in FP64), each step
    to Err < 1e-8 or to its floor (no new minimum of Err for 10 iterations),
    and the error of the result against the FP64 run."""
    ce, sw = FP32_STALL
    opt = td_options(gsis, precision=gsis.FP32_SWEEP, check_every=ce, stall_window=sw)
    wl.run(gsis, opt, workspace=ws, stream=stream)   # warm-up (workspace)
    e0, e1 = _events(torch)
    e0.record(stream)
    r = wl.run(gsis, opt, stream=stream)
    e1.record(stream)
    e1.synchronize()
    s = e0.elapsed_time(e1) * 1e-3
    its, err = r["step_iters"], r["step_err"]
    return {"precision": "fp32 sweeps and moment accumulation (fp32 intensities and accumulators), fp64 HoT / "
                              "synthetic solve / material update / Err",
            "tol": TOL, "stall": f"a step ends after {ce * sw} iterations without a new minimum of Err",
            "s": s, "status": r["status"], "iters_total": int(its.sum()),
            "iters_per_step_mean": float(its.mean()), "updates_per_s": float(its.sum()) * wl.upd / s,
            "steps_reaching_tol": int((err < TOL).sum()), "steps_at_floor": int((err >= TOL).sum()),
            "step_err_median": float(np.median(err)), "step_err_max": float(err.max()),
            "rel_err_vs_fp64": {"rho": _rel(r["rho"], ref64["rho"]), "T": _rel(r["T"], ref64["T"])}}


def td_adjoint_measure(gsis, torch, stream, wl, nsteps=None):
    """Gradient of J = sum of rho^N over the channel cells of the first 64
    columns (a detector next to the source wall) after the full run, with
    respect to sigma_a, sigma_s, rho^0 and T^0, by gsis_td_adjoint: FP64,
    forward steps and adjoint iterations to Err < 1e-8, checkpoints every
    ceil(sqrt(steps)) steps.  Device time with CUDA events around the forward
    run alone and around the whole adjoint call (forward run with
    checkpoints, one recomputation, the step adjoints), inputs resident; a
    second, instrumented call gives the kernel classes."""
    p, tp = wl.p, wl.tp
    n = nsteps or tp["nsteps"]
    cols = np.arange(p.N) % p.nx
    g = torch.from_numpy((((p.sigma_a + p.sigma_s) < 1.0) & (cols < 64)).astype(np.float64)).to(wl.sa.device)
    opt = td_options(gsis)
    e0, e1 = _events(torch)

    def timed(fn):
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) * 1e-3

    # the forward run the adjoint differentiates (and recomputes from its checkpoints)
    f, s_fwd = timed(lambda: wl.run(gsis, opt, nsteps=n, stream=stream))
    adj = lambda ws=None: gsis.td_adjoint(p.dx, p.dy, p.mu, p.eta, p.w, wl.sa, wl.ss, wl.q, wl.rho0, wl.T0,
                                          tp["dt"], n, dJ_drho=g, c=tp["c"], a=tp["a"], cv=tp["cv"],
                                          inflow=wl.inflow, options=opt, workspace=ws, stream=stream,
                                          predictor=TD_PREDICTOR)
    r, s_adj = timed(adj)
    gsis.profile_enable(True)
    r2, _ = timed(lambda: adj(r["workspace"]))
    prof = gsis.profile_read()
    gsis.profile_enable(False)
    out = {"workload": f"channel_td_1024x1024_S16, {n} steps of dt = 1e-3, J = sum of rho^N over the channel "
                       "cells of the first 64 columns",
           "nsteps": n, "precision": "fp64", "tol": TOL, "checkpoint_every": r["checkpoint_every"],
           "status": r["status"], "forward_s": s_fwd, "forward_iters": int(f["step_iters"].sum()),
           "adjoint_call_s": s_adj, "adjoint_over_forward": s_adj / s_fwd,
           "adj_iters_per_step_mean": float(np.mean(r["adj_iters"])),
           "workspace_gb": r["workspace"].numel() / 1e9,
           "kernel_ms": {k: v["total_ms"] for k, v in prof.items()},
           "repeat_bit_equal": bool(torch.equal(r["grad_sigma_a"], r2["grad_sigma_a"])),
           "grad_sigma_a_max": float(r["grad_sigma_a"].abs().max())}
    del r, r2
    return out


# ----------------------------------------- the steady 256^2 channel (extra)
def channel_measure(gsis, torch, stream, flush, fp64_peak, steps=5, warmup=2, no_si=False, no_uw2=False):
    """The steady multiscale workload: 256 x 256 cells, S12 (84 directions),
    channel sigma_t 0.2 (8 cells wide) in a medium of sigma_t 2000, ratio
    0.999, unit isotropic intensity through the left wall.  GSIS (FP64,
    local pseudo-time beta = 10, synthetic solve capped at SYNTH_CAP inner
    iterations) to Err < 1e-8 against SI to Err < 1e-8, the difference of the
    two converged results, the sweep's ALU roofline, and the second-order
    upwind form.  L2 flushed before every solve; device time with CUDA
    events, inputs resident."""
    p = W.config_channel()
    dev = flush.device
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    sa, ss, q, inflow = t(p.sigma_a), t(p.sigma_s), t(p.q), t(p.inflow.reshape(-1))
    opt = gsis.default_options(scheme=gsis.SCHEME_GSIS, precision=gsis.FP64, tol=TOL, beta=BETA, max_iter=5000,
                               check_every=16, synth_max_iter=SYNTH_CAP)
    ws = torch.empty(gsis.workspace_bytes(p.dx, p.dy, p.mu, p.eta, p.w, opt), dtype=torch.uint8, device=dev)
    solve = lambda o=opt, w=ws: gsis.solve(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, q, inflow, o, workspace=w,
                                           want_P=False)
    for _ in range(warmup):
        solve()
    ms, r = [], None
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = _events(torch)
        e0.record(stream)
        r = solve()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    gsis.profile_enable(True)
    flush.fill_(1.0)
    ri = solve()
    prof = gsis.profile_read()
    gsis.profile_enable(False)
    upd = p.N * p.K
    sweep_ms = prof["sweep"]["total_ms"] / max(1, ri["iters"])
    ach = 5.0 * upd / (sweep_ms * 1e-3) / 1e9
    out = {"workload": "channel_256x256_S12_seed2 (steady), GSIS FP64, beta = 10, Err < 1e-8",
           "gsis": {"s": statistics.median(ms) * 1e-3, "iters": r["iters"], "status": r["status"],
                    "synth_inner_iters": r["synth_inner_iters"],
                    "updates_per_s": r["iters"] * upd / (statistics.median(ms) * 1e-3)},
           "sweep_roofline": {"bound": "alu", "kernel": "sweep (fp64, pseudo-time, per-ordinate source)",
                              "achieved": ach, "peak": fp64_peak, "unit": "GFLOP/s", "frac": ach / fp64_peak,
                              "avg_launch_ms": sweep_ms, "traffic": _sweep_traffic("channel")},
           "kernel_ms_per_iter": {k: v["total_ms"] / max(1, ri["iters"]) for k, v in prof.items() if k != "setup"}}
    if not no_si:
        opt_si = gsis.default_options(scheme=gsis.SCHEME_SI, precision=gsis.FP64, tol=TOL, max_iter=100000,
                                      check_every=256)
        flush.fill_(3.0)
        e0, e1 = _events(torch)
        e0.record(stream)
        rs = gsis.solve(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, q, inflow, opt_si, want_P=False)
        e1.record(stream)
        e1.synchronize()
        s = e0.elapsed_time(e1) * 1e-3
        out["si"] = {"s": s, "iters": rs["iters"], "status": rs["status"], "updates_per_s": rs["iters"] * upd / s}
        out["gsis_over_si_time"] = out["gsis"]["s"] / s
        # the two schemes converge to different discrete solutions (GSIS
        # corrects UW1 towards the diffusion limit)
        out["rel_diff_rho_gsis_vs_si"] = _rel(r["rho"], rs["rho"])
    if not no_uw2:
        out["uw2"] = uw2_measure(gsis, torch, stream, p, sa, ss, q, inflow, flush)
    return out


# ------------------------------------------------ the other workloads
def small_measure(gsis, torch, stream):
    """Time to Err < 1e-8 of FP64 GSIS and SI on the 64x64 S8 uniform problem
    (sigma_t = 10, ratio 0.99, q = 1, vacuum): the latency-bound size, where
    a sweep is 164K updates.  Device time with CUDA events, inputs resident,
    best of three after one warm-up solve."""
    p = W.config_small()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    sa, ss, q = t(p.sigma_a), t(p.sigma_s), t(p.q)
    out = {"workload": "uniform_64x64_S8 (sigma_t 10, ratio 0.99, q 1, vacuum), FP64, Err < 1e-8"}
    # GSIS with the synthetic system solved to its default tolerance each
    # iteration, and with the multigrid-CG capped at SYNTH_CAP inner
    # iterations (warm-started; the same fixed point), as in the channel solve
    for name, scheme, cap in (("gsis", gsis.SCHEME_GSIS, 0), ("gsis_synth_cap", gsis.SCHEME_GSIS, SYNTH_CAP),
                              ("si", gsis.SCHEME_SI, 0)):
        kw = {"synth_max_iter": cap} if cap else {}
        opt = gsis.default_options(scheme=scheme, precision=gsis.FP64, tol=TOL, max_iter=100000,
                                   check_every=16 if scheme == gsis.SCHEME_GSIS else 64, **kw)
        best, r = None, None
        for i in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = gsis.solve(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, q, None, opt, want_P=False)
            e1.record(stream)
            e1.synchronize()
            if i and (best is None or e0.elapsed_time(e1) < best):
                best = e0.elapsed_time(e1)
        out[name] = {"ms": best, "iters": r["iters"], "status": r["status"],
                     "updates_per_s": r["iters"] * p.N * p.K / (best * 1e-3)}
    return out


def adjoint_measure(gsis, torch, stream):
    """Forward solve and adjoint gradient of J = sum of rho over 16 seed-3
    detector cells on the 64x64 S8 workload (sigma_t = 10, ratio 0.99, q = 1,
    vacuum), FP32 sweeps with the FP64 synthetic solve (and the FP64 form for
    reference); device time with CUDA events, inputs resident."""
    p = W.config_small()
    rng = np.random.Generator(np.random.PCG64(3))
    g = np.zeros(p.N)
    g[rng.choice(p.N, 16, replace=False)] = 1.0
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    sa, ss, q, gd = t(p.sigma_a), t(p.sigma_s), t(p.q), t(g)
    out = {"workload": "uniform_64x64_S8, J = sum of rho over 16 detector cells (seed 3)"}
    for name, prec, tol in (("fp32_sweeps", gsis.FP32_SWEEP, 1e-6), ("fp64", gsis.FP64, 1e-8)):
        opt = gsis.default_options(precision=prec, tol=tol, stall_window=4, max_iter=2000)
        ws = None
        for _ in range(3):   # two warm-up rounds, the last one timed
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            r = gsis.solve(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, q, None, opt, want_P=False)
            e1.record(stream)
            a = gsis.adjoint(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, q, r["rho"], gd, options=opt, workspace=ws)
            ws = a["workspace"]
            e2.record(stream)
            e2.synchronize()
        out[name] = {"forward_ms": e0.elapsed_time(e1), "adjoint_ms": e1.elapsed_time(e2),
                     "forward_iters": r["iters"], "adjoint_iters": a["iters"], "adjoint_err": a["err"],
                     "tol": tol}
    return out


def batch_measure(gsis, torch, stream, hbm, steps=3):
    """The 64-problem batch (seed 4: sides 32-256 log-uniform, S8-S16,
    sigma_t log-uniform in [1e-2, 1e4] on smooth random fields, one ratio in
    [0.5, 0.9999] per problem, q = 1, vacuum), one gsis_solve_batch call per
    step: FP32 sweeps, FP64 synthetic solve capped at SYNTH_CAP inner
    iterations, local pseudo-time beta = 10, Err < 1e-6 per problem.  The
    autotuner runs first (untimed); device time with CUDA events, inputs
    resident, the first solve untimed."""
    ps = W.config_batch()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    probs = [dict(dx=p.dx, dy=p.dy, mu=p.mu, eta=p.eta, w=p.w, sigma_a=t(p.sigma_a), sigma_s=t(p.sigma_s),
                  q=t(p.q), inflow=None) for p in ps]
    opt = gsis.default_options(precision=gsis.FP32_SWEEP, tol=1e-6, beta=10.0, synth_rtol=1e-12,
                               synth_max_iter=SYNTH_CAP, stall_window=8, check_every=8, max_iter=5000)
    at = gsis.batch_autotune(probs, opt, trial_iters=3)
    ws = at["workspace"]
    times = []
    for i in range(1 + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = gsis.solve_batch(probs, opt, workspace=ws)
        e1.record(stream)
        e1.synchronize()
        if i:
            times.append(e0.elapsed_time(e1))
    iters = [x["iters"] for x in r["results"]]
    per_sweep = sum(p.N * p.K for p in ps)
    updates = sum(it * p.N * p.K for it, p in zip(iters, ps))
    ms = statistics.median(times)
    sweep_ms = at["class_ms"]["sweep"]
    # algorithmic bytes of one batched FP32 pseudo-time sweep over its per-ordinate
    # source X = src + shift I^m: read X and write I (4 + 4 B per update), the
    # diagonal sigma_t + shift (FP32) once per cell
    algo = 8.0 * per_sweep + 4.0 * sum(p.N for p in ps)
    ach = algo / (sweep_ms * 1e-3) / 1e9
    return {"workload": "batch_64_seed4 (sides 32-256, S8-S16, sigma_t 1e-2..1e4, ratio 0.5..0.9999)",
            "problems": len(ps), "updates_per_batch_sweep": per_sweep, "precision": "fp32 sweeps, fp64 synthetic",
            "tol": 1e-6, "beta": 10.0, "synth_cap": SYNTH_CAP,
            "tuning": at["tuning"].as_dict(), "tuned_ms_per_iter": at["ms_per_iter"],
            "class_ms_per_iter": at["class_ms"],
            "solve_ms": ms, "solve_ms_all": times, "iters_max": max(iters), "iters_mean": float(np.mean(iters)),
            "status_ok": sum(1 for x in r["results"] if x["status"] == 0),
            "updates_per_s": updates / (ms * 1e-3),
            "sweep_updates_per_s": per_sweep / (sweep_ms * 1e-3),
            "sweep_roofline": {"bound": "hbm", "kernel": "batched sweep", "achieved": ach, "peak": hbm,
                               "unit": "GB/s", "frac": ach / hbm, "traffic": _sweep_traffic("batch"),
                               "algorithmic_bytes": algo}}


def uw2_measure(gsis, torch, stream, p, sa, ss, q, inflow, flush):
    """The channel workload with second-order upwind face values (the paper's
    transport scheme): GSIS, FP64, beta = 10, Err < 1e-8, synthetic solve
    capped at SYNTH_CAP inner iterations; Barth-Jespersen limiter and
    unlimited reconstruction, and the limiter at the paper's own stopping
    criterion Err < 1e-6 (below ~3e-8 its switching puts the iteration into
    a limit cycle, which the stall window ends).  Device time with CUDA
    events (L2 flushed before each solve), a second, instrumented solve for
    the class times."""
    out = {"workload": "channel_256x256_S12_seed2, UW2", "tol": TOL}
    for name, lim, tol in (("barth_jespersen", 0, TOL), ("unlimited", 1, TOL), ("barth_jespersen_tol1e-6", 0, 1e-6)):
        opt = gsis.default_options(scheme=gsis.SCHEME_GSIS, precision=gsis.FP64, tol=tol, beta=BETA, max_iter=3000,
                                   check_every=16, stall_window=8, synth_rtol=1e-12, synth_max_iter=SYNTH_CAP,
                                   spatial_order=2, limiter=lim)
        res = {}
        for prof in (False, True):
            gsis.profile_enable(prof)
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = gsis.solve(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, q, inflow, opt, want_P=False)
            e1.record(stream)
            e1.synchronize()
            if not prof:
                s = e0.elapsed_time(e1) * 1e-3
                res = {"s": s, "tol": tol, "iters": r["iters"], "status": r["status"], "err": r["err"],
                       "updates_per_s": r["iters"] * p.N * p.K / s}
            else:
                pr = gsis.profile_read()
                res["kernel_ms_per_iter"] = {k: v["total_ms"] / max(1, r["iters"]) for k, v in pr.items()
                                             if k != "setup"}
        gsis.profile_enable(False)
        out[name] = res
    return out


# ------------------------------------------------------- the oracle on CPU
def _td_oracle_inputs():
    from oracle import timedep as TD
    p = W.config_timedep()
    td = W.TIMEDEP
    tp = TD.TimeParams(dt=td["dt"], c=td["c"], a=td["a"], cv=td["cv"])
    T0 = np.full(p.N, td["T0"])
    rho0 = td["a"] * td["c"] * T0 ** 4
    return TD, p, tp, rho0, T0


def cpu_baseline_sample(threads=False):
    """The FP64 oracle as it stands on a bounded sample of the headline
    workload: one GSIS iteration of its first time step from the cold start
    (the kinetic step over all 144 ordinates and 1,048,576 cells, the
    adaptive gradients, the synthetic operator and its sparse LU solve, the
    material update).  threads: the -fopenmp build of the oracle's C sweeps
    (ordinates on all host cores, the same results) instead of one thread.
    Returns (updates/s, seconds, threads used)."""
    from oracle import gsis as G
    TD, p, tp, rho0, T0 = _td_oracle_inputs()
    I0 = TD.isotropic(p, rho0)
    G.use_threads(threads)
    try:
        cores = G.threads()
        t0 = time.perf_counter()
        TD.gsis_time_step(p, tp, rho0, T0, I0, fixed_iters=1)
        dt = time.perf_counter() - t0
    finally:
        G.use_threads(False)
    return p.N * p.K / dt, dt, cores


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on the headline
    workload.  One of its GSIS iterations takes ~20 s (its sparse LU of the
    1,048,576-cell synthetic system alone ~15 s), so each step is a bounded
    sample: the oracle's kinetic step of the first time step (the UW1 sweep
    of all 144 ordinates with the shift 1/(c dt) and I^n, moments and
    boundary fluxes; C sweeps on every host core).  The synthetic solve is
    outside the sample, so this rate bounds the oracle's whole-iteration rate
    from above; one whole iteration is timed once after the steps and
    reported beside it."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import gsis as G
    TD, p, tp, rho0, T0 = _td_oracle_inputs()
    cfg = _td_config(p, W.TIMEDEP)
    I0 = TD.isotropic(p, rho0)
    src = p.sigma_a * TD.emission(T0, tp) + p.q
    G.use_threads(True)
    try:
        cores = G.threads()
        for _ in range(args.warmup):
            TD.kinetic_step(p, tp, rho0, src, I0)
        secs = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            TD.kinetic_step(p, tp, rho0, src, I0)
            secs.append(time.perf_counter() - t0)
        full = None
        if not args.no_cpu_baseline:
            t0 = time.perf_counter()
            TD.gsis_time_step(p, tp, rho0, T0, I0, fixed_iters=1)
            dt = time.perf_counter() - t0
            full = {"value": p.N * p.K / dt, "unit": UNIT, "s": dt, "cores": cores,
                    "sample": "one whole oracle GSIS iteration of the first time step (kinetic step, gradients, "
                              "synthetic operator and its sparse LU solve, material update)"}
    finally:
        G.use_threads(False)
    value = args.steps * p.N * p.K / sum(secs)
    sample = ("one oracle kinetic step of the first time step per bench step: UW1 sweep of all 144 ordinates over "
              "the 1,048,576 cells (diagonal shift 1/(c dt), I^n on the right), moments and boundary fluxes, C "
              "sweeps on every host core; the oracle's synthetic solve is outside the sample (an upper bound of "
              "its whole-iteration rate)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "oracle_full_iteration": full,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    from paper_2507_03975_gb300 import gsis

    ws, rank, local = _dist()
    if args.gpus > 1 or ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    if args.batch_only:   # the batched-solve measurement alone (profiling runs)
        print(json.dumps({"batch": batch_measure(gsis, torch, stream, hbm)}))
        return 0
    if args.channel_only:   # the steady channel measurement alone (profiling runs)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)
        print(json.dumps({"channel_256": channel_measure(gsis, torch, stream, flush, gsis.measure_fp64_fma(),
                                                         no_si=True, no_uw2=True)}))
        return 0

    wl = TdWorkload(torch, dev)
    p, tpd = wl.p, wl.tp
    cfg = _td_config(p, tpd)
    opt = td_options(gsis)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)   # 512 MiB > L2
    workspace = torch.empty(gsis.td_workspace_bytes(p.dx, p.dy, p.mu, p.eta, p.w, opt), dtype=torch.uint8,
                            device=dev)
    gsis.profile_enable(False)
    for _ in range(args.warmup):
        wl.run(gsis, opt, workspace=workspace, stream=stream)
    torch.cuda.synchronize()

    # ---- timed: K complete runs, inputs resident in HBM (no instrumentation)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    proc, cf = _clock_sampler() if rank == 0 else (None, None)
    step_ms, iters, res = [], [], None
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = _events(torch)
        e0.record(stream)
        res = wl.run(gsis, opt, workspace=workspace, stream=stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        iters.append(int(res["step_iters"].sum()))
        if res["status"] != gsis.GSIS_OK:
            raise RuntimeError(f"time-dependent run did not converge: status {res['status']}")
    torch.cuda.synchronize()
    clocks = _clock_summary(proc, cf, device_uuid(torch, dev), torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    units, total_ms = replica_totals(dist, sum(iters) * wl.upd, sum(step_ms), dev)
    if dist:
        dist.barrier()
    value = units / (total_ms * 1e-3)
    ref64 = {"rho": res["rho"].clone(), "T": res["T"].clone()}
    step_iters = res["step_iters"]

    # ---- one instrumented run: CUDA events around every kernel class
    gsis.profile_enable(True)
    flush.fill_(1.0)
    ri = wl.run(gsis, opt, workspace=workspace, stream=stream)
    torch.cuda.synchronize()
    prof = gsis.profile_read()
    gsis.profile_enable(False)
    prof_iters = int(ri["step_iters"].sum())
    launches_per_run = int(sum(v["kernels"] for v in prof.values()))

    # ---- end to end through the C ABI: pinned host inputs in, result out
    h_in = [torch.from_numpy(a).pin_memory() for a in wl.host]
    h_rho = torch.empty(p.N, dtype=torch.float64).pin_memory()
    h_T = torch.empty(p.N, dtype=torch.float64).pin_memory()
    e2e_ms, e2e_iters = [], []
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record(stream)
        d_in = [h.to(dev, non_blocking=True) for h in h_in]
        r = wl.run(gsis, opt, workspace=workspace, stream=stream, inputs=d_in)
        h_rho.copy_(r["rho"], non_blocking=True)
        h_T.copy_(r["T"], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        e2e_iters.append(int(r["step_iters"].sum()))
    h2d = sum(h.numel() * 8 for h in h_in)
    d2h = (h_rho.numel() + h_T.numel()) * 8
    e2e_value = None
    if e2e_ms:
        e2e_units, e2e_total = replica_totals(dist, sum(e2e_iters) * wl.upd, sum(e2e_ms), dev)
        e2e_value = e2e_units / (e2e_total * 1e-3)

    # ---- time to converge: Fleck-Cummings source iteration on the same run, once
    si = None
    if not args.no_si:
        opt_si = td_options(gsis, scheme=gsis.SCHEME_SI, max_iter=20000, check_every=16)
        flush.fill_(3.0)
        e0, e1 = _events(torch)
        e0.record(stream)
        rs = wl.run(gsis, opt_si, stream=stream)
        e1.record(stream)
        e1.synchronize()
        s = e0.elapsed_time(e1) * 1e-3
        its = rs["step_iters"]
        si = {"s": s, "status": rs["status"], "iters_total": int(its.sum()),
              "iters_per_step_mean": float(its.mean()), "updates_per_s": float(its.sum()) * wl.upd / s,
              # GSIS and SI converge to different discrete solutions
              "rel_diff_gsis_vs_si": {"rho": _rel(ref64["rho"], rs["rho"]), "T": _rel(ref64["T"], rs["T"])}}
        del rs

    fp32 = None
    if not args.no_fp32:
        fp32 = td_fp32_measure(gsis, torch, stream, wl, ref64)

    td_adj = None
    if not args.no_td_adjoint:
        td_adj = td_adjoint_measure(gsis, torch, stream, wl)
    del workspace
    torch.cuda.empty_cache()

    # ---- roofline of the dominant kernel class (algorithmic work per launch)
    try:
        FP64_PEAK = gsis.measure_fp64_fma()
        fp64_src = "measured in this run: FP64 FMA kernel (gsis_measure_fp64_fma)"
    except Exception as ex:   # noqa: BLE001
        FP64_PEAK = 1250.0
        fp64_src = f"nominal GB300 FP64 rate 1.25 TFLOP/s (measurement failed: {ex})"
    try:
        fp32_rate = gsis.measure_fp32_fma()
    except Exception:   # noqa: BLE001
        fp32_rate = None
    shares = {k: v["total_ms"] for k, v in prof.items()}
    tot = sum(shares.values()) or 1.0
    model = lambda c: td_class_model(c, prof, prof_iters, wl.upd, p.N, FP64_PEAK, hbm)
    dom = max(("sweep", "moments", "synth", "update", "hot_rhs"), key=lambda k: shares[k])
    roof = model(dom)
    roof.update({"traffic": _sweep_traffic("timedep_fp64") if dom == "sweep" else None,
                 "share": {k: v / tot for k, v in shares.items()},
                 "peak_source": ("measured hbm_gbs (MEASURED_PEAKS.json)" if roof["bound"] != "alu"
                                 else fp64_src),
                 "fp64_fma_gflops": FP64_PEAK, "fp32_fma_gflops": fp32_rate,
                 "others": {k: model(k) for k in ("sweep", "moments", "synth", "update", "hot_rhs") if k != dom}})

    # ---- the other workloads, once each
    extra = {}
    if not args.no_channel:
        extra["channel_256"] = channel_measure(gsis, torch, stream, flush, FP64_PEAK, no_si=args.no_si,
                                               no_uw2=args.no_uw2)
    if not args.no_adjoint:
        extra["adjoint"] = adjoint_measure(gsis, torch, stream)
        extra["uniform_64x64_S8"] = small_measure(gsis, torch, stream)
    if not args.no_batch:
        extra["batch"] = batch_measure(gsis, torch, stream, hbm)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline:
        v, dt, cores = cpu_baseline_sample(threads=False)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one oracle GSIS iteration of the first time step of the same workload ({dt:.1f} s: "
                         "kinetic step of 144 ordinates x 1,048,576 cells, adaptive gradients, synthetic "
                         "operator with its sparse LU solve, material update), one thread"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": max(ws, 1), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "time_to_converge": {"gsis": {"s": total_ms / args.steps * 1e-3, "iters_total": iters[0],
                                          "iters_per_step_mean": float(np.mean(step_iters)),
                                          "iters_per_step_max": int(step_iters.max()),
                                          "step_err_max": float(res["step_err"].max())},
                                 "si": si,
                                 "note": "both schemes, 100 backward-Euler steps, Err(rho) < 1e-8 in every step"},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_run * args.steps,
            "gpu_launches_note": "library kernel launches per run (its launch counters) x timed runs",
            "kernel_ms": {k: v["total_ms"] for k, v in prof.items()},
            "fp32_intensities": fp32,
            "td_adjoint": td_adj,
            "clocks": clocks}
    line.update(extra)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_oracle_times(args):
    """The FP64 oracle's own timings on the host cores (CPU only; prints one
    JSON line): time per sweep (64^2 S8 uniform, 256^2 S12 channel); time to
    Err < 1e-8 by SI and GSIS on the 64^2 problem and by GSIS on the channel
    (beta = 10); the headline time-dependent workload for real: its first
    --oracle-td-steps time steps by GSIS to Err < 1e-8 on every core, and one
    GSIS iteration on one core."""
    import platform

    import oracle
    from oracle import gsis as G

    def timed(fn):
        t0 = time.perf_counter()
        r = fn()
        return r, time.perf_counter() - t0

    out = {"impl": "oracle_times", "host": platform.machine(), "nproc": os.cpu_count(), "arms": {}}
    c1, c2 = W.config_small(), W.config_channel()
    for threads in (False, True):
        G.use_threads(threads)
        try:
            arm = {"threads": G.threads()}
            for name, p in (("uniform_64x64_S8", c1), ("channel_256x256_S12", c2)):
                rho = np.zeros(p.N)
                G.transport_sweep(p, rho)
                ts = [timed(lambda: G.transport_sweep(p, rho))[1] for _ in range(3)]
                arm[f"sweep_s_{name}"] = min(ts)
            for name, fn in (("si", oracle.si_solve), ("gsis", oracle.gsis_solve)):
                r, dt = timed(lambda: fn(c1, tol=TOL))
                arm[f"uniform_64x64_S8_{name}"] = {"s": dt, "iters": int(r["iters"])}
            if threads:
                r, dt = timed(lambda: oracle.gsis_solve(c2, tol=TOL, beta=BETA))
                arm["channel_256x256_S12_gsis"] = {"s": dt, "iters": int(r["iters"])}
            out["arms"]["all_cores" if threads else "one_core"] = arm
        finally:
            G.use_threads(False)
    if args.oracle_td_steps > 0:
        TD, p5, tp, rho0, T0 = _td_oracle_inputs()
        v, dt, cores = cpu_baseline_sample(threads=False)
        out["arms"]["one_core"]["channel_td_1024x1024_S16_one_gsis_iteration"] = {"s": dt, "updates_per_s": v}
        G.use_threads(True)
        try:
            n = args.oracle_td_steps
            r, dt = timed(lambda: TD.run(p5, tp, n, rho0, T0, scheme="gsis", tol=TOL))
            out["arms"]["all_cores"][f"channel_td_1024x1024_S16_gsis_{n}_steps"] = {
                "s": dt, "iters": r["iters"].tolist(), "updates_per_s": float(r["iters"].sum()) * p5.N * p5.K / dt,
                "note": f"the first {n} of the 100 time steps, every step to Err < 1e-8 (sparse LU of the "
                        "synthetic system in every iteration)"}
        finally:
            G.use_threads(False)
    print(json.dumps(out))
    return 0


PROFILE_CASES = {
    # name: (mesh side, sweep precision); one backward-Euler step of the
    # time-dependent channel workload from the cold start, two GSIS iterations
    "td1024_fp64": (1024, "fp64"),
    "td1024_fp32": (1024, "fp32"),
    "td512_fp64": (512, "fp64"),
}


def run_profile_case(name):
    """One small run of the headline workload for a profiler (ncu): the
    first time step of the time-dependent channel problem on a side x side
    mesh (S16, the channel scaled from the 256^2 mask), two GSIS iterations
    at the benchmark's synthetic settings.  Nothing is timed."""
    import torch

    from paper_2507_03975_gb300 import gsis
    side, prec = PROFILE_CASES[name]
    torch.cuda.set_device(0)
    p = W.config_timedep() if side == 1024 else W.channel_td_problem(side)
    td = W.TIMEDEP
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    opt = td_options(gsis, precision=gsis.FP64 if prec == "fp64" else gsis.FP32_SWEEP, fixed_iters=2)
    r = gsis.td_solve(p.dx, p.dy, p.mu, p.eta, p.w, t(p.sigma_a), t(p.sigma_s), t(p.q),
                      t(np.full(p.N, td["a"] * td["c"] * td["T0"] ** 4)), t(np.full(p.N, td["T0"])), td["dt"], 1,
                      c=td["c"], a=td["a"], cv=td["cv"], inflow=t(p.inflow.reshape(-1)), options=opt)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "status": r["status"], "iters": r["step_iters"].tolist()}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-si", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-intensity form of the headline")
    ap.add_argument("--no-channel", action="store_true", help="skip the steady 256^2 channel measurement")
    ap.add_argument("--channel-only", action="store_true", help="run only the steady channel GSIS measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the steady adjoint-gradient measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve measurement")
    ap.add_argument("--batch-only", action="store_true", help="run only the batched-solve measurement")
    ap.add_argument("--no-uw2", action="store_true", help="skip the second-order upwind measurement")
    ap.add_argument("--no-td-adjoint", action="store_true", help="skip the time-dependent adjoint measurement")
    ap.add_argument("--oracle-times", action="store_true",
                    help="time the FP64 oracle itself on the host cores (CPU only) and exit")
    ap.add_argument("--oracle-td-steps", type=int, default=0,
                    help="with --oracle-times: time this many real oracle steps of the headline workload")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES),
                    help="run one small instance of the headline workload once (for ncu) and exit")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args.profile_case)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.oracle_times:
        return run_oracle_times(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
