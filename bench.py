#!/usr/bin/env python3
"""Benchmark of the batched FP64 AdS4 collapse evolution (one JSON line on stdout).

Workload: the amplitude scan -- B = 256 Gaussian pulses Pi(x,0) = (2 eps/pi) exp(-4 tan^2 x /
(pi^2 sigma^2)), sigma = 1/16, eps log-uniform in [5, 80] (seed 0), N = 4097 grid points each,
RK4 with dt ~ 0.5 dx, constraints solved in every RK stage, per-instance stop when min A < 2^-7.
One bench step = one persistent launch that advances every running instance by STEP_RK RK4
steps.  Metric: FP64 RK4 point-substeps per second (sum over instances of N x 4 x RK4 steps
actually taken, over the device time of the timed launches).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun the workload is one batch of B x world instances (one seed), split over the ranks
by longest-processing-time first on the estimated work (N x RK4 steps to the job's end): every
rank evolves its share (B instances of the amplitude scan), no collective on the data path
(weak scaling); rank 0 gathers the per-instance results and prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1706_07413_b300 import workloads as W  # noqa: E402

METRIC = "batched FP64 RK4 point-substeps/s"
UNIT = "point-substeps/s"
STEP_RK = 256             # RK4 steps per bench step (one persistent launch)
B_DEFAULT, N_DEFAULT = 256, 4097
THETA = 2.0 ** -7
SIGMA_KO = 0.5
# Algorithmic FP64 flops (FMA = 2) per point-substep, tallied from the evolution kernel's
# source for the sequential scheme it computes: cell data 40 (rho and its node factors 5,
# midpoint interpolation, rho and factors 13, Simpson increment 3, RK4-in-x affine map
# 19); sequential scans, A, the fused A e^{-delta} (13, table-driven exp on the argument in
# units of ln2/256), fluxes 20.75; RHS stencils with dissipation 30; RK4 update 7.  The
# parallel-scan overheads (per-thread aggregates, warp shuffles, ~7 flops) are not counted.
FLOPS_PER_POINT_SUBSTEP = 97.75
# The same tally for the evolved-A schemes (A from Eq. (eq:adot), SSP Runge-Kutta), per stage:
# delta cell data 20, delta scan 1, fused A e^{-delta} 13, fluxes 3, A-dot 3 and the A update
# (SSP-RK3: 4 on average over the stages), slice mass 2 (once per step), RHS 30, Phi/Pi update
# (SSP-RK3: 8 on average); the re-integration of A every 64 steps adds < 0.2 and is not counted.
SCHEMES = {   # name: (config value, stages per step, flops per point-substep, A re-integration)
    "rk4": (0, 4, FLOPS_PER_POINT_SUBSTEP, 0),
    "evolved_a_rk3": (1, 3, 84.0, 64),
    "evolved_a_rk2": (2, 2, 83.5, 64),
    # A = 1, delta = 0 held fixed (the paper's Table II case): per point-substep u = tan^2 x Phi
    # (1), the RHS with dissipation (30), the Shu-Osher update (8 averaged over the 3 stages) and
    # the step-end mass sum (5 per step)
    "fixed_metric_rk3": (3, 3, 1.0 + 30.0 + 8.0 + 5.0 / 3.0, 0),
}
# FP64 instructions per point-substep of the adjoint: the forward pass recorded by the evolution
# kernel (evolve_kernel<8, 128, 4, true>) and the adjoint kernel's backward sweep (phase B, per
# segment): ncu's smsp__sass_thread_inst_executed_op_d{add,mul,fma}_pred_on.sum of those launches
# divided by their point-substeps, captured on a reduced adjoint batch (38 instances at N = 4097,
# 96 steps in two 48-step segments; per point-substep the same instruction mix as the bench's
# 64-instance batch); used only while the kernel sources are unchanged
ADJ_ISSUE = {"sha256": "647182ea36803fad5233ec8fbc9159e2263c8bd13a710fae2f524ca4085b6e8d",
             "forward_record": (24925416 + 3955116 + 4205327532) / (38 * 4097 * 96 * 4),
             "phase_B": (3954432 + 122056 + 2894894720) / (38 * 4097 * 48 * 4)}
L2_FLUSH_BYTES = 512 << 20
CPU_SAMPLE_STEPS = 800    # oracle sample of the cpu_baseline leg: ~10 s on 16 host threads
REF_SAMPLE_STEPS = 100    # oracle sample per bench step of the reference arm
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one timed evolve_kernel launch of
# the amplitude scan, from an ncu capture of this script's headline launch; reported only while
# the kernel source and the kernel shape are the ones the counters were taken on.
TRAFFIC = {"kernel_sha256": "ca296d6613958823a02695a1cacccc351e232a7f9d64edbcb3234f81141078f6",
           "shape_P_NT_CL": [8, 256, 2], "dram_bytes_per_launch": 17760000 + 64856320,
           # FP64 instructions (DADD + DMUL + DFMA, thread level) per point-substep, same capture
           "fp64_instr_per_point_substep": (328507392 + 54013952 + 75394985984) / 1074003968}


def kernel_digest(files=("evolve.cuh", "expneg.cuh")):
    """SHA-256 of the evolution kernel's code (comments and blank lines removed)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1706_07413_b300", "csrc", f)) as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def oracle_rate(insts, nsteps, threads):
    """The CPU oracle, as it stands, on a bounded sample: point-substeps/s with `threads` host
    threads (one instance per thread at a time; the ctypes call releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    oracle.build()

    def run(it):
        N = it.N
        dt = oracle.dt_for(N)
        r = oracle.evolve(np.zeros(N), W.gaussian_pi(N, it.eps, it.sigma), dt, nsteps,
                          sigma=SIGMA_KO, theta=THETA)
        return N * 4 * r.steps

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        work = sum(ex.map(run, insts))
    el = time.perf_counter() - t0
    return work / el, el, work


def batch_fields(insts, sol):
    """Set the initial slices of `insts` on solver `sol`: mode sums through the library's own
    synthesis, Gaussian pulses uploaded (Phi = 0)."""
    B = len(insts)
    modes = [it for it in insts if it.kind == "modes"]
    if modes:
        K = max(len(it.coeffs) for it in modes)
        a = np.zeros((B, K))
        for b, it in enumerate(insts):
            if it.kind == "modes":
                a[b, : len(it.coeffs)] = it.coeffs
        sol.set_initial_modes(a)
        for b, it in enumerate(insts):
            if it.kind == "gauss":
                sol.set_state(b, np.zeros(it.N), W.gaussian_pi(it.N, it.eps, it.sigma), 0)
    else:
        Pi0 = W.packed([W.gaussian_pi(it.N, it.eps, it.sigma) for it in insts])
        sol.set_initial(np.zeros_like(Pi0), Pi0)


# per-GPU batch of every workload: (generator, instances per GPU, seed, job end time t_end)
WORKLOADS = {"amp_scan": (W.amp_scan, B_DEFAULT, 0, 100.0), "large": (W.large, 148, 3, 200.0),
             "uneven": (W.uneven, 192, 1, 200.0), "production": (W.production, 15, 4, 500.0)}


def workload_insts(name, rank, world=1):
    """This rank's share of the workload's global batch (B x world instances, one seed), the
    share's indices in the global batch, and the workload's description."""
    from paper_1706_07413_b300 import shard
    gen, B, seed, t_end = WORKLOADS[name]
    glob = gen(B=B * world, seed=seed)
    if world == 1:
        idx = list(range(len(glob)))
    else:
        idx = shard.partition(shard.instance_work([it.N for it in glob], t_end), world)[rank]
    insts = [glob[i] for i in idx]
    desc = {
        "amp_scan": (f"amplitude scan: B={B_DEFAULT} Gaussian pulses per GPU, N={N_DEFAULT}, "
                     "sigma=1/16, eps log-uniform [5,80], RK4 dt=0.5dx, constraints every "
                     "substep, early exit at min A < 2^-7"),
        "large": ("large grids: B=148 per GPU at N=8193 (2-CTA clusters), half Gaussian pulses "
                  "(sigma U[1/32,1/8], eps log-uniform [5,80]), half two-mode data, early exit "
                  "at min A < 2^-7"),
        "uneven": ("uneven batch: B=192 per GPU, N uniform in {2049, 4097, 8193}, "
                   "Pi = sum_{j<16} eps e^{-j/3}(1+0.05 N(0,1)) e_j, eps U[0.05,0.2]"),
        "production": ("production resolution: B=15 Gaussian pulses per GPU at N=32769 (one "
                       "cluster each: the 15 clusters of 8 or 9 CTAs that fit at once), "
                       "sigma=1/16, eps log-uniform [5,80], early exit at min A < 2^-7"),
    }[name]
    return insts, idx, desc


def side_rate(insts, stream, local, rk_steps, flush, substeps=4, tune=True, **kw):
    """Point-substeps/s of one persistent launch of rk_steps time steps on another batch
    (substeps: Runge-Kutta stages per step of the scheme selected by kw; kernel shapes picked by
    the autotuner unless tune is false)."""
    import torch
    from paper_1706_07413_b300 import adscl
    sol = adscl.Solver([it.N for it in insts], ko_sigma=SIGMA_KO, collapse_threshold=THETA,
                       device=local, stream=stream.cuda_stream, **kw)
    batch_fields(insts, sol)
    if tune:
        sol.autotune(8)
    dt, _ = sol.clock()
    T = rk_steps * float(dt.max())
    sol.evolve(T / 8)
    torch.cuda.synchronize()
    _, s0 = sol.clock()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        sol.evolve(T / 8 + T)
        e1.record(stream)
    torch.cuda.synchronize()
    _, s1 = sol.clock()
    work = float(np.sum((s1 - s0) * sol.N.astype(np.float64) * substeps))
    sol.close()
    return work / (e0.elapsed_time(e1) / 1e3)


def autotune_report(stream, local):
    """Default kernel shape against the autotuned one on the two latency-bound cases: the single
    pulse (one instance, N = 1025, eps = 40, sigma = 1/16) and a batch smaller than the SM count
    (64 pulses at N = 4097); plus the single pulse run to t = 10 (or collapse) with the tuned
    shape."""
    import torch
    from paper_1706_07413_b300 import adscl
    out = {}
    cases = (("single_N1025", W.single(), 400), ("batch64_N4097", W.amp_scan(B=64), 64))
    for name, insts, steps in cases:
        res = {}
        for tuned in (False, True):
            sol = adscl.Solver([it.N for it in insts], ko_sigma=SIGMA_KO, collapse_threshold=THETA,
                               device=local, stream=stream.cuda_stream)
            batch_fields(insts, sol)
            shapes = sol.autotune(8) if tuned else sol.shapes()
            dt, _ = sol.clock()
            T = steps * float(dt.max())
            sol.evolve(T / 8)
            torch.cuda.synchronize()
            _, s0 = sol.clock()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                sol.evolve(T / 8 + T)
                e1.record(stream)
            torch.cuda.synchronize()
            _, s1 = sol.clock()
            ms = e0.elapsed_time(e1)
            work = float(np.sum((s1 - s0) * sol.N.astype(np.float64) * 4.0))
            res["tuned" if tuned else "default"] = {
                "shape_P_NT_CL": list(shapes[insts[0].N]), "value": work / (ms / 1e3),
                "unit": UNIT, "us_per_rk4_step": 1e3 * ms / max(1, int(np.max(s1 - s0)))}
            if tuned and name == "single_N1025":
                sol.set_initial(np.zeros(insts[0].N), W.gaussian_pi(insts[0].N, insts[0].eps,
                                                                     insts[0].sigma))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                tr, tc, m, st = sol.evolve(10.0)
                res["to_t10"] = {"wall_s": time.perf_counter() - t0, "t_reached": float(tr[0]),
                                 "t_collapse": float(tc[0]), "rk4_steps": int(sol.clock()[1][0]),
                                 "theta": THETA}
            sol.close()
        out[name] = res
    return out


def paper_configs_report(stream, local, steps=64):
    """The configurations the paper times (Sec. IV, Tables I and II), one instance each: N = 32769
    with A and delta dynamical (the paper's scheme: A evolved by Eq. (eq:adot), re-integrated
    every 64 steps, SSP-RK3; and the classic RK4 with A integrated every stage), and the fixed
    metric A = 1, delta = 0 at the Table II grid N = 65537; each on the cluster shape the
    autotuner picks for the single instance (a 16-CTA cluster for both grids); the fixed metric
    also on the whole GPU (adscl_evolve_wide)."""
    import torch
    from paper_1706_07413_b300 import adscl
    out = {}
    for name, N, scheme, stages, reint in (("table1_evolved_A_rk3", 32769, 1, 3, 64),
                                           ("table1_rk4_constraint_A", 32769, 0, 4, 0),
                                           ("table2_fixed_metric_rk3", 65537, 3, 3, 0)):
        sol = adscl.Solver([N], ko_sigma=SIGMA_KO, collapse_threshold=THETA, device=local,
                           stream=stream.cuda_stream, scheme=scheme, a_reint_every=reint)
        sol.set_initial(np.zeros(N), W.gaussian_pi(N, 40.0, 1.0 / 16))
        shape = sol.autotune(8)[N]
        dt, _ = sol.clock()
        sol.evolve(4 * dt[0])
        torch.cuda.synchronize()
        _, s0 = sol.clock()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            sol.evolve((4 + steps) * dt[0])
            e1.record(stream)
        torch.cuda.synchronize()
        _, s1 = sol.clock()
        ms = e0.elapsed_time(e1)
        n = int(s1[0] - s0[0])
        out[name] = {"N": N, "steps": n, "kernel_shape_P_NT_CL": list(shape), "ms_per_step": ms / max(n, 1),
                     "point_substeps_per_s": N * stages * n / (ms / 1e3),
                     "wall_s_per_unit_time": ms / max(n, 1) / 1e3 / float(dt[0])}
        if scheme == 3:
            # the same single instance on the whole GPU (adscl_evolve_wide: one cooperative
            # launch of ceil(N / 500) CTAs, a grid-wide barrier per step)
            sol.evolve_wide((8 + steps) * dt[0])
            torch.cuda.synchronize()
            _, s0 = sol.clock()
            with torch.cuda.stream(stream):
                e0.record(stream)
                sol.evolve_wide((8 + 2 * steps) * dt[0])
                e1.record(stream)
            torch.cuda.synchronize()
            _, s1 = sol.clock()
            ms = e0.elapsed_time(e1)
            n = int(s1[0] - s0[0])
            out[name]["whole_gpu"] = {"ctas": -(-N // 500), "ms_per_step": ms / max(n, 1),
                                      "point_substeps_per_s": N * stages * n / (ms / 1e3),
                                      "wall_s_per_unit_time": ms / max(n, 1) / 1e3 / float(dt[0])}
        sol.close()
    return out


def full_job(sol, B, stages, stream, T, retune, dist=None):
    """The whole job: every instance from its current slice to t = T (or its collapse) in evolve
    calls of one time unit; wall time on the host clock, device-resident fields.  With retune,
    autotune is called after every unit of t: its choice is cached per number of running
    instances (a half-octave bucket), so it re-tunes only when collapses have thinned the batch
    enough (the time of those tunings is part of the job)."""
    import torch
    outs = [torch.empty(B, dtype=torch.float64, device="cuda") for _ in range(3)] + \
        [torch.empty(B, dtype=torch.int32, device="cuda")]
    Ns = sol.N.astype(np.float64)
    _, s0 = sol.clock()
    running = []
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    t = 0.0
    tunes = []
    with torch.cuda.stream(stream):
        while t < T - 1e-12:
            t = min(T, t + 1.0)
            sol.evolve(t, out=outs)
            if retune:
                before = sol.shapes()
                sol.autotune(8)
                after = sol.shapes()
                if after != before:
                    tunes.append({"t": t, "shapes": {str(k): list(v) for k, v in after.items()}})
            # instances still evolving (RUNNING or DONE at this t), sampled every 10 units of t
            running.append(int((outs[3] <= 1).sum().item()) if int(t) % 10 == 0 or t >= T else None)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    _, s1 = sol.clock()
    work = float(np.sum((s1 - s0) * Ns * stages))
    st = outs[3].cpu().numpy()
    collapsed = int(np.sum(st == 2))
    if dist is not None:
        from paper_1706_07413_b300 import shard
        wall, work = shard.reduce_timing(wall, work, dist, device="cuda")
        c = torch.tensor([collapsed], dtype=torch.float64, device="cuda")
        dist.all_reduce(c)
        collapsed = int(c.item())
    return {"t_end": T, "wall_s": wall, "point_substeps": work, "point_substeps_per_s": work / wall,
            "collapsed": collapsed, "running_every_10": [r for r in running if r is not None],
            "shape_changes": tunes,
            "note": "wall time on the host clock around all evolve calls (one per unit of t)"}


def run_full_job(args, sol, insts, wl_desc, stages, shapes, stream, ws, rank, dist):
    """--full-job T: the whole job instead of the bench line (one JSON line)."""
    res = full_job(sol, len(insts), stages, stream, args.full_job,
                   not (args.no_autotune or args.shape), dist)
    if rank == 0:
        line = {"mode": "full_job", "workload": wl_desc, "instances": len(insts) * ws,
                "n_gpus": ws, **res,
                "kernel_shape_P_NT_CL": {str(k): list(v) for k, v in shapes.items()}}
        print(json.dumps(line), flush=True)


def job_amp_scan(stream, local, T=100.0):
    """The amplitude-scan job from t = 0 to T (every pulse to T or its collapse), as one side
    figure of the default bench: the autotuner's start-up choice and its re-tunes are included."""
    from paper_1706_07413_b300 import adscl
    insts, _, desc = workload_insts("amp_scan", 0)
    sol = adscl.Solver([it.N for it in insts], ko_sigma=SIGMA_KO, collapse_threshold=THETA,
                       device=local, stream=stream.cuda_stream)
    batch_fields(insts, sol)
    t0 = time.perf_counter()
    sol.autotune(8)
    tune0 = time.perf_counter() - t0
    res = full_job(sol, len(insts), 4, stream, T, True)
    res["wall_s_with_first_tune"] = res["wall_s"] + tune0
    res["workload"] = desc
    sol.close()
    return res


def job_uneven_spectra(stream, local, T=10.0, precision_name="BF16X3"):
    """The uneven batch with its spectra (192 instances, N in {2049, 4097, 8193}, mode-sum data)
    from t = 0 to T: evolve one unit of t, then the 64 mode energies of every instance on the
    tensor cores and the TTF quantities (adscl_track), timed as one job on the host clock; the
    spectrum's share is the time of the same number of spectrum calls on the final slices, timed
    alone with CUDA events.  Also: the tensor-core energies against the FP64 projection on the
    last slice, and how far the particle number and the total energy moved over the job."""
    import torch
    from paper_1706_07413_b300 import adscl
    insts, _, desc = workload_insts("uneven", 0)
    prec = getattr(adscl, "PREC_" + precision_name)
    sol = adscl.Solver([it.N for it in insts], ko_sigma=SIGMA_KO, collapse_threshold=THETA,
                       out_dt=1.0, device=local, stream=stream.cuda_stream)
    batch_fields(insts, sol)
    t0 = time.perf_counter()
    shapes = sol.autotune(8)
    tune_s = time.perf_counter() - t0
    n_snap = int(round(T)) + 1
    sol.spectrum(64, prec)          # builds the split mode tables once (outside the job)
    torch.cuda.synchronize()
    _, s0 = sol.clock()
    t0 = time.perf_counter()
    th, qh, Eh = sol.track(0.0, 1.0, n_snap, 64, prec, energies=True)
    wall = time.perf_counter() - t0
    _, s1 = sol.clock()
    work = float(np.sum((s1 - s0) * sol.N.astype(np.float64) * 4.0))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    E = torch.empty((len(insts), 64), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(n_snap):
            sol.lib.adscl_spectrum(sol.ctx, 64, prec, E.data_ptr(), 1)
        e1.record(stream)
    torch.cuda.synchronize()
    spec_s = e0.elapsed_time(e1) / 1e3
    E64 = sol.spectrum(64, adscl.PREC_FP64)
    _, _, mass, _ = sol.evolve(T)
    tc_err = float((np.abs(Eh[-1] - E64).max(axis=1) / mass).max())
    dN = np.abs(qh[:, :, 1] / qh[0, :, 1] - 1.0).max(axis=0)
    dE = np.abs(qh[:, :, 0] / qh[0, :, 0] - 1.0).max(axis=0)
    sol.close()
    return {"t_end": T, "snapshots": n_snap, "workload": desc + f"; spectra every unit of t ({precision_name})",
            "wall_s": wall, "point_substeps_per_s": work / wall, "autotune_s": tune_s,
            "kernel_shape_P_NT_CL": {str(k): list(v) for k, v in shapes.items()},
            "spectrum_s": spec_s, "spectrum_share": spec_s / wall,
            "tc_vs_fp64_max_dE_over_M": tc_err,
            "ttf": {"particle_number_max_rel_change": {"median": float(np.median(dN)), "max": float(dN.max())},
                    "total_energy_max_rel_change": {"median": float(np.median(dE)), "max": float(dE.max())},
                    "temperature_range": [float(qh[:, :, 2].min()), float(qh[:, :, 2].max())]},
            "note": "wall time on the host clock around one adscl_track call (evolve + spectrum + "
                    "TTF per unit of t, history copied to the host at the end)"}


def job_large_spectra_refine(stream, local, T=4.0, refine_iters=3, refine_steps=256):
    """The large-grid configuration as a bounded job: 148 instances at N = 8193 (2-CTA clusters;
    half Gaussian pulses, half two-mode data) from t = 0 to T with the 64 mode energies on the
    tensor cores (BF16x3) and the TTF quantities every unit of t (one adscl_track call, host
    clock), and the adjoint-driven refinement of the 8 approximate quasi-periodic seeds at the
    same resolution (refine_iters gradient steps, each gradient over refine_steps RK4 steps)."""
    import torch
    from paper_1706_07413_b300 import adscl
    from paper_1706_07413_b300.autograd import refine_modes
    insts, _, desc = workload_insts("large", 0)
    sol = adscl.Solver([it.N for it in insts], ko_sigma=SIGMA_KO, collapse_threshold=THETA,
                       out_dt=1.0, device=local, stream=stream.cuda_stream)
    batch_fields(insts, sol)
    shapes = sol.autotune(8)
    n_snap = int(round(T)) + 1
    sol.spectrum(64, adscl.PREC_BF16X3)
    torch.cuda.synchronize()
    _, s0 = sol.clock()
    t0 = time.perf_counter()
    th, qh, _ = sol.track(0.0, 1.0, n_snap, 64, adscl.PREC_BF16X3)
    wall = time.perf_counter() - t0
    _, s1 = sol.clock()
    work = float(np.sum((s1 - s0) * sol.N.astype(np.float64) * 4.0))
    tr, tc, m, st = sol.evolve(T)
    collapsed = int(np.sum(st == adscl.COLLAPSED))
    sol.close()
    seeds = W.qp_seeds(N=8193, K=32)
    a0 = np.stack([it.coeffs for it in seeds])
    sr = adscl.Solver([8193] * len(seeds), ko_sigma=SIGMA_KO, spec_J=32, ckpt_every=64, device=local,
                      stream=stream.cuda_stream)
    dt = float(sr.clock()[0][0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, hist = refine_modes(sr, a0, refine_steps * dt, iters=refine_iters, step=0.02)
    torch.cuda.synchronize()
    refine_s = time.perf_counter() - t0
    h = hist.numpy()
    sr.close()
    return {"t_end": T, "snapshots": n_snap, "workload": desc + "; spectra (BF16x3) and TTF every unit of t",
            "wall_s": wall, "point_substeps_per_s": work / wall, "collapsed": collapsed,
            "kernel_shape_P_NT_CL": {str(k): list(v) for k, v in shapes.items()},
            "refinement": {"seeds": len(seeds), "N": 8193, "iterations": refine_iters,
                           "gradient_window_steps": refine_steps, "wall_s": refine_s,
                           "gradients": refine_iters + 1,
                           "drift_J_last_over_first": {"median": float(np.median(h[-1] / h[0])),
                                                       "max": float(np.max(h[-1] / h[0]))}},
            "note": "wall time on the host clock around one adscl_track call, and around the "
                    "refinement (its gradients, each a forward pass, checkpoint recomputation "
                    "and backward sweep)"}


def run_reference(args):
    """The reference arm: the sequential FP64 CPU oracle on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    threads = min(os.cpu_count() or 1, 16)
    insts = W.amp_scan()[: 2 * threads]
    nsteps = REF_SAMPLE_STEPS
    for _ in range(args.warmup):
        oracle_rate(insts[:threads], 4, threads)
    rates, total_t, total_w = [], 0.0, 0
    for _ in range(args.steps):
        r, el, w = oracle_rate(insts, nsteps, threads)
        rates.append(r)
        total_t += el
        total_w += w
    value = total_w / total_t
    sample = f"{len(insts)} of the 256 N=4097 pulses x {nsteps} RK4 steps per bench step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_insts("amp_scan", 0)[2],
                   "step": f"bounded sample of the same workload: {len(insts)} of the pulses x "
                           f"{nsteps} RK4 steps per bench step",
                   "scheme": "rk4",
                   "oracle": "sequential FP64 C, one instance per host thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-others", action="store_true")
    ap.add_argument("--no-jobs", action="store_true",
                    help="skip the whole-job side figures (amplitude scan to t = 100, uneven batch "
                         "with spectra to t = 10, large grids with spectra to t = 4 and the "
                         "refinement of the quasi-periodic seeds)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernel shapes instead of the autotuner's choice")
    ap.add_argument("--shape", default="",
                    help="P,NT,CL: run the timed batch with this kernel shape instead of tuning "
                         "(for profiling, where a profiler distorts the tuner's timings)")
    ap.add_argument("--workload", default="amp_scan", choices=["amp_scan", "large", "uneven", "production"],
                    help="batch to time (the metric's workload is amp_scan)")
    ap.add_argument("--scheme", default="rk4", choices=sorted(SCHEMES),
                    help="time-stepping scheme (the metric's scheme is rk4)")
    ap.add_argument("--adjoint-batch", type=int, default=64,
                    help="instances of the adjoint leg (64: the adjoint configuration; fewer for "
                         "counter captures of a few GB)")
    ap.add_argument("--adjoint-ckpt", type=int, default=256,
                    help="checkpoint interval of the adjoint leg in steps")
    ap.add_argument("--adjoint-steps", type=int, default=1024,
                    help="RK4 steps of the adjoint/forward-ratio window (32768 = the adjoint "
                         "batch's whole T = 2 pi)")
    ap.add_argument("--full-job", type=float, default=0.0, metavar="T",
                    help="instead of the bench line: evolve the whole workload to t = T (every "
                         "instance runs until T or its collapse) and print the job's wall time, "
                         "throughput and collapse count as one JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_1706_07413_b300 import adscl

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        host_group = dist.new_group(backend="gloo")

    stream = torch.cuda.Stream()
    insts, glob_idx, wl_desc = workload_insts(args.workload, rank, ws)
    B = len(insts)
    N = insts[0].N
    amp = args.workload == "amp_scan" and args.scheme == "rk4"
    Pi0 = W.packed([W.gaussian_pi(N, it.eps, it.sigma) for it in insts]) if amp else None
    Phi0 = np.zeros_like(Pi0) if amp else None

    tflops_peak = adscl.probe_fp64(local, stream.cuda_stream)

    scheme_id, stages, flops_pps, reint = SCHEMES[args.scheme]
    sol = adscl.Solver([it.N for it in insts], ko_sigma=SIGMA_KO, collapse_threshold=THETA,
                       device=local, stream=stream.cuda_stream, scheme=scheme_id,
                       a_reint_every=reint)
    batch_fields(insts, sol)
    t0 = time.perf_counter()
    fixed_shape = [int(v) for v in args.shape.split(",")] if args.shape else None
    if fixed_shape:
        for n in sorted(set(it.N for it in insts)):
            sol.set_shape(n, *fixed_shape)
    shapes = sol.shapes() if (args.no_autotune or fixed_shape) else sol.autotune(8)
    tune_s = time.perf_counter() - t0
    if args.full_job > 0:
        run_full_job(args, sol, insts, wl_desc, stages, shapes, stream, ws, rank, dist)
        if dist is not None:
            dist.destroy_process_group()
        return
    dt, _ = sol.clock()
    dstep = STEP_RK * float(dt.max())
    outs = [torch.empty(B, dtype=torch.float64, device="cuda") for _ in range(3)] + \
        [torch.empty(B, dtype=torch.int32, device="cuda")]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    t = 0.0
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            t += dstep
            sol.evolve(t, out=outs)
    torch.cuda.synchronize()
    _, step0 = sol.clock()
    launches0 = sol.launch_count()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()                    # L2 flush, outside the timed interval
                evs[k][0].record(stream)
                t += dstep
                sol.evolve(t, out=outs)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = sol.launch_count() - launches0
    _, step1 = sol.clock()
    ms = [a.elapsed_time(b) for a, b in evs]
    dev_s = sum(ms) / 1e3
    work = float(np.sum((step1 - step0) * sol.N.astype(np.float64) * stages))
    tr, tc, m, st = sol.evolve(t)   # (already there: reads statuses only)
    collapsed = int(np.sum(st == adscl.COLLAPSED))

    if dist is not None:
        from paper_1706_07413_b300 import shard
        dev_s, work_all = shard.reduce_timing(dev_s, work, dist, device="cuda")
        # per-instance results of the whole batch on rank 0 (host data over a gloo group)
        res = shard.gather_results(np.stack([st.astype(np.float64), tc, m], axis=1), glob_idx,
                                   B * ws, dist, group=host_group)
        if rank == 0:
            collapsed = int(np.sum(res[:, 0] == adscl.COLLAPSED))
    else:
        work_all = work
    value = work_all / dev_s

    # roofline of the evolution kernel (it is >99% of each timed launch)
    achieved_tflops = (work * flops_pps) / dev_s / 1e12
    traffic = issue = None
    if amp and kernel_digest() == TRAFFIC["kernel_sha256"] and \
            list(shapes.get(N_DEFAULT, ())) == TRAFFIC["shape_P_NT_CL"]:
        traffic = TRAFFIC["dram_bytes_per_launch"]
        # FP64 issue: instructions per second against the probe's FMA rate (one FMA = 2 flops)
        ipps = TRAFFIC["fp64_instr_per_point_substep"]
        issue = {"fp64_instr_per_point_substep": ipps,
                 "achieved_ginstr_per_s": work * ipps / dev_s / 1e9,
                 "peak_ginstr_per_s": tflops_peak * 1e12 / 2 / 1e9,
                 "frac": (work * ipps / dev_s) / (tflops_peak * 1e12 / 2)}
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": tflops_peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / tflops_peak, "traffic": traffic,
                "peak_source": "measured FP64 FMA-chain probe on this GPU (FMA = 2 flops)",
                "flops_per_point_substep": flops_pps, "fp64_issue": issue}

    # the other batch shapes, one launch of 128 RK4 steps each (default workload only)
    others = None
    if rank == 0 and amp and not args.no_others:
        others = {}
        for name in ("large", "uneven", "production"):
            oi, _, od = workload_insts(name, 0)
            others[name] = {"value": side_rate(oi, stream, local, 128, flush), "unit": UNIT,
                            "workload": od, "rk_steps": 128}
        # the paper's production scheme on the amplitude scan: A evolved with Eq. (eq:adot),
        # re-integrated every 64 steps, SSP-RK3 (3 substeps per step)
        oi, _, od = workload_insts("amp_scan", 0)
        v = side_rate(oi, stream, local, 128, flush, substeps=3, scheme=adscl.SCHEME_EVOLVED_A_RK3,
                      a_reint_every=64)
        vf = side_rate(oi, stream, local, 128, flush, substeps=3, scheme=adscl.SCHEME_FIXED_METRIC_RK3)
        others["autotune"] = autotune_report(stream, local)
        others["paper_configs"] = paper_configs_report(stream, local)
        others["amp_scan_evolved_A_rk3"] = {
            "value": v, "unit": UNIT, "rk_steps": 128,
            "workload": od + "; evolved-A scheme, SSP-RK3, A re-integrated every 64 steps",
            "rk_steps_per_s": v / (3.0 * N_DEFAULT * B_DEFAULT),
            "rk4_steps_per_s_same_batch": value / (4.0 * N_DEFAULT * B_DEFAULT)}
        others["amp_scan_fixed_metric_rk3"] = {
            "value": vf, "unit": UNIT, "rk_steps": 128,
            "workload": od + "; fixed metric A = 1, delta = 0 (no constraints), SSP-RK3",
            "rk_steps_per_s": vf / (3.0 * N_DEFAULT * B_DEFAULT)}

    # whole jobs of the configurations (default run on one GPU only)
    jobs = None
    if rank == 0 and ws == 1 and amp and not args.no_jobs:
        jobs = {"amp_scan_to_t100": job_amp_scan(stream, local, 100.0),
                "uneven_spectra_to_t10": job_uneven_spectra(stream, local, 10.0),
                "large_spectra_refine_to_t4": job_large_spectra_refine(stream, local, 4.0)}

    # one instance per launch, same workload, for the batched-vs-one-per-launch comparison
    opl = None
    if rank == 0 and amp:
        nopl = 4
        s1 = adscl.Solver([N] * nopl, ko_sigma=SIGMA_KO, collapse_threshold=THETA, device=local,
                          one_per_launch=True, stream=stream.cuda_stream)
        s1.set_initial(Phi0[: nopl * N].copy(), Pi0[: nopl * N].copy())
        with torch.cuda.stream(stream):
            s1.evolve(dstep / 4, out=[o[:nopl] for o in outs])
            torch.cuda.synchronize()
            _, sa = s1.clock()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s1.evolve(dstep / 4 + dstep / 2, out=[o[:nopl] for o in outs])
            e1.record(stream)
        torch.cuda.synchronize()
        _, sb = s1.clock()
        w1 = float(np.sum((sb - sa) * N * 4.0))
        opl = w1 / (e0.elapsed_time(e1) / 1e3)
        s1.close()

    # adjoint/forward time ratio on the adjoint batch: 64 instances at N = 4097, Pi(x,0) =
    # sum_{j<32} a_j e_j with a_j = U(0, 0.1) exp(-j/4), dt = 2 pi / 32768 (T = 2 pi is 32768 steps),
    # 256-step checkpoints; timed over a window of ADJ_STEPS steps (the ratio does not depend on
    # the window length: both passes scale with the step count)
    adj = None
    if rank == 0 and amp and not args.no_adjoint:
        ADJ_STEPS = args.adjoint_steps
        ainst = W.adjoint_batch(B=args.adjoint_batch)
        a = np.stack([it.coeffs for it in ainst])
        sa = adscl.Solver([ainst[0].N] * len(ainst), ko_sigma=SIGMA_KO, collapse_threshold=-1.0,
                          out_dt=2 * math.pi, spec_J=32, ckpt_every=args.adjoint_ckpt, device=local,
                          stream=stream.cuda_stream)
        dta, _ = sa.clock()
        Ta = ADJ_STEPS * dta[0]
        sa.grad(a, Ta)                      # warm-up (allocates the stage storage)
        sa.set_initial_modes(a)
        sa.evolve(Ta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sa.set_initial_modes(a)
        sa.evolve(Ta)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        Jv, gv = sa.grad(a, Ta)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        st_bytes, st_bufs, st_segs, st_recomp = sa.adjoint_storage()
        # the same with the autotuned forward shape (64 instances: fewer than the SMs, so the
        # tuner splits each instance over a cluster; the adjoint kernel keeps one CTA each)
        tuned = sa.autotune(8)
        sa.grad(a, Ta)
        sa.set_initial_modes(a)
        sa.evolve(Ta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sa.set_initial_modes(a)
        sa.evolve(Ta)
        torch.cuda.synchronize()
        t_fwd_t = time.perf_counter() - t0
        t0 = time.perf_counter()
        sa.grad(a, Ta)
        torch.cuda.synchronize()
        t_adj_t = time.perf_counter() - t0
        cpu_adj = None
        if ws == 1 and not args.no_cpu_baseline:
            # the oracle's own gradient / forward time ratio on a bounded sample of the same
            # problem (one instance, 64 steps; sequential C, one thread)
            import oracle
            oracle.build()
            n_s = 64
            t0 = time.perf_counter()
            oracle.functional(a[0], ainst[0].N, n_s, dta[0], sigma=SIGMA_KO, Jm=32)
            t_of = time.perf_counter() - t0
            t0 = time.perf_counter()
            oracle.grad(a[0], ainst[0].N, n_s, dta[0], sigma=SIGMA_KO, Jm=32)
            t_og = time.perf_counter() - t0
            cpu_adj = {"ratio": t_og / t_of, "forward_s": t_of, "grad_s": t_og,
                       "sample": f"1 instance, N={ainst[0].N}, {n_s} steps, oracle (1 thread)"}
        adj_issue = None
        if (kernel_digest(("adjoint.cuh", "evolve.cuh", "expneg.cuh")) == ADJ_ISSUE["sha256"] and
                kernel_digest() == TRAFFIC["kernel_sha256"]):
            # default-shape context: the recording forward pass and the backward sweep (when the
            # stages do not all fit: the plain forward pass over the segments recomputed later
            # and the recording recomputation of those); FP64 instructions of the whole window
            # against the probe's FMA issue rate (FMA = 2 flops)
            w_adj = len(ainst) * ainst[0].N * 4.0 * ADJ_STEPS
            ipps = ADJ_ISSUE["forward_record"] + ADJ_ISSUE["phase_B"]
            ipps += TRAFFIC["fp64_instr_per_point_substep"] * st_recomp / max(st_segs, 1)
            adj_issue = {"fp64_instr_per_point_substep": ipps,
                         "frac": (w_adj * ipps / t_adj) / (tflops_peak * 1e12 / 2)}
        adj = {"value": t_adj_t / t_fwd_t, "forward_ms": 1e3 * t_fwd_t, "grad_ms": 1e3 * t_adj_t,
               "forward_shape_P_NT_CL": list(tuned[ainst[0].N]),
               "against": "the autotuned forward pass of the same batch",
               "cpu_oracle": cpu_adj,
               "default_shapes": {"forward_shape_P_NT_CL": [8, 512, 1], "forward_ms": 1e3 * t_fwd,
                                  "grad_ms": 1e3 * t_adj, "ratio": t_adj / t_fwd,
                                  "fp64_issue": adj_issue},
               "workload": f"{len(ainst)} mode-sum instances, N=4097, {ADJ_STEPS} RK4 steps of "
                           f"dt=2pi/32768, checkpoint every {args.adjoint_ckpt} steps, "
                           "J = sum_{j<32}(E_j(T)-E_j(0))^2",
               "grad_includes": "E(0), the forward pass (storing every stage when all segments fit "
                                "in device memory; else checkpoints and the stages of the last "
                                "segments that fit, each earlier segment recomputed before its "
                                "sweep), E(T), the backward sweep, the projection onto the modes",
               "stage_storage": {"bytes": st_bytes, "segment_buffers": st_bufs, "segments": st_segs,
                                 "recomputed": st_recomp}}
        sa.close()

    # spectrum timing (current slices of the amplitude scan, 64 modes)
    spec = None
    if rank == 0 and amp:
        spec = {}
        for name, prec in (("fp64", adscl.PREC_FP64), ("bf16x3", adscl.PREC_BF16X3),
                           ("tf32x3", adscl.PREC_TF32X3)):
            sol.spectrum(64, prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(5):
                sol.spectrum(64, prec)
            torch.cuda.synchronize()
            spec[name + "_ms"] = 1e3 * (time.perf_counter() - t0) / 5
        spec["note"] = "256 instances x 4097 points, 64 modes; includes the constraint solve for A"

    # end to end through the public API with host buffers: upload a fresh batch of initial
    # data from pinned memory, solve, evolve one bench step, read the per-instance results
    e2e = None
    if not args.no_e2e and amp:
        hPhi = torch.from_numpy(Phi0).pin_memory().numpy()
        hPi = torch.from_numpy(Pi0).pin_memory().numpy()
        res = [torch.empty(B, dtype=torch.float64).pin_memory().numpy() for _ in range(3)] + \
            [torch.empty(B, dtype=torch.int32).pin_memory().numpy()]
        sol_e = adscl.Solver([N] * B, ko_sigma=SIGMA_KO, collapse_threshold=THETA, device=local,
                             stream=stream.cuda_stream)
        if fixed_shape:
            sol_e.set_shape(N, *fixed_shape)
        elif not args.no_autotune:
            sol_e.autotune(8)   # warms the process cache; each timed iteration re-applies it
        ne = max(3, args.steps // 4)
        tot, work_e = 0.0, 0.0
        for k in range(ne + 1):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol_e.set_initial(hPhi, hPi)
            if not (args.no_autotune or fixed_shape):
                # cached (fresh batch, every instance running): no timing runs, the chosen
                # shapes are re-applied
                sol_e.autotune(8)
            st = sol_e.lib.adscl_evolve(sol_e.ctx, dstep, res[0].ctypes.data, res[1].ctypes.data,
                                        res[2].ctypes.data, res[3].ctypes.data, 0)
            el = time.perf_counter() - t0
            assert st == 0
            if k > 0:   # first one is a warm-up
                tot += el
                _, se = sol_e.clock()
                work_e += float(np.sum(se * N * 4.0))
        sol_e.close()
        h2d = 2 * B * N * 8
        d2h = B * (3 * 8 + 4)
        if dist is not None:   # whole job: the work of every rank over the slowest rank's time
            from paper_1706_07413_b300 import shard
            tot, work_e = shard.reduce_timing(tot, work_e, dist, device="cuda")
        e2e_v = work_e / tot
        e2e = {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and ws == 1 and amp and not args.no_cpu_baseline:
        threads = min(os.cpu_count() or 1, 16)
        sample_insts = W.amp_scan()[: 2 * threads]
        rate, el, _ = oracle_rate(sample_insts, CPU_SAMPLE_STEPS, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{len(sample_insts)} of the 256 N=4097 pulses x {CPU_SAMPLE_STEPS} RK4 "
                         f"steps ({el:.1f} s wall)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl_desc,
                       "step": f"one persistent launch = {STEP_RK} RK4 steps of every running "
                               "instance",
                       "scheme": args.scheme,
                       "kernel_shape_P_NT_CL": {str(k): list(v) for k, v in shapes.items()},
                       "autotune_s": round(tune_s, 3) if not (args.no_autotune or fixed_shape) else None,
                       "window_t": [round(args.warmup * dstep, 6),
                                    round((args.warmup + args.steps) * dstep, 6)],
                       "collapsed_in_window": collapsed,
                       "l2": "flushed (512 MB write) before every timed launch",
                       "instances_total": B * ws,
                       "parallelism": (f"one batch of {B * ws} instances split over {ws} GPU(s) "
                                       "by longest-processing-time first, no collective on the "
                                       "data path; per-instance results gathered on rank 0")},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "one_per_launch": {"value": opl, "unit": UNIT, "instances": 4,
                               "batched_over_one_per_launch": (value / ws) / opl if opl else None},
            "adjoint_forward_ratio": adj,
            "spectrum": spec,
            "other_workloads": others,
            "jobs": jobs,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
