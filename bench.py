#!/usr/bin/env python3
"""Benchmark of the scaled-ILU Richardson smoother on GB300.

Workload (one "step"): one smoother application x <- x + M^{-1}(b - A x)
with 10 sweeps on L_s and 10 on the row-scaled Utilde_s (Alg. ILUJac; the
paper's model counts twenty Richardson iterations per smoother application),
on the 128^3 cut-cell pressure matrix (2,097,152 rows, ILUT(1e-3, 10), FP64,
one right-hand side).  Metric: algorithmic GB/s of the application (bytes
the method must move, defined below) and its fraction of the measured HBM
bandwidth.  Then, on the 27-point 256^3 matrix (16.8M rows, 449M entries),
the FGMRES(30) time to 1e-10 of the FP32-smoother path against the FP64
direct-trisolve path, and the FP32 smoother's GB/s.

Every rank runs an independent replica (the path does not shard on one
GPU: replicas only); value = bytes of all ranks / max time over ranks.

Algorithmic bytes (int32 CSR; vb = value bytes; R = right-hand sides):
  residual   nnz(A)*12 + 4(n+1) + 3 n R 8          (A, x, b read; r written)
  L sweep    nnz(L_s)(vb+4) + 4(n+1) + 3 n R vb     (L_s, y_in, r read; y_out written)
  U sweep    nnz(Ut_s)(vb+4) + 4(n+1) + 3 n R vb
  scaling    8 n  (dinv, read once, fused into the last L sweep)
  update     n R 8 (x read by the fused last U sweep)
  apply = residual + (mL-1) L sweeps + 8n + (mU-1) U sweeps + 8nR
(the first sweep of each factor starts from zero and costs no SpMV).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

EDGE = 128
TAU, FILL = 1e-3, 10
ML, MU = 10, 10
WORKLOAD = "cutcell7-128^3 ILUT(1e-3,10) FP64 smoother 10+10 sweeps, 1 RHS"


def sweep_bytes(n, nnz, R, vb):
    return nnz * (vb + 4) + 4 * (n + 1) + 3 * n * R * vb


def resid_bytes(n, nnzA, R):
    return nnzA * 12 + 4 * (n + 1) + 3 * n * R * 8


def apply_bytes(n, nnzA, nnzL, nnzU, R, vb, mL, mU):
    b = resid_bytes(n, nnzA, R)
    b += max(mL - 1, 0) * sweep_bytes(n, nnzL, R, vb)
    b += 8 * n
    b += max(mU - 1, 0) * sweep_bytes(n, nnzU, R, vb)
    b += 8 * n * R
    return b


def spmv_bytes(rows, cols, nnz):
    """y = T v for a CSR operator with `rows` rows over `cols` columns (FP64): T, v read, y written."""
    return nnz * 12 + 4 * (rows + 1) + 8 * cols + 8 * rows


def vcycle_bytes(st, nnzL, nnzU, mL, mU, nu):
    """Algorithmic bytes of one V-cycle from x = 0 (the preconditioner inside FGMRES): FP64 ILU
    smoother with m_L + m_U sweeps on the finest level (pre-smoothing from zero: no residual, no read
    of x; post-smoothing: a full application), per level r = b - A x, R r and x += P v, nu steps of
    l1-Jacobi before and after on the levels below (the first from zero: x = D^{-1} b), and the dense
    solve on the coarsest level.  The same counting as the smoother's (each operand read once per
    use), level sizes from silu_amg_stats."""
    rows, nza, nzp = st["rows"], st["nnz_A"], st["nnz_P"]
    L = st["levels"]
    n0 = rows[0]
    post = apply_bytes(n0, nza[0], nnzL, nnzU, 1, 8, mL, mU)
    pre = post - resid_bytes(n0, nza[0], 1) - 8 * n0
    total = pre + post
    for l in range(L - 1):
        n, nc = rows[l], rows[l + 1]
        if l > 0:
            jac = spmv_bytes(n, n, nza[l]) + 3 * 8 * n  # x + D^{-1}(b - A x): b, l1 diagonal, x read
            total += (3 * 8 * n if nu > 0 else 8 * n) + max(2 * nu - 1, 0) * jac
        total += resid_bytes(n, nza[l], 1)               # r = b - A x
        total += spmv_bytes(nc, n, nzp[l])               # b_{l+1} = R r (R = P^T, as many entries as P)
        total += spmv_bytes(n, nc, nzp[l]) + 8 * n       # x += P v (x read too)
    nc = rows[L - 1]
    total += 8 * nc * nc + 16 * nc                       # dense inverse of the coarsest operator
    return total


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sweep_source_hash():
    h = hashlib.sha256()
    for f in ("kernels_staged.cu", "device.cuh"):
        with open(os.path.join(ROOT, "paper_2111_09512_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_values(name):
    """key = value lines of a committed ncu traffic summary under profiles/, or
    None when the kernel source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_hash") != sweep_source_hash():
        return None
    return vals


def recorded_traffic():
    """Per-launch DRAM bytes of the sweep kernel on the headline workload."""
    vals = recorded_values("k_sweep_cutcell128_ilut_traffic.txt")
    try:
        return float(vals["dram_bytes_per_sweep_launch"]) if vals else None
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        if which == 0:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((t, parts))
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.15 <= r[0] <= (self.t1 or 1e30) + 0.15]
        use = inside or rows
        if not use:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[1]) for _, p in use if num(p[1]) is not None]
        mx = [num(p[2]) for _, p in use if num(p[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, p in use:
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(use), "in_timed_region": bool(inside)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, dist, device) -> float:
    """Max of a per-rank number over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(step_bytes: int, steps: int, world: int, max_ms: float) -> float:
    """Replicas: every rank moves step_bytes per step; the job's rate is all
    ranks' bytes over the slowest rank's time."""
    return step_bytes * steps * world / (max_ms * 1e-3) / 1e9


def build_workload():
    import synth
    A = synth.cutcell7(EDGE, seed=1)
    n = len(A[0]) - 1
    b = synth.rhs(n, 1, seed=1)
    return A, b


# --------------------------------------------------------------- CPU oracle

def oracle_rate(A, b, budget_s: float):
    """Time the oracle's smoother application (single thread) on the workload;
    repeats until budget_s elapses (at least one application)."""
    import numpy as np
    import oracle
    F = oracle.ilut(A, TAU, FILL)
    S = oracle.row_scale(F)
    n = len(A[0]) - 1
    nbytes = apply_bytes(n, len(A[1]), len(S.L[1]), len(S.Us[1]), 1, 8, ML, MU)
    x0 = np.zeros((n, 1))
    reps, t = 0, 0.0
    while reps == 0 or t < budget_s:
        t0 = time.perf_counter()
        oracle.smooth(A, S, x0, b, ML, MU)
        t += time.perf_counter() - t0
        reps += 1
    return nbytes * reps / t / 1e9, reps, t


def oracle_fgmres_poisson32():
    """The oracle's FGMRES(30) to 1e-8 on the 32^3 Poisson system (ILU(0), 5+5 sweeps, first right-hand
    side of seed 0), single thread: (seconds, iterations, true relres)."""
    import oracle
    import synth
    A = synth.poisson7(32)
    n = len(A[0]) - 1
    b = synth.rhs(n, 4, seed=0)[:, 0].copy()
    S = oracle.row_scale(oracle.ilu0(A))
    t0 = time.perf_counter()
    _, st, its, rel = oracle.fgmres(A, S, b, tol=1e-8, restart=30, maxit=2000, mL=5, mU=5, precond=0)
    return time.perf_counter() - t0, its, rel


def slab_sample(nz: int):
    """A 128 x 128 x nz slab of the same cut-cell generator: the same rows,
    couplings and bandwidth as the full workload, fewer planes."""
    import synth
    A = synth.cutcell7(EDGE, EDGE, nz, seed=1)
    n = len(A[0]) - 1
    return A, synth.rhs(n, 1, seed=1)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.build()
    total_steps = args.steps + args.warmup
    # size the per-step sample so the whole run stays within ~150 s
    per_step_budget = min(2.0, 150.0 / max(total_steps, 1))
    As, bs = slab_sample(8)
    Fs = oracle.row_scale(oracle.ilut(As, TAU, FILL))
    t0 = time.perf_counter()
    oracle.smooth(As, Fs, np.zeros_like(bs), bs, ML, MU)
    t8 = time.perf_counter() - t0
    nz = int(max(1, min(EDGE, 8 * per_step_budget / max(t8, 1e-6))))
    A, b = slab_sample(nz)
    S = oracle.row_scale(oracle.ilut(A, TAU, FILL))
    n = len(A[0]) - 1
    nbytes = apply_bytes(n, len(A[1]), len(S.L[1]), len(S.Us[1]), 1, 8, ML, MU)
    x0 = np.zeros((n, 1))
    for _ in range(args.warmup):
        oracle.smooth(A, S, x0, b, ML, MU)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.smooth(A, S, x0, b, ML, MU)
    dt = time.perf_counter() - t0
    value = nbytes * args.steps / dt / 1e9
    sample = f"128x128x{nz} slab of the cut-cell generator ({n} rows), ILUT(1e-3,10), 10+10 sweeps per step"
    line = {
        "impl": "reference", "metric": "Richardson ILU-apply GB/s", "value": round(value, 3), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * dt / max(args.steps, 1), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample, "l2": "oracle runs on host cores"},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm

def run_silu(args):
    import numpy as np
    import torch
    import paper_2111_09512_gb300 as silu

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    silu.build()
    stream = torch.cuda.current_stream()
    ctx = silu.Context(local, stream)

    A, b_np = build_workload()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", TAU, FILL)
    st = F.stats()
    nnzA, nnzL, nnzU = len(A[1]), st["nnz_L"], st["nnz_U"]
    step_bytes = apply_bytes(n, nnzA, nnzL, nnzU, 1, 8, ML, MU)
    F.reserve(1, 30)
    b = torch.from_numpy(b_np).cuda()
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")

    for _ in range(args.warmup):
        x.zero_()
        silu.ilu_smooth(F, x, b, ML, MU)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark(0)
    e0.record(stream)
    for _ in range(args.steps):
        silu.ilu_smooth(F, x, b, ML, MU)
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(1)
    ctx.profile(False)
    if dist:
        dist.barrier()
    launches = ctx.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    clocks = sampler.stop()
    ms = reduce_max(ms, dist, "cuda")
    value = whole_job_gbs(step_bytes, args.steps, world, ms)

    # roofline of the dominant kernel: the sweep SpMV (L_s and Utilde_s)
    nL, msL = prof["sweep_L"]
    nU, msU = prof["sweep_U"]
    sw_bytes = nL * sweep_bytes(n, nnzL, 1, 8) + nU * sweep_bytes(n, nnzU, 1, 8)
    achieved = sw_bytes / ((msL + msU) * 1e-3) / 1e9 if msL + msU > 0 else None
    peak, peak_kind = load_peaks()
    traffic = recorded_traffic()
    total_prof_ms = sum(v[1] for v in prof.values())
    # the FP64 pipe, the sweeps' other bound: with one lane per row a tile costs as many warp-wide FMAs as
    # its longest row has entries (silu_ilu_layout's slots per entry); GB300 retires 2 FP64 lanes per clock
    # per SM
    padL, padU = (float(v) for v in F.layout()["pad_natural"])
    slots = nL * nnzL * padL + nU * nnzU * padU
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp64_peak = sms * 2 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    fp64_rate = slots / ((msL + msU) * 1e-3) if msL + msU > 0 else None

    # end to end through the public API with host buffers, copies inside the region: every step uploads
    # its x and b from pinned host memory, applies the smoother and reads x back.  Steps are independent
    # applications, so x and b are double-buffered on the device and the uploads of step k+1 (one copy
    # stream) and the readback of step k (another) overlap the smoother of step k on the library's stream.
    xh_in = torch.zeros(n, 1, dtype=torch.float64).pin_memory()
    bh = torch.from_numpy(b_np.copy()).pin_memory()
    xo = [torch.empty(n, 1, dtype=torch.float64).pin_memory() for _ in range(2)]
    xd = [torch.empty(n, 1, dtype=torch.float64, device="cuda") for _ in range(2)]
    bd = [torch.empty(n, 1, dtype=torch.float64, device="cuda") for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(steps):
        e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_start.record(stream)

        def upload(k):
            buf = k % 2
            s_in.wait_event(e_start)
            if k >= 2:
                s_in.wait_event(ev_out[buf])  # step k-2 has read xd[buf] back (after its smoother)
            with torch.cuda.stream(s_in):
                xd[buf].copy_(xh_in, non_blocking=True)
                bd[buf].copy_(bh, non_blocking=True)
                ev_in[buf].record(s_in)

        upload(0)
        for k in range(steps):
            buf = k % 2
            if k + 1 < steps:
                upload(k + 1)
            stream.wait_event(ev_in[buf])
            silu.ilu_smooth(F, xd[buf], bd[buf], ML, MU)
            ev_comp[buf].record(stream)
            s_out.wait_event(ev_comp[buf])
            with torch.cuda.stream(s_out):
                xo[buf].copy_(xd[buf], non_blocking=True)
                ev_out[buf].record(s_out)
        stream.wait_event(ev_out[(steps - 1) % 2])
        if steps > 1:
            stream.wait_event(ev_out[(steps - 2) % 2])
        e_end.record(stream)
        torch.cuda.synchronize()
        return e_start.elapsed_time(e_end)

    e2e_run(3)
    ms_e2e = e2e_run(args.steps)
    ms_e2e = reduce_max(ms_e2e, dist, "cuda")
    e2e = whole_job_gbs(step_bytes, args.steps, world, ms_e2e)
    e2e_ok = bool(torch.equal(xo[(args.steps - 1) % 2], xo[args.steps % 2])) if args.steps > 1 else True

    solve = None
    if not args.no_solve and rank == 0:
        solve = solve_comparison(silu, ctx, torch, args.solve_edge)

    batch = None
    if not args.no_batch and rank == 0:
        batch = batch_workload(silu, ctx, torch, args.batch_count)

    serve = None
    if not args.no_serve and rank == 0:
        serve = serving(silu, args)

    amg = amg_comparison(silu, ctx, torch, args.amg_edge) if (args.amg_edge > 0 and rank == 0) else None
    place = (smoother_placement(silu, ctx, torch, args.placement_edge)
             if (args.placement_edge > 0 and rank == 0) else None)

    p32 = poisson32(silu, ctx, torch) if rank == 0 else None
    mrhs = multi_rhs(silu, ctx, torch, F, n, nnzA, nnzL, nnzU) if rank == 0 else None
    f32err = fp32_error(silu, ctx, torch) if rank == 0 else None
    study = None
    if rank == 0 and args.study:
        study = sweep_study(silu, ctx, torch)
    elif rank == 0 and not args.no_scaling_study:
        study = {"scaling": scaling_study(silu, ctx, torch), "nrbe_amg": nrbe_amg_study(silu, ctx, torch)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gbs, reps, t = oracle_rate(A, b_np, args.cpu_budget)
        cpu = {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{reps} full application(s) of the 128^3 workload, {t:.1f} s, single thread"}
        fs, fits, frel = oracle_fgmres_poisson32()
        cpu["fgmres_poisson32"] = {"seconds": round(fs, 4), "iterations": fits, "relres": frel,
                                   "what": "oracle FGMRES(30) to 1e-8, 32^3 Poisson ILU(0), 5+5 sweeps, one thread"}

    if rank == 0:
        line = {
            "metric": "Richardson ILU-apply GB/s", "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": n, "nnz_A": nnzA, "nnz_L": nnzL, "nnz_U": nnzU,
                       "bytes_per_step": step_bytes, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (factors + A = %.0f MB > 129 MB)"
                             % ((nnzA * 12 + (nnzL + nnzU) * 12) / 1e6)},
            "hbm_frac_of_" + peak_kind: round(value / world / peak, 4),
            "roofline": {"bound": "hbm", "kernel": "k_sweep (Richardson sweep SpMV on L_s / Utilde_s)",
                         "achieved": round(achieved, 2) if achieved else None, "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4) if achieved else None, "peak_kind": peak_kind,
                         "traffic": traffic, "launches": nL + nU,
                         # consecutive sweeps reuse what L2 holds, so DRAM moves less than the algorithmic
                         # bytes: the DRAM rate is the recorded per-launch traffic over the same mean duration
                         "dram_achieved": round(traffic / ((msL + msU) * 1e-3 / (nL + nU)) / 1e9, 2)
                         if (traffic and msL + msU > 0) else None,
                         "dram_frac": round(traffic / ((msL + msU) * 1e-3 / (nL + nU)) / 1e9 / peak, 4)
                         if (traffic and msL + msU > 0) else None,
                         "share_of_timed_kernels": round((msL + msU) / total_prof_ms, 4) if total_prof_ms else None,
                         "fp64": {"fma_slots_per_entry": [round(padL, 4), round(padU, 4)],
                                  "achieved_gfma_s": round(fp64_rate / 1e9, 1) if fp64_rate else None,
                                  "peak_gfma_s": round(fp64_peak / 1e9, 1),
                                  "frac": round(fp64_rate / fp64_peak, 4) if fp64_rate else None,
                                  "peak_basis": f"2 FP64 lanes per clock per SM x {sms} SMs x max SM clock"}},
            "kernel_ms": {k: [v[0], round(v[1], 4)] for k, v in prof.items() if v[0]},
            "e2e": {"value": round(e2e, 2), "unit": "GB/s", "h2d_bytes_per_step": 2 * n * 8,
                    "d2h_bytes_per_step": n * 8, "ms_per_step": round(ms_e2e / args.steps, 5),
                    "pipelined": "x, b double-buffered; uploads of step k+1 and readback of step k overlap step k",
                    "last_two_results_equal": e2e_ok},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if solve:
            line["solve"] = solve
        if batch:
            line["batch"] = batch
        if serve:
            line["serving"] = serve
        if amg:
            line["amg"] = amg
        if place:
            line["smoother_placement"] = place
        if p32:
            line["poisson32"] = p32
        if mrhs:
            line["multi_rhs"] = mrhs
        if f32err:
            line["fp32_error"] = f32err
        if study:
            line["sweep_study"] = study
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def class_split(ctx, torch, fn, reps: int, cls_bytes: dict) -> dict:
    """Run fn() reps times with the library's event timing on and return, per
    kernel class, launches, total ms and (for the classes in cls_bytes, bytes
    per launch) the algorithmic GB/s.  Runs of consecutive sweeps are timed as
    one record, so gaps inside a run count."""
    ctx.profile(True)
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    split = {}
    for k, (cnt, kms) in prof.items():
        if cnt:
            split[k] = {"launches": cnt, "ms": round(kms, 4)}
            if k in cls_bytes and kms > 0:
                split[k]["gbs"] = round(cnt * cls_bytes[k] / (kms * 1e-3) / 1e9, 1)
    return split


def solve_comparison(silu, ctx, torch, edge: int):
    """The 27-point workload: FGMRES(30) to 1e-10 relative residual with the
    FP32 scaled-ILU(0) Richardson smoother (3+3 FP32 sweeps, FP64 residual and
    Krylov) against FGMRES(30) with FP64 exact triangular solves of the same
    factors (the faster of the persistent and the per-level schedule), on the 27-point perturbed-hex Laplacian
    (edge^3 rows; 256^3 = 16.8M rows, 449M entries).  Also the FP32 smoother
    application's algorithmic GB/s."""
    import synth
    A = synth.hex27(edge, seed=2)
    n = len(A[0]) - 1
    b_np = synth.rhs(n, 1, seed=2)
    t0 = time.perf_counter()
    M = silu.Matrix(ctx, *A)
    F = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP32)
    setup_s = time.perf_counter() - t0
    # launch shape of the FP64 products with A (residual, FGMRES), timed on A; both paths below use it
    a_shape, a_ms = M.autotune()
    st = F.stats()
    F.reserve(1, 30)
    out = {"workload": f"hex27-{edge}^3 ILU(0)", "rows": n, "nnz_A": len(A[1]), "tol": 1e-10, "restart": 30,
           "setup_s": round(setup_s, 2), "a_shape": {"lanes": a_shape[0], "rows_per_lane": a_shape[1],
                                                      "chunk": a_shape[2], "residual_ms": round(a_ms, 4)}}
    del A
    b = torch.from_numpy(b_np[:, 0].copy()).cuda()
    # FP32 smoother application rate (x != 0 after the first application, so the FP64 residual runs)
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    b2 = b.reshape(n, 1)
    for _ in range(3):
        silu.ilu_smooth(F, x, b2, 3, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record()
    for _ in range(reps):
        silu.ilu_smooth(F, x, b2, 3, 3)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = apply_bytes(n, out["nnz_A"], st["nnz_L"], st["nnz_U"], 1, 4, 3, 3)
    split = class_split(ctx, torch, lambda: silu.ilu_smooth(F, x, b2, 3, 3), reps,
                        {"residual": resid_bytes(n, out["nnz_A"], 1), "sweep_L": sweep_bytes(n, st["nnz_L"], 1, 4),
                         "sweep_U": sweep_bytes(n, st["nnz_U"], 1, 4)})
    out["fp32_apply"] = {"ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1), "bytes": nbytes,
                         "kernels": split}
    # fraction of the measured HBM bandwidth by DRAM bytes: the recorded per-launch traffic of this
    # workload's sweeps (full size, live L2 state) over this run's mean launch durations
    rec = recorded_values("k_sweep_hex27_256_fp32_traffic.txt") if edge == 256 else None
    if rec:
        peak, kind = load_peaks()
        dram = {}
        for cls, key in (("sweep_L", "dram_bytes_per_L_sweep"), ("sweep_U", "dram_bytes_per_U_sweep"),
                         ("residual", "dram_bytes_per_residual")):
            if cls in split and key in rec and split[cls]["ms"] > 0:
                per = split[cls]["ms"] / split[cls]["launches"] * 1e-3
                gbs = float(rec[key]) / per / 1e9
                dram[cls] = {"dram_gbs": round(gbs, 1), "dram_frac": round(gbs / peak, 4)}
        out["fp32_apply"]["dram"] = dram
        out["fp32_apply"]["dram_peak"] = {"gbs": peak, "kind": kind}
    for name, pc in (("fp32_sweeps_3_3", silu.PRECOND_SWEEPS), ("fp64_direct", silu.PRECOND_DIRECT)):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        # one restart cycle first: every inner iteration's graph is captured before the timed solve
        silu.fgmres_solve(F, x, b, tol=1e-10, restart=30, maxit=30, sweeps_L=3, sweeps_U=3, precond=pc)
        x.zero_()
        torch.cuda.synchronize()
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        sampler.mark(0)
        t0 = time.perf_counter()
        stt, its, rel = silu.fgmres_solve(F, x, b, tol=1e-10, restart=30, maxit=3000, sweeps_L=3, sweeps_U=3,
                                          precond=pc)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sampler.mark(1)
        out[name] = {"seconds": round(dt, 4), "iterations": its, "relres": rel, "converged": stt == silu.OK,
                     "clocks": sampler.stop()}
    if out["fp32_sweeps_3_3"]["seconds"] > 0:
        out["speedup_sweeps_vs_direct"] = round(out["fp64_direct"]["seconds"] / out["fp32_sweeps_3_3"]["seconds"], 3)
    del F
    return out


def batch_workload(silu, ctx, torch, count: int):
    """512 independent cut-cell 7-point systems with edges uniform in [8, 64]
    (512 to 262,144 rows each), FP32 ILU(0) factors packed block-diagonally:
    setup time, autotuned launch shape, batched smoother GB/s (3+3 sweeps),
    and the batched FGMRES(20) (one Krylov process per system) to 1e-8."""
    import numpy as np
    import synth
    edges = synth.randint(3, 0, count, 8, 64)
    systems = [synth.cutcell7(int(e), seed=10_000 + k) for k, e in enumerate(edges)]
    nnzA = sum(len(A[1]) for A in systems)
    t0 = time.perf_counter()
    B = silu.Batch(ctx, systems, "ilu0", prec=silu.FP32)
    setup_s = time.perf_counter() - t0
    del systems
    st = B.factors.stats()
    n = B.n
    choice, tune_ms = B.factors.autotune(3, 3)
    b = torch.from_numpy(synth.rhs(n, 1, seed=3)[:, 0].copy()).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        silu.silu_batch_smooth(B, x, b, 3, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record()
    for _ in range(reps):
        silu.silu_batch_smooth(B, x, b, 3, 3)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = apply_bytes(n, nnzA, st["nnz_L"], st["nnz_U"], 1, 4, 3, 3)
    # per-kernel-class split of the same loop
    split = class_split(ctx, torch, lambda: silu.silu_batch_smooth(B, x, b, 3, 3), reps,
                        {"residual": resid_bytes(n, nnzA, 1), "sweep_L": sweep_bytes(n, st["nnz_L"], 1, 4),
                         "sweep_U": sweep_bytes(n, st["nnz_U"], 1, 4)})
    x.zero_()
    silu.silu_batch_fgmres(B, x, b, tol=1e-8, restart=20, maxit=20, sweeps_L=3, sweeps_U=3)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stt, its, rel = silu.silu_batch_fgmres(B, x, b, tol=1e-8, restart=20, maxit=5000, sweeps_L=3, sweeps_U=3)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    out = {"workload": f"{count} cut-cell 7-point systems, edges U[8,64], FP32 ILU(0)", "rows": n,
           "nnz_A": nnzA, "setup_s": round(setup_s, 2), "autotune_choice": choice,
           "smooth_3_3": {"ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1), "kernels": split},
           "fgmres20_1e-8": {"seconds": round(solve_s, 4), "all_converged": stt == silu.OK,
                             "iterations_max": int(np.max(its)), "iterations_mean": round(float(np.mean(its)), 1),
                             "relres_max": float(np.max(rel))}}
    # the same solves with 5+5 sweeps (fewer, dearer iterations)
    x.zero_()
    silu.silu_batch_fgmres(B, x, b, tol=1e-8, restart=20, maxit=20, sweeps_L=5, sweeps_U=5)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stt, its, rel = silu.silu_batch_fgmres(B, x, b, tol=1e-8, restart=20, maxit=5000, sweeps_L=5, sweeps_U=5)
    torch.cuda.synchronize()
    out["fgmres20_1e-8_sweeps_5_5"] = {"seconds": round(time.perf_counter() - t0, 4), "all_converged": stt == silu.OK,
                                       "iterations_max": int(np.max(its)),
                                       "iterations_mean": round(float(np.mean(its)), 1),
                                       "relres_max": float(np.max(rel))}
    B.close()
    return out


def serve_pool(args):
    """The pool of distinct systems the serving client draws matrices from
    (generated before any clock starts): args.serve_pool cut-cell matrices
    with edges log-uniform in [16, 192] (seed 4), each with its right-hand side."""
    import numpy as np
    import synth
    P = args.serve_pool
    ue = synth.uniform(4, 6, P, 0.0, 1.0)
    edges = np.rint(np.exp(np.log(16.0) + ue * (np.log(192.0) - np.log(16.0)))).astype(int)
    pool = []
    for k, e in enumerate(edges):
        A = synth.cutcell7(int(e), seed=40_000 + k)
        pool.append((A, synth.rhs(int(e) ** 3, 1, seed=50_000 + k)[:, 0]))
    return edges, pool


def serve_stream(silu, pool, arrivals, path, workers, max_queue):
    """Offer the arrival stream to a fresh server on one path; per-request
    latency is completion minus submission on the server's clock."""
    import numpy as np
    prec, pc, sw = path
    P = len(pool)
    S = silu.Server(0, 120 << 30, workers=workers, max_queue=max_queue)
    tickets, refused = [], 0
    start = time.perf_counter()
    for k, t_k in enumerate(arrivals):
        now = time.perf_counter() - start
        if now < t_k:
            time.sleep(t_k - now)
        A, b = pool[k % P]
        st, t = S.submit(A, b, prec=prec, tol=1e-8, restart=30, maxit=20000, sweeps_L=sw, sweeps_U=sw, precond=pc)
        if st == silu.OK:
            tickets.append(t)
        else:
            refused += 1
    lat, solved, iters, t_first, t_last, setup = [], 0, [], None, None, []
    for t in tickets:
        _, res, _ = S.poll(t, wait=True, want_x=False)
        if res.status == silu.OK:
            solved += 1
            lat.append(res.t_done - res.t_submit)
            iters.append(res.iterations)
            setup.append(res.t_setup_done - res.t_admit)
            t_first = res.t_submit if t_first is None else min(t_first, res.t_submit)
            t_last = res.t_done if t_last is None else max(t_last, res.t_done)
    S.close()
    span = (t_last - t_first) if solved else 0.0
    offered = len(arrivals)
    return {"offered": offered, "admitted": len(tickets), "refused": refused,
            "refused_fraction": round(refused / offered, 4) if offered else None, "solved": solved,
            "goodput_solves_per_s": round(solved / span, 3) if span > 0 else None,
            "p50_s": round(float(np.percentile(lat, 50)), 4) if lat else None,
            "p99_s": round(float(np.percentile(lat, 99)), 4) if lat else None,
            "max_s": round(float(np.max(lat)), 4) if lat else None,
            "iterations_mean": round(float(np.mean(iters)), 1) if iters else None,
            "host_setup_mean_s": round(float(np.mean(setup)), 3) if setup else None}


def poisson_arrivals(rate, count, seed_stream):
    """count exponential inter-arrival times of mean 1/rate (counter-based
    uniforms of the given stream), as absolute offsets in seconds."""
    import numpy as np
    import synth
    gaps = -np.log1p(-synth.uniform(4, seed_stream, count, 0.0, 1.0)) / rate
    return np.cumsum(gaps)


def serving(silu, args):
    """Continuous-batching solve server (cut-cell pressure solves with grid
    edges log-uniform in [16, 192], each FGMRES(30) from zero to 1e-8, under
    a 120 GB HBM budget), two runs.

    offered: the stream of the workload's definition, Poisson arrivals at
    args.serve_rate per second (200; seed 4) until args.serve_requests
    requests (1000) have been offered, on three paths: the FP32 scaled-ILU(0)
    Richardson smoother with 3+3 sweeps (the default) and with 5+5 sweeps
    (about the fewest sweeps that bring FGMRES to the iteration count of exact
    solves on these matrices), and the plain FP64 direct-trisolve path.  One
    GPU serves a few solves of ~1M rows per second, so this stream saturates
    it: the server admits what its slots and queue hold and refuses the rest;
    the run reports the refused fraction, the goodput and the latency of the
    admitted requests (queue-bound).

    sustained: Poisson arrivals at args.serve_low_rate per second (below what
    one GPU serves on either path) for args.serve_low_seconds, FP32 5+5 sweeps
    against FP64 direct, with a queue long enough that nothing is refused, so
    p50/p99 are latencies of a server that keeps up.

    The client draws every request's edge from the stream but takes its
    matrix from a pool of args.serve_pool distinct systems generated before
    the clock starts (request k uses pool entry k mod pool), so submission is
    never held up by generation."""
    import numpy as np
    edges, pool = serve_pool(args)
    out = {"workload": "cut-cell 7-point solves, edges log-uniform [16,192], FGMRES(30) to 1e-8",
           "pool": args.serve_pool, "pool_rows_mean": int(np.mean(edges.astype(np.int64) ** 3)),
           "hbm_budget_gb": 120, "workers": args.serve_workers}
    paths = {"fp32_sweeps_3_3": (silu.FP32, silu.PRECOND_SWEEPS, 3),
             "fp32_sweeps_5_5": (silu.FP32, silu.PRECOND_SWEEPS, 5),
             "fp64_direct": (silu.FP64, silu.PRECOND_DIRECT, 3)}
    arr = poisson_arrivals(args.serve_rate, args.serve_requests, 5)
    off = {"rate_per_s": args.serve_rate, "requests": args.serve_requests,
           "seconds_of_arrivals": round(float(arr[-1]), 3), "max_queue": args.serve_queue}
    for name, path in paths.items():
        off[name] = serve_stream(silu, pool, arr, path, args.serve_workers, args.serve_queue)
    out["offered"] = off
    if args.serve_low_seconds > 0:
        low = poisson_arrivals(args.serve_low_rate, int(args.serve_low_rate * args.serve_low_seconds * 3) + 16, 7)
        low = low[low < args.serve_low_seconds]
        sus = {"rate_per_s": args.serve_low_rate, "seconds_of_arrivals": args.serve_low_seconds,
               "max_queue": len(low)}
        for name in ("fp32_sweeps_5_5", "fp64_direct"):
            sus[name] = serve_stream(silu, pool, low, paths[name], args.serve_workers, len(low))
        out["sustained"] = sus
    return out


def amg_comparison(silu, ctx, torch, edge: int):
    """GMRES + AMG, the paper's solver configuration (Sec. 3, Sec. 6): the
    cut-cell 7-point matrix on edge^3 (seed 1; 224^3 = 11.2M rows, the size of
    the paper's 11M-row PeleLM system), one right-hand side U[-1,1) (seed 1),
    FP64 ILU(0) factors smoothing the finest level of a Ruge-Stueben
    hierarchy (theta 0.25, coarsest <= 400 rows, one l1-Jacobi sweep before
    and after each coarser correction).  FGMRES(30) to 1e-8 with one V-cycle
    as the preconditioner, the finest level smoothed by m + m Richardson
    sweeps (m = 3, 5, 10; the paper reports 20 SpMVs as sufficient at 11M rows
    and fewer as insufficient) against the same cycle smoothed by exact
    level-scheduled triangular solves (the comparison behind the paper's
    GMRES + AMG gains), the single-level 3+3-sweep smoother for reference,
    and the cycle with FP32 factors and sweeps on the finest level.  Also one
    V-cycle's time alone."""
    import synth
    A = synth.cutcell7(edge, seed=1)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    a_shape, _ = M.autotune()  # launch shape of the products with A, used by every path below
    F = silu.ilu_setup(ctx, M, "ilu0")
    t0 = time.perf_counter()
    F.amg_setup(theta=0.25, max_levels=25, coarse_size=400, jacobi_sweeps=1)
    setup_s = time.perf_counter() - t0
    st = F.amg_stats()
    st_f = F.stats()
    out = {"workload": f"cutcell7-{edge}^3 ILU(0) FP64 + AMG", "rows": n, "nnz_A": len(A[1]),
           "amg_setup_s": round(setup_s, 2), "levels": st["levels"], "level_rows": st["rows"],
           "operator_complexity": round(sum(st["nnz_A"]) / st["nnz_A"][0], 3),
           "ilu_levels": [st_f["levels_L"], st_f["levels_U"]], "tol": 1e-8, "restart": 30, "maxit": 600,
           "a_shape": {"lanes": a_shape[0], "rows_per_lane": a_shape[1], "chunk": a_shape[2]}}
    b = torch.from_numpy(synth.rhs(n, 1, seed=1)[:, 0].copy()).cuda()
    F.reserve(1, 30)
    peak_gbs, _ = load_peaks()
    for label, sL, sU in (("vcycle_sweeps_10_10_ms", 10, 10), ("vcycle_direct_ms", -1, -1)):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        for _ in range(3):
            F.amg_vcycle(x, b, sL, sU)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            F.amg_vcycle(x, b, sL, sU)
        e1.record()
        torch.cuda.synchronize()
        out[label] = round(e0.elapsed_time(e1) / 10, 3)
    # Sec. 6.3's V-cycle model in kind: the cycle's algorithmic bytes over the measured HBM bandwidth,
    # against the measured cycle (the paper assumes CSR reads at 2/3 of peak)
    vb = vcycle_bytes(st, st_f["nnz_L"], st_f["nnz_U"], 10, 10, 1)
    ms_model = vb / (peak_gbs * 1e9) * 1e3
    out["vcycle_model_10_10"] = {"bytes": int(vb), "ms_at_measured_peak": round(ms_model, 3),
                                 "ms_at_two_thirds_of_peak": round(1.5 * ms_model, 3),
                                 "measured_ms": out["vcycle_sweeps_10_10_ms"],
                                 "fraction_of_peak": round(ms_model / out["vcycle_sweeps_10_10_ms"], 3)}
    runs = [("amg_direct", silu.PRECOND_AMG_DIRECT, 0, 0)]
    runs += [(f"amg_sweeps_{m}_{m}", silu.PRECOND_AMG, m, m) for m in (3, 5, 10)]
    runs += [("single_level_sweeps_3_3", silu.PRECOND_SWEEPS, 3, 3)]
    for label, pre, mL, mU in runs:
        for rep in range(2):  # the first solve also captures the iteration graphs
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            status, its, rr = silu.fgmres_solve(F, x, b, tol=1e-8, restart=30, maxit=600 if pre != silu.PRECOND_SWEEPS
                                                else 5000, sweeps_L=mL, sweeps_U=mU, precond=pre)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            if status != silu.OK:
                break  # a stalled configuration is reported once
        out[label] = {"seconds": round(sec, 4), "iterations": its, "relres": float(f"{rr:.3e}"),
                      "converged": status == silu.OK}
    # the same cycle with FP32 factors and FP32 sweeps on the finest level (FP64 elsewhere)
    del F
    F32 = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP32)
    F32.amg_setup(theta=0.25, max_levels=25, coarse_size=400, jacobi_sweeps=1)
    F32.reserve(1, 30)
    for m in (5, 10):
        for rep in range(2):
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            status, its, rr = silu.fgmres_solve(F32, x, b, tol=1e-8, restart=30, maxit=600, sweeps_L=m, sweeps_U=m,
                                                precond=silu.PRECOND_AMG)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
        out[f"amg_fp32_sweeps_{m}_{m}"] = {"seconds": round(sec, 4), "iterations": its, "relres": float(f"{rr:.3e}"),
                                           "converged": status == silu.OK}
    del F32
    best = min((v["seconds"], k) for k, v in out.items()
               if k.startswith(("amg_sweeps", "amg_fp32")) and isinstance(v, dict) and v["converged"])
    out["fastest_amg_sweeps"] = best[1]
    out["speedup_amg_sweeps_vs_amg_direct"] = round(out["amg_direct"]["seconds"] / best[0], 2)
    return out


def smoother_placement(silu, ctx, torch, edge: int, sweeps=(5, 10)):
    """Where the ILU smoother sits in the V-cycle (Sec. 6, Fig. multi-level-ilu:
    ILU on the finest level only, ILU on all levels, polynomial Gauss-Seidel):
    the cut-cell 7-point matrix on edge^3 (seed 1), FP64, one right-hand side
    (seed 1), Ruge-Stueben hierarchy (theta 0.25, coarsest <= 400 rows),
    FGMRES(30) to 1e-8 from zero with one V-cycle as the preconditioner.
      ilu_finest_jacobi_m: ILU(0) on the finest level (m + m sweeps), one
                           l1-Jacobi step before and after below;
      ilu_finest_gs_m:     the same with one polynomial Gauss-Seidel step (two
                           terms) below (the paper's mixed V-cycle);
      ilu_all_levels_m:    ILU(0) factors of every A_l above the coarsest,
                           each swept m + m times;
      gs_all_levels:       polynomial Gauss-Seidel (two terms) on every level,
                           the finest one included.
    Each with its V-cycle's time (CUDA events over 10 cycles) and the host
    setup of the hierarchy (and of the coarse factors)."""
    import synth
    A = synth.cutcell7(edge, seed=1)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    del A
    b = torch.from_numpy(synth.rhs(n, 1, seed=1)[:, 0].copy()).cuda()
    out = {"workload": f"cutcell7-{edge}^3 FP64, FGMRES(30) to 1e-8 from x = 0, one V-cycle per iteration",
           "rows": n}

    def run(F, mL, mU):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        for _ in range(3):
            F.amg_vcycle(x, b, mL, mU)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            F.amg_vcycle(x, b, mL, mU)
        e1.record()
        torch.cuda.synchronize()
        rec = {"vcycle_ms": round(e0.elapsed_time(e1) / 10, 3)}
        for rep in range(2):  # the first solve also captures the iteration graphs
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, its, rr = silu.fgmres_solve(F, x, b, tol=1e-8, restart=30, maxit=600, sweeps_L=mL, sweeps_U=mU,
                                            precond=silu.PRECOND_AMG)
            torch.cuda.synchronize()
            rec.update({"seconds": round(time.perf_counter() - t0, 4), "iterations": its,
                        "relres": float(f"{rr:.3e}"), "converged": st == silu.OK})
            if st != silu.OK:
                break
        return rec

    F = silu.ilu_setup(ctx, M, "ilu0")
    for label, coarse, nilu in (("ilu_finest_jacobi", silu.AMG_L1_JACOBI, 1), ("ilu_finest_gs", silu.AMG_POLY_GS, 1),
                                ("ilu_all_levels", silu.AMG_L1_JACOBI, 25)):
        t0 = time.perf_counter()
        F.amg_setup(theta=0.25, max_levels=25, coarse_size=400, jacobi_sweeps=1, coarse_smoother=coarse, gs_terms=2,
                    ilu_levels=nilu)
        setup_s = round(time.perf_counter() - t0, 2)
        out.setdefault("levels", F.amg_stats()["levels"])
        for m in sweeps:
            out[f"{label}_{m}"] = dict(run(F, m, m), amg_setup_s=setup_s)
    del F
    G = silu.ilu_setup(ctx, M, "gs")
    t0 = time.perf_counter()
    G.amg_setup(theta=0.25, max_levels=25, coarse_size=400, jacobi_sweeps=1, coarse_smoother=silu.AMG_POLY_GS,
                gs_terms=2)
    setup_s = round(time.perf_counter() - t0, 2)
    out["gs_all_levels"] = dict(run(G, 2, 1), amg_setup_s=setup_s)  # L_s = L D^{-1}: two terms, U = D
    del G
    return out


def fp32_error(silu, ctx, torch):
    """FP32 factors and sweeps against FP64 ones on the 128^3 cut-cell matrix
    (ILU(0), one right-hand side, seed 1): relative 2-norm difference of one
    smoother application from zero (3+3 and 10+10 sweeps), and FGMRES(30) to
    1e-8 with either (iterations, true relative residual)."""
    import synth
    A = synth.cutcell7(EDGE, seed=1)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    b = torch.from_numpy(synth.rhs(n, 1, seed=1)).cuda()
    F64 = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP64)
    F32 = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP32)
    out = {"workload": "cutcell7-128^3 ILU(0), FP32 vs FP64 factors and sweeps"}
    for m in (3, 10):
        x64 = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
        x32 = torch.zeros_like(x64)
        silu.ilu_smooth(F64, x64, b, m, m)
        silu.ilu_smooth(F32, x32, b, m, m)
        out[f"apply_{m}_{m}_relerr"] = float(f"{float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64)):.3e}")
    for name, F in (("fgmres_fp64", F64), ("fgmres_fp32", F32)):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(F, x, b[:, 0].contiguous(), tol=1e-8, restart=30, maxit=5000,
                                         sweeps_L=3, sweeps_U=3)
        out[name] = {"iterations": its, "relres": float(f"{rel:.3e}"), "converged": st == silu.OK}
    return out


def multi_rhs(silu, ctx, torch, F, n, nnzA, nnzL, nnzU):
    """The headline factors with 4 interleaved right-hand sides (seed 5): one
    10+10 application reads each factor once per sweep for all four columns
    (the FP64 pipe bounds it: 4 FMAs per stored entry); time per application
    and per column against one column."""
    import synth
    out = {"workload": WORKLOAD.replace("1 RHS", "4 RHS")}
    for R in (1, 4):
        b = torch.from_numpy(synth.rhs(n, R, seed=5)).cuda()
        x = torch.zeros(n, R, dtype=torch.float64, device="cuda")
        for _ in range(3):
            silu.ilu_smooth(F, x, b, ML, MU)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            silu.ilu_smooth(F, x, b, ML, MU)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        nbytes = apply_bytes(n, nnzA, nnzL, nnzU, R, 8, ML, MU)
        out[f"rhs_{R}"] = {"ms": round(ms, 4), "ms_per_column": round(ms / R, 4),
                           "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1)}
    return out


def poisson32(silu, ctx, torch):
    """7-point Poisson 32^3 (32,768 rows), ILU(0), 4 interleaved right-hand
    sides U[-1,1] (seed 0): one smoother application (5+5 sweeps) against
    one direct level-scheduled application.  L2-resident, so reported as time
    and GB/s only, not as a fraction of HBM."""
    import synth
    A = synth.poisson7(32)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    st = F.stats()
    F.reserve(4, 0)
    b = torch.from_numpy(synth.rhs(n, 4, seed=0)).cuda()
    x = torch.zeros(n, 4, dtype=torch.float64, device="cuda")
    out = {"workload": "poisson7-32^3 ILU(0), 4 RHS", "levels": st["levels_L"]}
    nbytes = apply_bytes(n, len(A[1]), st["nnz_L"], st["nnz_U"], 4, 8, 5, 5)
    for name, fn in (("smooth_5_5", lambda: silu.ilu_smooth(F, x, b, 5, 5)),
                     ("direct", lambda: silu.direct_trisolve(F, x, b))):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(200):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 200
        out[name] = {"us": round(1e3 * ms, 2)}
        if name == "smooth_5_5":
            out[name]["gbs"] = round(nbytes / (ms * 1e-3) / 1e9, 1)
    out["speedup_smooth_vs_direct"] = round(out["direct"]["us"] / out["smooth_5_5"]["us"], 2)
    # FGMRES(30) to 1e-8 on the first right-hand side, 5+5 sweeps (the oracle's FGMRES on the same
    # system is timed in the CPU leg)
    b1 = b[:, 0].contiguous()
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    silu.fgmres_solve(F, x1, b1, tol=1e-8, restart=30, maxit=2000, sweeps_L=5, sweeps_U=5)
    x1.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status, its, rel = silu.fgmres_solve(F, x1, b1, tol=1e-8, restart=30, maxit=2000, sweeps_L=5, sweeps_U=5)
    torch.cuda.synchronize()
    out["fgmres_5_5"] = {"seconds": round(time.perf_counter() - t0, 4), "iterations": its, "relres": rel,
                         "converged": status == silu.OK}
    return out


def nrbe_amg_study(silu, ctx, torch, edge: int = 24):
    """Table NRBE2 in kind (Sec. 6.1): GMRES+AMG with the ILUT(1e-3, 5)
    smoother on the finest level and m + m Richardson sweeps (m = 1..5), the
    upper factor row-scaled or row/column (Ruiz) scaled, on the cut-cell
    7-point matrix of edge^3 rows (24^3 = 13,824, the size of the paper's
    smallest PeleLM system), theta 0.25, one l1-Jacobi step below, FGMRES(30)
    to 1e-9 from zero (at most 300 iterations), right-hand side U[-1,1)
    (seed 1).  Reports the iterations and the norm-wise relative backward
    error ||b - A x|| / (||b|| + ||A||_2 ||x||) (Eq. nbre) and the true relative
    residual of the result (iterations null: not converged), the
    residual and ||A||_2 computed by the library on the device (A is
    symmetric positive definite, so ||A||_2 is its largest eigenvalue: 200
    power-iteration steps)."""
    import synth
    A = synth.cutcell7(edge, seed=1)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    b = torch.from_numpy(synth.rhs(n, 1, seed=1)[:, 0].copy()).cuda()
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    v = torch.from_numpy(synth.rhs(n, 1, seed=2)[:, 0].copy()).cuda()
    w = torch.empty_like(v)
    lam = 0.0
    for _ in range(200):  # w = -A v
        M.residual(w, v / torch.linalg.norm(v), zero)
        lam = float(torch.linalg.norm(w))
        v = w.clone()
    normA = lam
    nb = float(torch.linalg.norm(b))
    sweeps = [1, 2, 3, 4, 5]
    out = {"workload": f"cutcell7-{edge}^3 ({n} rows), ILUT(1e-3, 5) + AMG, FGMRES(30) to 1e-9",
           "norm2_A": float(f"{normA:.6e}"), "sweeps": sweeps}
    for label, sc in (("row", silu.SCALE_ROW), ("rowcol", silu.SCALE_ROWCOL)):
        F = silu.ilu_setup(ctx, M, "ilut", 1e-3, 5, scale=sc)
        F.amg_setup(theta=0.25, max_levels=25, coarse_size=400, jacobi_sweeps=1)
        its_l, nrbe_l, rel_l = [], [], []
        for m in sweeps:
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st, its, rr = silu.fgmres_solve(F, x, b, tol=1e-9, restart=30, maxit=300, sweeps_L=m, sweeps_U=m,
                                            precond=silu.PRECOND_AMG)
            r = torch.empty_like(b)
            M.residual(r, x, b)
            its_l.append(its if st == silu.OK else None)
            rel_l.append(float(f"{float(torch.linalg.norm(r)) / nb:.3e}"))
            nrbe_l.append(float(f"{float(torch.linalg.norm(r)) / (nb + normA * float(torch.linalg.norm(x))):.3e}"))
        out[label] = {"iterations": its_l, "relres": rel_l, "nrbe": nrbe_l}
        del F
    return out


def scaling_study(silu, ctx, torch):
    """Scaled against unscaled factors (the paper's Sec. 6.1, Table NRBE2's
    question) on the cut-cell 128^3 matrix, ILUT(1e-3, 10), FP64, one
    right-hand side (seed 1): for m = 1..20 sweeps on each factor, one
    smoother application from zero with the row-scaled factors (the method),
    row/column (Ruiz) scaled factors, unscaled Jacobi and unscaled plain
    Richardson; reports the residual reduction ||b - A x_m|| / ||b|| and the
    distance ||x_m - x*|| / ||x*|| to the exact application x* (direct
    solves), all computed by the library on the device."""
    import synth

    def norms_of(M, x, bt):
        r = torch.empty_like(bt)
        M.residual(r, x, bt)
        return float(torch.linalg.norm(r) / torch.linalg.norm(bt))

    A = synth.cutcell7(EDGE, seed=1)
    n = len(A[0]) - 1
    bh = synth.rhs(n, 1, seed=1)
    b = torch.from_numpy(bh).cuda()
    M = silu.Matrix(ctx, *A)
    sweeps = list(range(1, 21))
    sc_out = {"workload": WORKLOAD.split(" smoother")[0], "sweeps": sweeps}
    xstar = None
    for name, sc in (("row_scaled_richardson", silu.SCALE_ROW), ("rowcol_scaled_richardson", silu.SCALE_ROWCOL),
                     ("unscaled_jacobi", silu.SCALE_NONE), ("unscaled_richardson", silu.SCALE_NONE_RICH)):
        F = silu.ilu_setup(ctx, M, "ilut", TAU, FILL, scale=sc)
        if xstar is None:
            xstar = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
            silu.direct_trisolve(F, xstar, b)
        rel, dist = [], []
        for m in sweeps:
            x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
            silu.ilu_smooth(F, x, b, m, m)
            if not bool(torch.isfinite(x).all()):
                rel.append(None)
                dist.append(None)
                continue
            rel.append(norms_of(M, x, b))
            dist.append(float(torch.linalg.norm(x - xstar) / torch.linalg.norm(xstar)))
        sc_out[name] = {"relres": [None if v is None else float(f"{v:.4e}") for v in rel],
                        "dist_to_exact": [None if v is None else float(f"{v:.4e}") for v in dist]}
        del F
    return sc_out


def sweep_study(silu, ctx, torch):
    """Sweep studies (the paper's Sec. 5.2 and Sec. 6.1 questions on synthetic
    matrices), all computed by the library on the device.

    scaling: cut-cell 128^3, ILUT(1e-3, 10), FP64, one right-hand side
    (seed 1): for m = 1..20 sweeps on each factor, one smoother application
    from zero with the row-scaled factors (the method), row/column (Ruiz)
    scaled factors, unscaled Jacobi and unscaled plain Richardson; reports
    ||b - A x_m|| / ||b|| and the distance ||x_m - x*|| / ||x*|| to the exact
    application x* (direct solves).

    kinds: the same matrix under ILU(0), ILU(1), ILUT(1e-2, 10),
    ILUT(1e-3, 10), ILUT(1e-4, 20) and the polynomial Gauss-Seidel
    splittings: relres of one application for m = 1..20, the factor sizes
    and level counts, and FGMRES(30) to 1e-8 with 3+3 sweeps against the
    direct solves (iterations, seconds).

    nilpotence: ||T_s^p||_2 for p = 1..40 (power iteration, 30 steps per p)
    on a 24^3 cut-cell matrix (13,824 rows, the size of the paper's
    14,186-row PeleLM matrix of Fig. Up), upper factor of ILUT(tau, 30) for
    tau in {1e-2, 1e-3, 1e-4} with row and with row/column scaling, and L_s;
    with the departure from normality (Eq. depB) of L, U and the scaled U
    (Table dep).

    schur: the ILUT Schur complement smoother over 8 and 64 row blocks
    (schur_study).

    time_to_solution_vs_sweeps: FGMRES(30) to 1e-8 on cut-cell matrices of
    64^3 to 160^3 rows with FP32 ILU(0) factors and m + m sweeps (m = 2..10)
    against direct solves of the same factors (iterations, seconds)."""
    import numpy as np
    import synth
    out = {}

    out["scaling"] = scaling_study(silu, ctx, torch)
    out["nrbe_amg"] = nrbe_amg_study(silu, ctx, torch)
    A = synth.cutcell7(EDGE, seed=1)
    n = len(A[0]) - 1
    bh = synth.rhs(n, 1, seed=1)
    b = torch.from_numpy(bh).cuda()
    M = silu.Matrix(ctx, *A)
    sweeps = list(range(1, 21))

    def norms_of(M, x, bt):
        r = torch.empty_like(bt)
        M.residual(r, x, bt)
        return float(torch.linalg.norm(r) / torch.linalg.norm(bt))

    kinds = [("ilu0", "ilu0", 0.0, 0), ("iluk1", "iluk", 0.0, 1), ("ilut_1e-2_10", "ilut", 1e-2, 10),
             ("ilut_1e-3_10", "ilut", 1e-3, 10), ("ilut_1e-4_20", "ilut", 1e-4, 20), ("gs", "gs", 0.0, 0),
             ("sgs", "sgs", 0.0, 0)]
    k_out = {"workload": "cutcell7-128^3 FP64, 1 RHS (seed 1)", "sweeps": sweeps,
             "fgmres": "FGMRES(30) to 1e-8 from x = 0, 3+3 sweeps vs direct solves"}
    for name, kind, tau, fill in kinds:
        t0 = time.perf_counter()
        F = silu.ilu_setup(ctx, M, kind, tau, fill)
        setup_s = time.perf_counter() - t0
        st = F.stats()
        rel = []
        for m in sweeps:
            x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
            silu.ilu_smooth(F, x, b, m, 1 if kind == "gs" else m)
            rel.append(float(f"{norms_of(M, x, b):.4e}") if bool(torch.isfinite(x).all()) else None)
        rec = {"setup_s": round(setup_s, 2), "nnz_L": st["nnz_L"], "nnz_U": st["nnz_U"],
               "levels_L": st["levels_L"], "levels_U": st["levels_U"], "relres_one_application": rel}
        for label, pre, mL, mU in (("sweeps_3_3", silu.PRECOND_SWEEPS, 3, 1 if kind == "gs" else 3),
                                   ("direct", silu.PRECOND_DIRECT, 0, 0)):
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            status, its, rr = silu.fgmres_solve(F, x, b[:, 0].contiguous(), tol=1e-8, restart=30, maxit=3000,
                                                sweeps_L=mL, sweeps_U=mU, precond=pre)
            torch.cuda.synchronize()
            rec[label] = {"seconds": round(time.perf_counter() - t0, 3), "iterations": its,
                          "relres": float(f"{rr:.3e}"), "converged": status == silu.OK}
        k_out[name] = rec
        del F
    out["kinds"] = k_out

    B = synth.cutcell7(24, seed=1)
    nb = len(B[0]) - 1
    MB = silu.Matrix(ctx, *B)
    v0 = synth.rhs(nb, 1, seed=5)[:, 0]
    P, iters = 40, 30
    nil = {"workload": "cutcell7-24^3 (13,824 rows), ILUT(tau, 30), FP64", "p": list(range(1, P + 1)),
           "iterations_per_p": iters}
    for tau in (1e-2, 1e-3, 1e-4):
        for label, sc in (("row", silu.SCALE_ROW), ("rowcol", silu.SCALE_ROWCOL)):
            F = silu.ilu_setup(ctx, MB, "ilut", tau, 30, scale=sc)
            nu = F.power_norms("U", P, iters, v0)
            below = [p + 1 for p in range(P) if nu[p] < 1.0]
            dep = F.dep()
            rec = {"norm_Us_p": [float(f"{v:.4e}") for v in nu], "first_p_below_1": below[0] if below else None,
                   "levels_U": F.stats()["levels_U"], "dep_L": float(f"{dep['L']:.4e}"),
                   "dep_U": float(f"{dep['U']:.4e}"), "dep_scaled_U": float(f"{dep['scaled']:.4e}")}
            if label == "row":
                nl = F.power_norms("L", P, iters, v0)
                rec["norm_Ls_p"] = [float(f"{v:.4e}") for v in nl]
            nil[f"ilut_{tau:g}_{label}"] = rec
            del F
    out["nilpotence"] = nil

    # time to solution against the sweep count: FP32 ILU(0) factors of cut-cell matrices, FGMRES(30) to 1e-8
    # from zero with m + m sweeps, and with direct solves of the same factors
    tts = {}
    for edge in (64, 96, 128, 160):
        A = synth.cutcell7(edge, seed=1)
        n = len(A[0]) - 1
        M = silu.Matrix(ctx, *A)
        F = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP32)
        F.reserve(1, 30)
        b = torch.from_numpy(synth.rhs(n, 1, seed=2)[:, 0].copy()).cuda()
        rec = {}
        for m in (2, 3, 4, 5, 6, 8, 10, 0):
            pc = silu.PRECOND_SWEEPS if m else silu.PRECOND_DIRECT
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            silu.fgmres_solve(F, x, b, tol=1e-8, restart=30, maxit=30, sweeps_L=m, sweeps_U=m, precond=pc)
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, its, _ = silu.fgmres_solve(F, x, b, tol=1e-8, restart=30, maxit=5000, sweeps_L=m, sweeps_U=m,
                                           precond=pc)
            torch.cuda.synchronize()
            rec[f"sweeps_{m}_{m}" if m else "direct"] = {"iterations": its,
                                                         "seconds": round(time.perf_counter() - t0, 4),
                                                         "converged": st == silu.OK}
        tts[f"cutcell7_{edge}"] = rec
        del F, M
    out["time_to_solution_vs_sweeps"] = tts
    out["schur"] = schur_study(silu, ctx, torch)
    return out


def schur_study(silu, ctx, torch, edge=EDGE, parts=(8, 64), kind="cutcell7", sweeps=(3,), maxit=3000, tau=1e-3,
                fill=10, theta=0.25):
    """The ILUT Schur complement smoother (Sec. 3.1, Eq. schur) on an edge^3
    matrix (cut-cell 7-point by default; Poisson or the 27-point perturbed
    hex), FP64, the rows split into `parts` contiguous blocks (as ranks would
    hold them): setup time, interior and interface rows, one smoother
    application (3+3 sweeps on each block's ILUT(tau, fill) factors, no
    residual of the whole system formed), and FGMRES(30) to 1e-8 from zero
    preconditioned by it (m+m sweeps for each m in `sweeps`), against the
    single-level smoother (ILUT(tau, fill), m+m sweeps) and exact solves of
    the same factors.  Then the smoother where the paper places it: on the
    finest level of the Ruge-Stueben V-cycle (strength theta, coarsest <= 400
    rows, l1-Jacobi below), against the same cycle smoothed by ILUT(tau, fill)
    sweeps on the whole finest level.  Both placements again with the
    smoother's interface iteration right-preconditioned by diag(C) (`diag_*`,
    not in the paper).  A configuration that has not converged after `maxit`
    iterations is reported once (no second, graph-replayed solve)."""
    import synth
    A = {"cutcell7": lambda: synth.cutcell7(edge, seed=1), "poisson7": lambda: synth.poisson7(edge),
         "hex27": lambda: synth.hex27(edge, seed=2)}[kind]()
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    del A
    b = torch.from_numpy(synth.rhs(n, 1, seed=1)[:, 0].copy()).cuda()
    out = {"workload": f"{kind}-{edge}^3 FP64, FGMRES(30) to 1e-8 from x = 0", "rows": n,
           "ilut": {"tau": tau, "fill": fill}, "theta": theta}

    def solve(F, pre, mL, mU):
        rec = None
        for _ in range(2):  # the first solve also captures the iteration graphs
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, its, rr = silu.fgmres_solve(F, x, b, tol=1e-8, restart=30, maxit=maxit, sweeps_L=mL, sweeps_U=mU,
                                            precond=pre)
            torch.cuda.synchronize()
            rec = {"seconds": round(time.perf_counter() - t0, 4), "iterations": its, "relres": float(f"{rr:.3e}"),
                   "converged": st == silu.OK}
            if st != silu.OK:
                break
        return rec

    def amg(F):
        t0 = time.perf_counter()
        F.amg_setup(theta=theta, max_levels=25, coarse_size=400, jacobi_sweeps=1)
        return round(time.perf_counter() - t0, 2)

    for p in parts:
        F = silu.ilu_setup(ctx, M, "ilu0")
        t0 = time.perf_counter()
        F.schur_setup(p, tau, fill)
        setup_s = time.perf_counter() - t0
        st = F.schur_stats()
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        for _ in range(3):
            F.schur_smooth(x, b, 3, 3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            F.schur_smooth(x, b, 3, 3)
        e1.record()
        torch.cuda.synchronize()
        rec = {"setup_s": round(setup_s, 2), "interior_rows": st["interior"], "interface_rows": st["interface"],
               "apply_3_3_ms": round(e0.elapsed_time(e1) / 20, 4)}
        for m in sweeps:
            rec[f"fgmres_{m}_{m}"] = solve(F, silu.PRECOND_SCHUR, m, m)
        rec["amg_setup_s"] = amg(F)
        rec["amg_levels"] = F.amg_stats()["levels"]
        for m in sweeps:
            rec[f"amg_schur_fgmres_{m}_{m}"] = solve(F, silu.PRECOND_AMG_SCHUR, m, m)
        # the interface iteration right-preconditioned by diag(C) (not in the paper)
        F.schur_set_interface_prec(silu.SCHUR_IFACE_DIAG)
        for m in sweeps:
            rec[f"diag_fgmres_{m}_{m}"] = solve(F, silu.PRECOND_SCHUR, m, m)
            rec[f"diag_amg_schur_fgmres_{m}_{m}"] = solve(F, silu.PRECOND_AMG_SCHUR, m, m)
        out[f"parts_{p}"] = rec
        del F
    F = silu.ilu_setup(ctx, M, "ilut", tau, fill)
    for m in sweeps:
        out[f"single_level_ilut_{m}_{m}"] = solve(F, silu.PRECOND_SWEEPS, m, m)
    out["single_level_ilut_direct"] = solve(F, silu.PRECOND_DIRECT, 0, 0)
    amg(F)
    for m in sweeps:
        out[f"amg_ilut_{m}_{m}"] = solve(F, silu.PRECOND_AMG, m, m)
    del F
    return out


def run_schur_study(args):
    """Only the Schur complement smoother study (schur_study) on one GPU, one
    JSON line: --schur-study KIND:EDGE (cutcell7 or poisson7)."""
    import torch
    import paper_2111_09512_gb300 as silu
    silu.build()
    ctx = silu.Context(0, torch.cuda.current_stream())
    kind, edge = args.schur_study.split(":")
    if kind not in ("cutcell7", "poisson7", "hex27"):
        raise SystemExit(f"unknown matrix kind {kind}")
    sweeps = tuple(int(m) for m in args.schur_sweeps.split(","))
    parts = tuple(int(p) for p in args.schur_parts.split(","))
    out = schur_study(silu, ctx, torch, edge=int(edge), parts=parts, kind=kind, sweeps=sweeps, maxit=args.schur_maxit,
                      tau=args.schur_tau, fill=args.schur_fill, theta=args.schur_theta)
    print(json.dumps({"schur_study": out}), flush=True)
    return 0


def run_vcycle_only(args):
    """Only V-cycles of the GMRES+AMG workload, for profiling and quick timing:
    the 224^3 cut-cell matrix (seed 1), FP64 ILU(0) factors with 10+10 sweeps
    on the finest level, Ruge-Stueben hierarchy (theta 0.25, coarsest <= 400
    rows), one l1-Jacobi step below; W untimed and K timed cycles, one JSON
    line (time per cycle, the cycle's algorithmic bytes and their fraction of
    the measured HBM bandwidth, per-class kernel split)."""
    import torch
    import paper_2111_09512_gb300 as silu
    import synth
    silu.build()
    stream = torch.cuda.current_stream()
    ctx = silu.Context(0, stream)
    A = synth.cutcell7(224, seed=1)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    del A
    F = silu.ilu_setup(ctx, M, "ilu0")
    F.amg_setup(theta=0.25, max_levels=25, coarse_size=400, jacobi_sweeps=1)
    st, sf = F.amg_stats(), F.stats()
    b = torch.from_numpy(synth.rhs(n, 1, seed=1)[:, 0].copy()).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        F.amg_vcycle(x, b, 10, 10)
    torch.cuda.synchronize()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        F.amg_vcycle(x, b, 10, 10)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms = e0.elapsed_time(e1) / args.steps
    peak, _ = load_peaks()
    nbytes = vcycle_bytes(st, sf["nnz_L"], sf["nnz_U"], 10, 10, 1)
    line = {"vcycle_only": "cutcell7-224^3 ILU(0) FP64 + AMG, 10+10 sweeps on the finest level", "rows": n,
            "levels": st["levels"], "steps": args.steps, "warmup": args.warmup, "ms_per_cycle": round(ms, 4),
            "algorithmic_bytes": int(nbytes), "fraction_of_measured_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peak, 3),
            "launches_per_cycle": {k: v[0] // args.steps for k, v in prof.items() if v[0]},
            "kernel_ms_per_cycle": {k: round(v[1] / args.steps, 4) for k, v in prof.items() if v[0]}}
    print(json.dumps(line), flush=True)
    return 0


def run_apply_only(args):
    """Only smoother applications of one workload, for profiling and quick
    timing: W untimed and K timed applications from x = 0 on one GPU, one
    JSON line (time per application, algorithmic GB/s, per-class split).
      cutcell128: the headline workload (128^3 cut-cell, ILUT(1e-3,10), FP64,
                  10+10 sweeps, 1 RHS; 19 launches per application)
      hex27_256:  the 27-point 256^3 perturbed-hex matrix, ILU(0) factors in
                  FP32, 3+3 FP32 sweeps, FP64 residual (5 launches each)
      hex27_128:  the same at 128^3
      hex27_128_direct: 128^3 27-point ILU(0) in FP64, exact triangular solves
                  (direct_trisolve, the automatic schedule) instead of sweeps
      cutcell128_r4: the headline factors with 4 interleaved right-hand sides
      poisson32_r4: 32^3 Poisson ILU(0), 4 interleaved right-hand sides, 5+5
                  sweeps (a system small enough for the fused application)"""
    import torch
    import paper_2111_09512_gb300 as silu
    import synth
    silu.build()
    stream = torch.cuda.current_stream()
    ctx = silu.Context(0, stream)
    w = args.apply_only
    direct = False
    if w in ("cutcell128", "cutcell128_r4"):
        A = synth.cutcell7(EDGE, seed=1)
        kind, prec, mL, mU, vb = "ilut", silu.FP64, ML, MU, 8
        R = 4 if w.endswith("r4") else 1
    elif w in ("hex27_256", "hex27_128"):
        A = synth.hex27(256 if w == "hex27_256" else 128, seed=2)
        kind, prec, mL, mU, vb, R = "ilu0", silu.FP32, 3, 3, 4, 1
    elif w == "hex27_128_direct":
        A = synth.hex27(128, seed=2)
        kind, prec, mL, mU, vb, R, direct = "ilu0", silu.FP64, 0, 0, 8, 1, True
    elif w == "poisson32_r4":
        A = synth.poisson7(32)
        kind, prec, mL, mU, vb, R = "ilu0", silu.FP64, 5, 5, 8, 4
    else:
        raise SystemExit(f"unknown workload {w}")
    n = len(A[0]) - 1
    nnzA = len(A[1])
    M = silu.Matrix(ctx, *A)
    del A
    F = silu.ilu_setup(ctx, M, kind, TAU, FILL, prec=prec)
    st = F.stats()
    b = torch.from_numpy(synth.rhs(n, R, seed=1)).cuda()
    x = torch.zeros(n, R, dtype=torch.float64, device="cuda")
    def apply():
        if direct:
            silu.direct_trisolve(F, x, b)
        else:
            silu.ilu_smooth(F, x, b, mL, mU)

    for _ in range(args.warmup):
        x.zero_()
        apply()
    torch.cuda.synchronize()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        apply()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms = e0.elapsed_time(e1) / args.steps
    if direct:
        # residual, then each factor read once, with its row pointers; vectors: r and y (L solve),
        # y, dinv and x read and x written (U solve)
        nbytes = (resid_bytes(n, nnzA, R) + (st["nnz_L"] + st["nnz_U"]) * (vb + 4) + 8 * (n + 1)
                  + 6 * n * R * 8)
    else:
        # applications from the second on start from x != 0: residual + (mL-1) + (mU-1) sweeps
        nbytes = (resid_bytes(n, nnzA, R) + (mL - 1) * sweep_bytes(n, st["nnz_L"], R, vb) + 8 * n
                  + (mU - 1) * sweep_bytes(n, st["nnz_U"], R, vb) + 8 * n * R)
    line = {"apply_only": w, "rows": n, "rhs": R, "steps": args.steps, "warmup": args.warmup,
            "ms_per_application": round(ms, 5), "algorithmic_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
            "launches_per_application": {k: v[0] // args.steps for k, v in prof.items() if v[0]},
            "kernel_ms_per_launch": {k: round(v[1] / v[0], 5) for k, v in prof.items() if v[0]}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["silu", "reference"], default="silu")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--solve-edge", type=int, default=256)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--amg-edge", type=int, default=224,
                    help="grid edge of the GMRES+AMG comparison (0 = skip)")
    ap.add_argument("--placement-edge", type=int, default=128,
                    help="grid edge of the V-cycle smoother placement study (0 = skip)")
    ap.add_argument("--study", action="store_true",
                    help="add the sweep studies: factorisation kinds, ||T_s^p||_2, time to solution vs sweeps")
    ap.add_argument("--no-scaling-study", action="store_true",
                    help="skip the per-sweep residual reduction of scaled vs unscaled factors (run by default)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests offered at --serve-rate per path")
    ap.add_argument("--serve-low-rate", type=float, default=2.0,
                    help="arrival rate of the sustained (below-saturation) serving run")
    ap.add_argument("--serve-low-seconds", type=float, default=30.0,
                    help="arrival window of the sustained serving run (0 = skip it)")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-queue", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=32)
    ap.add_argument("--apply-only", choices=["cutcell128", "cutcell128_r4", "hex27_256", "hex27_128",
                                             "hex27_128_direct", "poisson32_r4"], default=None,
                    help="run only smoother applications of one workload (profiling, quick timing)")
    ap.add_argument("--vcycle-only", action="store_true",
                    help="run only V-cycles of the 224^3 GMRES+AMG workload (profiling, quick timing)")
    ap.add_argument("--schur-study", default=None, metavar="KIND:EDGE",
                    help="run only the Schur complement smoother study on cutcell7:EDGE, poisson7:EDGE or hex27:EDGE")
    ap.add_argument("--schur-parts", default="8,64", metavar="P[,P...]")
    ap.add_argument("--schur-tau", type=float, default=1e-3)
    ap.add_argument("--schur-fill", type=int, default=10)
    ap.add_argument("--schur-theta", type=float, default=0.25)
    ap.add_argument("--schur-maxit", type=int, default=3000)
    ap.add_argument("--schur-sweeps", default="3", metavar="M[,M...]",
                    help="m_L = m_U sweep counts of the Schur complement smoother study")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.apply_only:
        return run_apply_only(args)
    if args.schur_study:
        return run_schur_study(args)
    if args.vcycle_only:
        return run_vcycle_only(args)
    return run_silu(args)


if __name__ == "__main__":
    sys.exit(main())
