"""Benchmark of the RBSOG force step on GB300: particle-steps/s at N = 1e6.

Workload: Yukawa one-component plasma, N = 1e6 uniform (seeded), Gamma = 0.1, kappa = 2,
r_c = 3a, P = 500, dt = 0.01, BAOAB Langevin, FP32 forces with FP64 integration (the
FP64 form is timed beside it).  One step = sample, cell list, near field, structure
factor, far gather and integration (Algorithm 2), replayed from a CUDA graph.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun each rank advances its own independent replica
(weak scaling, no collective on the data path); rank 0 prints the line with the
whole-job throughput and the max-over-ranks time.
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

from paper_2501_10946_gb300 import workloads as W  # noqa: E402

METRIC = "RBSOG particle-steps/s at N=1e6"
SMS = 152
MUFU_PER_CLK_SM = 16            # sin/cos and rsqrt special-function results per clock per SM (measured 15.9)
EX2_PER_CLK_SM = 32             # ex2 results per clock per SM (measured)
FP32_PER_CLK_SM = 128           # FP32 lanes per SM
NEAR_FP32_OPS_PER_PAIR = 25     # separation, r^2, Yukawa and Gaussian terms, force accumulation
NEAR_FILTER_OPS = 4             # pre-filter test of one candidate of one target: three FMAs, a compare
KERNELS_PER_STEP = 11
# DRAM bytes per launch of each kernel group from an ncu capture, with the SHA-256 of the
# kernel's source file at capture time: a kernel whose source has changed since gets no
# traffic figure.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_yocp_uniform_n1e6.txt")
CSRC = os.path.join(ROOT, "paper_2501_10946_gb300", "csrc")


def traffic_table():
    """{group: bytes per launch} for the groups whose source is unchanged since capture."""
    import hashlib
    out = {}
    if not os.path.exists(TRAFFIC_FILE):
        return out
    for line in open(TRAFFIC_FILE):
        parts = line.split()
        if len(parts) < 4 or line.startswith("#"):
            continue
        group, src, sha, nbytes = parts[:4]
        path = os.path.join(CSRC, src)
        if os.path.exists(path) and hashlib.sha256(open(path, "rb").read()).hexdigest() == sha:
            out[group] = float(nbytes)
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def rbsog_replica(w, precision, steps, warmup, rank, torch, R, profile_steps=10, e2e_steps=5, clocks=None):
    """Time K steps of one replica; returns the measurements of this rank."""
    dev = torch.device("cuda", torch.cuda.current_device())
    r = torch.tensor(W.positions(w), device=dev, dtype=torch.float64)
    v = torch.tensor(W.velocities(w), device=dev, dtype=torch.float64)
    p = R.make_params(w, precision=precision, seed=w.seed_k + 1000 * rank, device=dev.index)
    ctx = R.rbsog_init(p, w.N, W.charges(w), W.masses(w))
    stream = torch.cuda.current_stream(dev)
    out = {}
    try:
        R.rbsog_set_state(ctx, r, v, stream=stream)
        R.rbsog_step(ctx, warmup, stream=stream)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if clocks is not None:
            clocks.__enter__()
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        R.rbsog_step(ctx, steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        if clocks is not None:
            clocks.__exit__()
        out["ms"] = e0.elapsed_time(e1)
        energy = R.rbsog_step(ctx, 0, energy=True, stream=stream)
        out["energy_total"] = energy["total"] if energy else None
        # kernel-group durations: eager launches with CUDA events on the same stream
        if profile_steps:
            R.rbsog_profile(ctx, True)
            R.rbsog_step(ctx, profile_steps, stream=stream)
            torch.cuda.synchronize(dev)
            out["profile"] = R.rbsog_profile_read(ctx)
            R.rbsog_profile(ctx, False)
        # end to end through the C ABI with pinned host buffers: every step uploads the
        # integrator state (r, v and the forces at r), takes one step and reads the new
        # state back into the same buffers, which the next step uploads.  The FP32 build
        # moves its forces as FP32 (the values it computes), r and v as FP64.
        if e2e_steps:
            f32 = precision == R.RBSOG_FP32
            fdt = torch.float32 if f32 else torch.float64
            set_sf = R.rbsog_set_state_forces_f32 if f32 else R.rbsog_set_state_forces
            get_f = R.rbsog_get_forces_f32 if f32 else R.rbsog_get_forces
            hr = torch.empty((w.N, 3), dtype=torch.float64, pin_memory=True)
            hv = torch.empty((w.N, 3), dtype=torch.float64, pin_memory=True)
            hF = torch.empty((w.N, 3), dtype=fdt, pin_memory=True)
            R.rbsog_get_state(ctx, hr, hv, stream=stream)
            get_f(ctx, hF, stream=stream)

            def e2e_step():
                set_sf(ctx, hr, hv, hF, stream=stream)
                R.rbsog_step_get(ctx, 1, hr, hv, hF, stream=stream)

            e2e_step()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                e2e_step()
            torch.cuda.synchronize(dev)
            out["e2e_s"] = time.perf_counter() - t0
            out["e2e_steps"] = e2e_steps
            nbytes = hr.numel() * hr.element_size() + hv.numel() * hv.element_size() + hF.numel() * hF.element_size()
            out["e2e_h2d"] = nbytes
            out["e2e_d2h"] = nbytes
            out["e2e_path"] = (f"{set_sf.__name__}(host r, v FP64; F {'FP32' if f32 else 'FP64'}) + "
                               "rbsog_step_get(1; host r read back beside the step's force kernels, host v and F "
                               "after it), pinned buffers, each step's outputs the next step's inputs (one force "
                               "evaluation per step)")
    finally:
        R.rbsog_free(ctx)
    return out


def sharded_evaluations(w, steps, warmup, rank, ws, torch, R):
    """Domain-decomposed force evaluations of the workload: rank k owns slab k of ws slabs
    along x (with its halo of width r_c), and every evaluation is rbsog_forces_partial, an
    all-reduce of the 2P values of rho (NCCL across ranks), and rbsog_forces_complete.  No
    integration and no particle migration: the decomposition stays that of the initial
    state.  Returns the max-over-ranks milliseconds of `steps` evaluations."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    r, q, m = W.positions(w), W.charges(w), W.masses(w)
    idx, n_owned = R.rbsog_slab_split(r, w.box, 0, ws, rank, w.r_c)
    p = R.make_params(w, precision=R.RBSOG_FP32, device=dev.index, q2_total=float(np.sum(q * q)),
                      qsum_total=float(np.sum(q)))
    ctx = R.rbsog_init(p, len(idx), q[idx], m[idx])
    try:
        R.rbsog_set_owned(ctx, n_owned)
        R.rbsog_set_state(ctx, torch.tensor(r[idx], device=dev, dtype=torch.float64), stream=stream)
        rho = torch.zeros((w.P, 2), device=dev, dtype=torch.float64)
        F = torch.zeros((len(idx), 3), device=dev, dtype=torch.float64)

        def evaluate():
            R.rbsog_forces_partial(ctx, rho, stream=stream)
            if ws > 1:
                torch.distributed.all_reduce(rho)
            R.rbsog_forces_complete(ctx, rho, F, stream=stream)

        for _ in range(warmup):
            evaluate()
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            evaluate()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        if ws > 1:
            t = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
    finally:
        R.rbsog_free(ctx)
    return {"value": w.N * steps / (ms * 1e-3), "unit": "particle-evaluations/s", "ms_per_evaluation": ms / steps,
            "ranks": ws, "owned_on_rank0": n_owned, "halo_on_rank0": len(idx) - n_owned,
            "form": "slabs along x, halo r_c; rbsog_forces_partial + all-reduce of rho (2P doubles) + "
                    "rbsog_forces_complete; no integration or migration",
            "measured_ranks": ws}


def batched_sweep(torch, R, steps, warmup, R_systems=256):
    """Batched replica sweep: R_systems independent systems of uneven N in one graph per
    step (autotuned shapes) against the same systems advanced one context at a time."""
    ws = W.cfg_replicas(R_systems)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    params = [R.make_params(w, precision=R.RBSOG_FP32, device=dev.index) for w in ws]
    r = torch.tensor(np.concatenate([W.positions(w) for w in ws]), device=dev, dtype=torch.float64)
    v = torch.tensor(np.concatenate([W.velocities(w) for w in ws]), device=dev, dtype=torch.float64)
    q = np.concatenate([W.charges(w) for w in ws])
    m = np.concatenate([W.masses(w) for w in ws])
    Ns = [w.N for w in ws]
    Ntot = int(sum(Ns))
    out = {"workload": f"yocp_replicas{R_systems}", "systems": R_systems, "N_total": Ntot, "N_min": min(Ns),
           "N_max": max(Ns), "steps": steps, "warmup": warmup, "dtype": "f32"}
    b = R.rbsog_batch_init(params, Ns, q, m)
    try:
        R.rbsog_batch_set_state(b, r, v, stream=stream)
        near_t, rho_t = R.rbsog_batch_tune(b, 3, stream=stream)
        out["shapes"] = {"near_target": near_t, "rho_target": rho_t}
        R.rbsog_batch_step(b, R_systems, warmup, stream=stream)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R.rbsog_batch_step(b, R_systems, steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        out["value"] = Ntot * steps / (ms * 1e-3)
        out["unit"] = "particle-steps/s"
        out["ms_per_step"] = ms / steps
        prof = R.rbsog_batch_profile(b, 3, stream=stream)
        out["groups_ms_per_step"] = {k: round(t / 3, 4) for k, t in prof.items()}
        out["gpu_launches_per_step"] = KERNELS_PER_STEP
        # the persistent form: the whole step as one cooperative launch (graph-captured)
        R.rbsog_batch_set_persistent(b, True)
        R.rbsog_batch_step(b, R_systems, warmup, stream=stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        R.rbsog_batch_step(b, R_systems, steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        R.rbsog_batch_get_state(b, stream=stream)          # reports a barrier wait that ran out
        pms = e0.elapsed_time(e1)
        out["persistent"] = {"value": Ntot * steps / (pms * 1e-3), "unit": "particle-steps/s",
                             "ms_per_step": pms / steps, "gpu_launches_per_step": 1,
                             "form": "one persistent cooperative launch per step, CUDA-graph replay"}
    finally:
        R.rbsog_batch_free(b)
    # the plain form: each system its own context, one after another
    rh = r.cpu().numpy()
    vh = v.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(Ns)])
    tot_ms = 0.0
    for i, w in enumerate(ws):
        ctx = R.rbsog_init(params[i], w.N, W.charges(w), W.masses(w))
        try:
            R.rbsog_set_state(ctx, rh[off[i]:off[i + 1]], vh[off[i]:off[i + 1]], stream=stream)
            R.rbsog_step(ctx, warmup, stream=stream)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            R.rbsog_step(ctx, steps, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tot_ms += e0.elapsed_time(e1)
        finally:
            R.rbsog_free(ctx)
    out["plain"] = {"value": Ntot * steps / (tot_ms * 1e-3), "unit": "particle-steps/s",
                    "ms_per_step": tot_ms / steps, "form": "one rbsog context per system, run one after another"}
    out["speedup_vs_plain"] = out["value"] / out["plain"]["value"]
    return out


def percentile(x, q):
    return float(np.percentile(np.asarray(x, dtype=np.float64), q))


def served_stream(torch, R, n_jobs=64, rate=50.0, plain=True):
    """Served request stream through the job server (continuous batching) against the
    plain form: the same jobs in arrival order, one rbsog context at a time."""
    js = W.cfg_stream(n_jobs, rate)
    dev = torch.device("cuda", torch.cuda.current_device())
    work = sum(w.N * n for w, n, _ in js)
    out = {"workload": f"yocp_stream{n_jobs}", "jobs": n_jobs, "arrival_rate_per_s": rate,
           "N_range": [min(w.N for w, _, _ in js), max(w.N for w, _, _ in js)],
           "steps_range": [min(n for _, n, _ in js), max(n for _, n, _ in js)], "particle_steps": work}
    wl = [w for w, _, _ in js]
    if len(wl) > 64:
        # long streams: the placements with a minimum separation in worker processes
        # (started by spawn: this process already holds a CUDA context)
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            data = pool.map(W.job_inputs, wl, chunksize=8)
    else:
        data = [W.job_inputs(w) for w in wl]
    inputs = [(R.make_params(w, precision=R.RBSOG_FP32, device=dev.index),) + d for w, d in zip(wl, data)]
    cap = 6_000_000
    cfg = R.make_server_config(cap, cap // 4, 64 * 256, 64, steps_per_round=32, device=dev.index)
    s = R.rbsog_server_create(cfg)
    try:
        t0 = R.rbsog_server_clock(s) + 0.05
        ids = [R.rbsog_server_submit(s, p, q, m, r, v, n, t0 + ta)
               for (p, q, m, r, v), (_, n, ta) in zip(inputs, js)]
        R.rbsog_server_run(s)
        infos = [R.rbsog_server_job(s, i)[0] for i in ids]
        stats = R.rbsog_server_stats(s)
    finally:
        R.rbsog_server_free(s)
    failed = sum(1 for i in infos if i["status"] != R.RBSOG_JOB_DONE)
    lat = [i["t_done"] - i["t_arrival"] for i in infos]
    span = max(i["t_done"] for i in infos) - min(i["t_arrival"] for i in infos)
    out["served"] = {"p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99), "makespan_s": span,
                     "value": work / span, "unit": "particle-steps/s", "failed": failed,
                     "rounds": stats["rounds"], "peak_resident_jobs": stats["peak_jobs"],
                     "peak_resident_particles": stats["peak_particles"], "device_busy_s": stats["busy_s"],
                     "admission_setup_s": stats["setup_s"],
                     "form": "rbsog_server: continuous batching, 32-step rounds, up to 64 resident jobs"}
    if not plain:
        return out
    # plain: first come first served, one context per job (its own rbsog_init, which
    # builds the same SOG, sampler tables and S the server builds at admission)
    clock = 0.0
    lat_p = []
    first = js[0][2]
    for (p, q, m, r, v), (w, n, ta) in zip(inputs, js):
        start = max(clock, ta)
        tb = time.perf_counter()
        ctx = R.rbsog_init(p, w.N, q, m)
        try:
            R.rbsog_set_state(ctx, r, v)
            R.rbsog_step(ctx, n)
            rr = np.empty((w.N, 3))
            vv = np.empty((w.N, 3))
            R.rbsog_get_state(ctx, rr, vv)
        finally:
            R.rbsog_free(ctx)
        clock = start + (time.perf_counter() - tb)
        lat_p.append(clock - ta)
    out["plain"] = {"p50_s": percentile(lat_p, 50), "p99_s": percentile(lat_p, 99), "makespan_s": clock - first,
                    "value": work / (clock - first), "unit": "particle-steps/s",
                    "form": "one rbsog context per job, first come first served (same arrival times)"}
    out["p50_speedup_vs_plain"] = out["plain"]["p50_s"] / out["served"]["p50_s"]
    out["p99_speedup_vs_plain"] = out["plain"]["p99_s"] / out["served"]["p99_s"]
    out["throughput_vs_plain"] = out["served"]["value"] / out["plain"]["value"]
    return out


def near_pairs(w):
    """In-range pairs of one near-field launch, counted from both ends as the kernel
    evaluates them: N (4 pi / 3) r_c^3 n."""
    dens = w.N / w.volume
    return w.N * (4.0 / 3.0) * math.pi * w.r_c ** 3 * dens


def near_candidates(w):
    """27-cell candidates of one launch: N x 27 x mean cell occupancy."""
    nc = [max(int(math.floor(L / w.r_c)), 1) for L in w.box]
    nc = [n if n >= 3 else 1 for n in nc]
    return w.N * 27.0 * w.N / (nc[0] * nc[1] * nc[2])


def roofline(prof, w, pk, mtot):
    """Roofline of the dominant kernel group.  rho and far are bound by the special-function
    unit (one sin and one cos per particle-mode pair).  near is counted on the method's own
    work: the in-range pairs, each with 25 FP32 operations on the FP32 pipe and one rsqrt
    plus 1 + M_tot ex2 on the special-function unit; the cell-list candidate tests are
    reported apart, as overhead."""
    groups = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(groups, key=lambda k: groups[k][0])
    ms, n = groups[dom]
    avg_s = ms / n * 1e-3
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    clk = sm_mhz * 1e6
    extra = {}
    if dom in ("rho", "far"):
        units = 2.0 * w.N * w.P
        peak = SMS * MUFU_PER_CLK_SM * clk / 1e9
        basis = f"{SMS} SMs x {MUFU_PER_CLK_SM} MUFU/clk x {sm_mhz:.0f} MHz (sin+cos per particle-mode pair)"
    elif dom == "near":
        pairs = near_pairs(w)
        units = NEAR_FP32_OPS_PER_PAIR * pairs
        peak = SMS * FP32_PER_CLK_SM * clk / 1e9
        basis = (f"{SMS} SMs x {FP32_PER_CLK_SM} FP32 lanes/clk x {sm_mhz:.0f} MHz; work = "
                 f"{pairs / w.N:.1f} in-range pairs per particle x {NEAR_FP32_OPS_PER_PAIR} FP32 ops")
        xu_s = pairs * (1.0 / MUFU_PER_CLK_SM + (1.0 + mtot) / EX2_PER_CLK_SM) / (SMS * clk)
        extra["xu"] = {"frac": xu_s / avg_s, "basis": f"1 rsqrt at {MUFU_PER_CLK_SM}/clk/SM + {1 + mtot} ex2 at "
                                                      f"{EX2_PER_CLK_SM}/clk/SM per in-range pair"}
        # the pre-filter tests each candidate of a target with three FMAs and a compare
        cand = near_candidates(w)
        extra["overhead"] = {"candidates_per_particle": cand / w.N, "pairs_per_particle": pairs / w.N,
                             "filter_ops_per_candidate": NEAR_FILTER_OPS,
                             "frac_with_filter_ops": (units + NEAR_FILTER_OPS * cand) / avg_s / 1e9 / peak}
    else:
        units, peak, basis = None, None, ""
    achieved = units / avg_s / 1e9 if units else None
    traffic = traffic_table().get(dom) if w.N == 1_000_000 else None
    out = {"kernel": dom, "bound": "alu", "unit": "Gop/s", "achieved": achieved, "peak": peak,
           "frac": achieved / peak if achieved and peak else None, "traffic": traffic,
           "peak_basis": basis, "avg_launch_ms": avg_s * 1e3,
           "groups_ms_per_step": {k: round(v[0] / v[1], 4) for k, v in groups.items()}}
    out.update(extra)
    return out


FP64_PER_CLK_SM = 1.66          # DFMA results per clock per SM (measured)


def roofline_fp64(prof, w, pk, mtot):
    """Roofline of the FP64 build's dominant group against the FP64 pipe.  Operation counts
    of the method, each transcendental (exp, sqrt, reciprocal, sin, cos) counted as one
    operation: near 25 arithmetic + (3 + M_tot) per in-range pair; rho 2 + 3 and far 2 + 6
    per particle-mode pair.  The FP64 pipe spends some 20 issue slots on each
    transcendental, so these fractions are low by construction: they say how much of the
    pipe the method's own operations use."""
    groups = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(groups, key=lambda k: groups[k][0])
    ms, n = groups[dom]
    avg_s = ms / n * 1e-3
    clk = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    peak = SMS * FP64_PER_CLK_SM * clk / 1e9
    if dom == "near":
        units = near_pairs(w) * (25.0 + 3.0 + mtot)
    elif dom == "rho":
        units = 5.0 * w.N * w.P
    elif dom == "far":
        units = 8.0 * w.N * w.P
    else:
        units = None
    achieved = units / avg_s / 1e9 if units else None
    return {"kernel": dom, "bound": "fp64", "unit": "Gop/s", "achieved": achieved, "peak": peak,
            "frac": achieved / peak if achieved else None, "traffic": None,
            "peak_basis": f"{SMS} SMs x {FP64_PER_CLK_SM} DFMA/clk x {clk / 1e6:.0f} MHz",
            "avg_launch_ms": avg_s * 1e3,
            "groups_ms_per_step": {k: round(v[0] / v[1], 3) for k, v in groups.items()}}


def oracle_step_time(w, steps: int = 1, warmup: int = 0):
    """The FP64 oracle as it stands (cell-list near field, random-batch far field, BAOAB)
    on this host's cores: `warmup` untimed steps, then `steps` timed steps of the
    workload; returns (seconds, threads)."""
    from oracle import core, integrate
    from oracle import sog as S
    from oracle.sampler import ModeSampler
    r = W.positions(w)
    v = W.velocities(w)
    q = W.charges(w)
    m = W.masses(w)
    sog = S.build(w.a_ws / w.kappa, w.r_c, w.sog_eps)
    Q2 = float(np.sum(q * q))
    S_ = core.S_sum(w.box, sog, w.kT, Q2)
    ms = ModeSampler(sog, w.box, w.kT, Q2)
    draws = {"d": 0}

    def force(x):
        kset, _ = ms.draw(w.seed_k, draws["d"], w.P)
        draws["d"] += 1
        Ft, _, _, _ = core.rb_forces(x, q, w.box, w.r_c, sog, kset, w.kT, S=S_)
        return Ft

    def step(r, v, F, n):
        if w.ensemble == "langevin":
            return integrate.baoab_step(r, v, F, m, w.box, w.dt, w.langevin_gamma, w.kT, w.seed_k, n, force)
        return integrate.vv_step(r, v, F, m, w.box, w.dt, force)

    F = force(r)
    n = 0
    for _ in range(warmup):
        r, v, F = step(r, v, F, n)
        n += 1
    t0 = time.perf_counter()
    for _ in range(steps):
        r, v, F = step(r, v, F, n)
        n += 1
    return time.perf_counter() - t0, core.num_threads()


def cpu_baseline(w):
    """The FP64 oracle as it stands on this host's cores: 3 steps of the workload after one
    warm-up step on every core; one step of the same state point at N = 1e5 on one core;
    and the full 10-step N = 1000 FP64 workload (velocity Verlet) on every core."""
    from oracle import core
    secs, thr = oracle_step_time(w, 3, 1)
    out = {"value": 3 * w.N / secs, "unit": "particle-steps/s", "cores": thr, "kind": "oracle",
           "sample": f"3 FP64 oracle steps (after 1 warm-up step) of the N={w.N} workload, OpenMP on {thr} threads"}
    w1 = W.scaled(w, min(100_000, w.N), name=w.name)
    core.set_threads(1)
    try:
        s1, _ = oracle_step_time(w1, 1, 0)
    finally:
        core.set_threads(thr)
    out["single_core"] = {"value": w1.N / s1, "unit": "particle-steps/s", "cores": 1,
                          "sample": f"1 FP64 oracle step of the same state point at N={w1.N}"}
    ws = W.cfg_small_fp64()
    s2, _ = oracle_step_time(ws, ws.steps, 0)
    out["small_full_run"] = {"value": ws.N * ws.steps / s2, "unit": "particle-steps/s", "cores": thr,
                             "workload": ws.name, "steps": ws.steps,
                             "sample": f"the whole {ws.steps}-step N={ws.N} FP64 velocity-Verlet run"}
    return out


# the reference arm's bounded sample: the same state point with 1e5 particles (the
# oracle's cost per particle-step does not depend on N: cell-list near field, N P far field)
REFERENCE_SAMPLE_N = 100_000


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=64,
                    help="jobs of the served stream (the full stream of the served workload is 2000)")
    ap.add_argument("--shard", action="store_true",
                    help="also time domain-decomposed force evaluations (one slab per rank)")
    ap.add_argument("--no-serve-plain", action="store_true",
                    help="skip the one-context-per-job comparison of the served stream")
    args = ap.parse_args()
    ws, rank, local = dist_info()
    w = W.cfg_large(args.N)
    pk, pk_kind = peaks()

    if args.impl == "reference":
        if rank != 0:
            return
        steps = max(1, args.steps)
        ws_ = W.scaled(w, min(REFERENCE_SAMPLE_N, w.N), name=w.name)
        secs, thr = oracle_step_time(ws_, steps, max(0, args.warmup))
        val = ws_.N * steps / secs
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "particle-steps/s", "n_gpus": 0,
                "steps": steps, "warmup": args.warmup, "ms_per_step": secs / steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": w.name, "N": w.N, "P": w.P, "Gamma": w.Gamma, "kappa": w.kappa,
                           "r_c_over_a": w.r_c / w.a_ws, "ensemble": w.ensemble},
                "cpu_baseline": {"value": val, "unit": "particle-steps/s", "cores": thr, "kind": "oracle",
                                 "sample": f"{steps} full FP64 oracle step(s) of the workload's state point "
                                           f"at N={ws_.N} (box scaled to the same density)"},
                "e2e": {"value": val, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_2501_10946_gb300 import rbsog as R
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        torch.cuda.set_device(0)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    res = rbsog_replica(w, R.RBSOG_FP32, args.steps, args.warmup, rank, torch, R, clocks=clocks,
                        profile_steps=10 if rank == 0 else 0, e2e_steps=5 if rank == 0 else 0)
    sharded = sharded_evaluations(w, args.steps, max(3, args.warmup), rank, ws, torch, R) if args.shard else None
    ms = res["ms"]
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    total = w.N * args.steps * ws
    value = total / (ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "P": w.P, "Gamma": w.Gamma, "kappa": w.kappa,
                       "r_c_over_a": w.r_c / w.a_ws, "ensemble": w.ensemble, "integrator": "fp32 increments, fp64 state",
                       "l2": "inputs larger than L2 (state + records > 129 MB)", "parallelism": f"replicas{ws}"}}
    sog = R.rbsog_build_sog(w.a_ws / w.kappa, w.r_c, w.sog_eps)
    rf = roofline(res["profile"], w, pk, sog["M1"] + sog["M2"] + 1)
    rf["peak_source"] = pk_kind
    line["roofline"] = rf
    line["clocks"] = clocks.summary() if clocks else None
    line["gpu_launches"] = KERNELS_PER_STEP * args.steps
    if sharded is not None:
        line["sharded"] = sharded
    e2e_rate = w.N * res["e2e_steps"] / res["e2e_s"]
    line["e2e"] = {"value": e2e_rate, "unit": "particle-steps/s", "h2d_bytes_per_step": res["e2e_h2d"],
                   "d2h_bytes_per_step": res["e2e_d2h"], "path": res["e2e_path"]}
    if not args.no_batch:
        line["batched"] = batched_sweep(torch, R, args.steps, max(3, args.warmup))
    if not args.no_serve:
        line["served"] = served_stream(torch, R, n_jobs=args.serve_jobs, plain=not args.no_serve_plain)
    if not args.no_fp64:
        r64 = rbsog_replica(w, R.RBSOG_FP64, 3, 1, rank, torch, R, profile_steps=2, e2e_steps=0)
        rf64 = roofline_fp64(r64["profile"], w, pk, sog["M1"] + sog["M2"] + 1)
        rf64["peak_source"] = "measured DFMA rate (csrc/peak_probe.cu)"
        line["fp64"] = {"value": w.N * 3 / (r64["ms"] * 1e-3), "ms_per_step": r64["ms"] / 3, "steps": 3,
                        "roofline": rf64}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
