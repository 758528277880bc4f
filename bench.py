#!/usr/bin/env python
"""Benchmark of the adjoint-gradient particle-mesh step on GB300.

One bench step is one full gradient evaluation of the large single-instance workload:
512^3 particles, 1024^3 FP32 mesh, 1000 Mpc/h box, Zel'dovich ICs at a = 1/64, 100 KDK
steps to a = 1, density MSE objective against a target from a second seed, then the
adjoint with reverse time integration back to dJ/domega and dJ/dtheta.  The metric is
PM gradient steps per second: 100 / (time of one evaluation); each counted step
includes its forward KDK step and its reverse adjoint step (ICs, loss and the IC adjoint
are amortised into it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own independent instance (replicas; the
path has no data-parallel exchange): weak scaling, value = all ranks' steps / max time.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
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

METRIC = "adjoint-gradient PM steps/s at 512^3 particles; achieved HBM BW fraction"
WORKLOADS = {
    # name: (box, n_mesh, n_ptcl, n_steps)
    "large": (1000.0, 1024, 512, 100),
    "medium": (400.0, 512, 256, 63),
    "small": (200.0, 256, 128, 63),
}
THETA = (2.1e-9, 0.965, 0.31, 0.049, 0.68)
SAMPLE_SCALE = 512.0  # the oracle sample covers 1/512 of the large workload's particles and cells
SAMPLE_TEXT = ("FP64 oracle (numpy, 1 thread): one forward + one adjoint PM step at 64^3 particles / 128^3 mesh / "
               "125 Mpc/h, scaled x512 in volume to the 512^3 / 1024^3 workload (FFT log factor ignored, "
               "which flatters the oracle)")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ algorithmic bytes
def algorithmic_bytes(n_steps, N, M, batch=1, fused_x=0):
    """Per-pass FP32 traffic per gradient evaluation and per kernel category: one read and
    one write of every mesh a pass touches, particle arrays read and written once.
    Forward: n+1 force evaluations; adjoint: n+1 forward + adjoint force evaluations.
    A deposit fused with the R2C x pass (fused_x bit 0: forward, bit 1: adjoint) writes
    the half spectra (the same bytes as the real meshes) and its x pass disappears."""
    f = n_steps + 1
    b = {
        "scatter": f * (4 * M + 12 * N) + f * (16 * M + 24 * N),
        "fft_x_r2c": (0 if fused_x & 1 else f * 8 * M) + (0 if fused_x & 2 else f * 32 * M),
        # y passes: forward chain delta (8M) + z force (8M) + the x/y split (4M in, 8M out);
        # adjoint chain delta, P_0 (16M) + the x/y merge (8M in, 4M out) + z force, psi
        # (16M) + split (12M)
        "fft_cols": f * (8 * M + 8 * M + 12 * M) + f * (16 * M + 12 * M + 16 * M + 12 * M),
        # z passes: 1 spectrum in, 2 out (force); 2 in, 1 out (adjoint)
        "fused_z_force": 2 * f * 12 * M,
        "fused_z_adjoint": f * 12 * M,
        "fft_x_c2r": f * 24 * M + f * 32 * M,
        "gather_fwd": f * (12 * M + 48 * N),
        "gather_adj": f * (16 * M + 96 * N),
    }
    return {k: v * batch for k, v in b.items()}


def compulsory_bytes_per_pm_step(N, M):
    """Compulsory FP32 traffic of one adjoint-gradient PM step: the forward step (CIC
    deposit 4M + 12N, R2C 8M, 3 C2R 24M, gather 12M + 48N) and the adjoint step (the forward
    force again, the pi deposit 12M + 12N, 3 R2C 24M, one C2R of the summed spectra 16M, the
    psi gather 4M, the particle arrays 48N more): 152 M + 180 N bytes."""
    return 152 * M + 180 * N


NOMINAL_HBM_GBS = 7900.0   # GB300 data-sheet HBM3e bandwidth, for context beside the measured copy


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- oracle sample
def oracle_sample_seconds(repeats=1):
    """FP64 oracle, one forward PM step plus one adjoint PM step (force, force VJP and
    the kicks/drift) at 64^3 particles on a 128^3 mesh in a 125 Mpc/h box -- the large
    workload's cell size and particle/mesh ratio at 1/512 of its volume."""
    from oracle import cosmo
    from oracle import pm as opm
    from paper_2211_09815_gb300 import inputs
    cfg = opm.PMConfig(box=125.0, n_mesh=128, n_ptcl=64, n_steps=100)
    om = inputs.white_noise(64, 1).astype(np.float64)
    s, p, _ = opm.za_initial_state(om, THETA, cfg)
    q = opm.lattice(cfg)
    k1, dd, k2 = cosmo.kdk_factors(cosmo.time_grid(cfg.a0, cfg.a1, cfg.n_steps), THETA[2])
    pi = np.zeros_like(s)
    xi = np.ones_like(s) * 1e-3
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        # forward step i = 1: kick, drift, force, kick
        a, _ = opm.pm_force(q + s, THETA[2], cfg)
        p1 = p + a * k1[0]
        s1 = s + p1 * dd[0]
        a, _ = opm.pm_force(q + s1, THETA[2], cfg)
        p1 = p1 + a * k2[0]
        # adjoint step: reverse kick, reverse drift, force + VJP, reverse kick
        p2 = p1 - a * k2[0]
        xi2 = xi + a * k2[0]
        s2 = s1 - p2 * dd[0]
        pi2 = pi + xi2 * dd[0]
        a2, f = opm.pm_force(q + s2, THETA[2], cfg)
        al = opm.force_vjp(q + s2, pi2 + 1e-3, f, THETA[2], cfg)
        _ = (p2 - a2 * k1[0], xi2 + al * k1[0])
        times.append(time.perf_counter() - t0)
    return times


def _oracle_worker(repeats):
    """One pool worker: the sample step's seconds (the oracle as it stands, one thread)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    return oracle_sample_seconds(repeats)


def oracle_pool_round(procs, repeats=1):
    """``procs`` oracle sample steps side by side, one per host core, in spawned processes
    (never forked: the caller may hold a CUDA context).  Returns (wall seconds of the round,
    [per-sample seconds])."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_worker, [0] * procs)        # start-up and imports outside the clock
        t0 = time.perf_counter()
        per = pool.map(_oracle_worker, [repeats] * procs)
        wall = time.perf_counter() - t0
    return wall, [t for ts in per for t in ts]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def bench_config(world, workload="large"):
    """The ``config`` object of both arms' JSON lines (the workload, not the launch shapes)."""
    box, nm, npc, n = WORKLOADS[workload]
    return {"workload": f"{npc}^3 particles, {nm}^3 mesh, {box:g} Mpc/h, {n} KDK steps a=1/64->1, ZA ICs, "
                        "density MSE, reverse-time adjoint; one bench step = one gradient evaluation",
            "batch": 1, "ckpt_every": 0, "l2": "inputs larger than L2 (every mesh pass streams 4.3-8.6 GB)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: each bench step is one round of one sample step
    per core in parallel processes; the rate is the sampled PM gradient steps per second of
    the round (each sample is 1/512 of a large-workload PM step).  ms_per_step is the wall
    time of a round, as timed."""
    if rank != 0:
        return
    procs = host_cores()
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    walls = []
    with ctx.Pool(procs) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_worker, [1] * procs)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_worker, [1] * procs)
            walls.append(time.perf_counter() - t0)
    t_round = float(np.mean(walls))
    pm_steps_per_round = procs / SAMPLE_SCALE
    value = pm_steps_per_round / t_round
    sample = SAMPLE_TEXT.replace("1 thread", "1 thread per process") + \
        f"; {procs} processes in parallel per bench step (one per host core)"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_round * 1e3,
           "pm_steps_per_bench_step": pm_steps_per_round, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(world, args.workload),
           "cpu_baseline": {"value": value, "unit": "steps/s", "cores": procs, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_oracle_full(args):
    """The oracle's whole gradient (ICs, forward, MSE loss, reverse-time adjoint, IC adjoint)
    at the 32^3 / 64^3 / 100 Mpc/h / 10-step workload in full, and at the 128^3 / 256^3 /
    200 Mpc/h workload for ``--oracle-steps`` steps (63 in full take close to an hour per
    process), with one process and with one process per host core."""
    import multiprocessing as mp
    import platform
    cases = [("32^3 particles, 64^3 mesh, 100 Mpc/h, 10 steps (in full)", (100.0, 64, 32, 10)),
             (f"128^3 particles, 256^3 mesh, 200 Mpc/h, {args.oracle_steps} of 63 steps", (200.0, 256, 128,
                                                                                            args.oracle_steps))]
    procs = host_cores()
    cpu = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    cpu = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    ctx = mp.get_context("spawn")
    res = {"mode": "oracle_full", "host_cores": procs, "cpu": cpu, "machine": platform.machine(), "cases": []}
    for name, c in cases:
        one = _oracle_gradient_seconds(c)
        with ctx.Pool(procs) as pool:
            t0 = time.perf_counter()
            per = pool.map(_oracle_gradient_seconds, [c] * procs)
            wall = time.perf_counter() - t0
        n = c[3]
        res["cases"].append({"workload": name, "seconds_1_process": one, "pm_steps_per_s_1_process": n / one,
                             "seconds_per_process_all_cores": float(np.mean(per)),
                             "pm_steps_per_s_all_cores": procs * n / wall, "processes": procs})
    print(json.dumps(res))


def _oracle_gradient_seconds(case):
    """Seconds of one oracle gradient evaluation (the target's forward run excluded)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import pm as opm
    from paper_2211_09815_gb300 import inputs
    box, nm, npc, n = case
    cfg = opm.PMConfig(box=box, n_mesh=nm, n_ptcl=npc, n_steps=n)
    tgt = opm.forward(inputs.white_noise(npc, 2).astype(np.float64), THETA, cfg)["delta"]
    om = inputs.white_noise(npc, 1).astype(np.float64)
    t0 = time.perf_counter()
    opm.loss_and_gradient(om, THETA, tgt, cfg)
    return time.perf_counter() - t0


# ------------------------------------------------------------------------ ours
def replica_seed(rank):
    """White-noise stream of a replica: every rank simulates its own universe."""
    return 1 + 10 * rank


def replica_throughput(ms_local, steps, n_steps, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` independent replicas (no collective on the data
    path): each rank ran `steps` gradient evaluations of `n_steps` PM steps in ms_local;
    the job takes the slowest rank's time.  Returns (max ms over ranks, PM steps/s)."""
    import torch
    t = torch.tensor([ms_local], device=device, dtype=torch.float64)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * n_steps * steps / (ms_max / 1e3)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2211_09815_gb300 import build, inputs, pm

    torch.cuda.set_device(local_rank)
    build.build()
    box, nm, npc, n = WORKLOADS[args.workload]
    N, M = npc ** 3, nm ** 3
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    seed = replica_seed(rank)
    om_host = torch.from_numpy(inputs.white_noise(npc, seed)).pin_memory()
    om = om_host.to("cuda")
    # target density from a second seed, made by the same forward model
    om2 = torch.from_numpy(inputs.white_noise(npc, seed + 1)).to("cuda")
    ctx_t = pm.PMContext(box, nm, npc, n, [THETA], om2)
    target = torch.empty(M, device="cuda")
    ctx_t.forward(dens=target)
    torch.cuda.synchronize()
    ctx_t.close()
    del om2
    # no stream synchronisation after each call inside the timed region: the device error
    # flag is checked once after it (ctx.check())
    ctx = pm.PMContext(box, nm, npc, n, [THETA], om, check_errors=False)
    djdd = torch.empty(M, device="cuda")
    gw = torch.empty(N, device="cuda")
    gt = torch.zeros(5, dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    if not args.no_autotune:
        # launch shapes from the autotuner, timed on the final (clustered) forward state
        ctx.forward()
        ctx.autotune()
    tuning = ctx.get_tuning()
    stream = torch.cuda.current_stream()
    marks = []

    def evaluation(timed=False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)] if timed else None
        ctx.forward()
        if timed:
            ev[0].record(stream)
        ctx.loss_mse(target, djdd, loss)
        if timed:
            ev[1].record(stream)
        ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
        if timed:
            ev[2].record(stream)
            marks.append(ev)

    for _ in range(args.warmup):
        evaluation()
    torch.cuda.synchronize()
    ctx.check()
    ctx.profile_read()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    if args.profile_range:
        torch.cuda.profiler.start()   # profilers started with capture off see the timed region only
    ev0.record(stream)
    for _ in range(args.steps):
        evaluation(timed=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    barrier()
    clk = clocks.stop()
    ctx.check()
    ms = ev0.elapsed_time(ev1)
    # forward (ICs + n steps) and adjoint (n reverse steps + IC adjoint) separately
    starts = [ev0] + [m[2] for m in marks[:-1]]
    ms_fwd = sum(a.elapsed_time(m[0]) for a, m in zip(starts, marks)) / args.steps
    ms_adj = sum(m[1].elapsed_time(m[2]) for m in marks) / args.steps
    prof = ctx.profile_read()
    ctx.profile(False)
    loss_val = float(loss.item())
    ms_max, value = replica_throughput(ms, args.steps, n, world, dist, "cuda")
    ms_per_eval = ms_max / args.steps

    # end to end through the C ABI with host buffers: omega and target in, loss and
    # gradients out, copies inside the timed region
    tgt_host = target.cpu().pin_memory()
    gw_host = torch.empty(N, dtype=torch.float32).pin_memory()
    gt_host = torch.zeros(5, dtype=torch.float64).pin_memory()
    loss_host = torch.zeros(1, dtype=torch.float64).pin_memory()
    ctx.gradient(tgt_host, omega=om_host, loss=loss_host, grad_omega=gw_host, grad_theta=gt_host)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.gradient(tgt_host, omega=om_host, loss=loss_host, grad_omega=gw_host, grad_theta=gt_host)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ctx.check()
    e2e_ms = max(e0.elapsed_time(e1), wall * 1e3)
    _, e2e_value = replica_throughput(e2e_ms, args.steps, n, world, dist, "cuda")
    ctx.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_kind = _peaks()
    alg = algorithmic_bytes(n, N, M, fused_x=int(tuning.get("fused_x", 0)))
    ms_pm_step = ms_per_eval / n
    # headline: the whole adjoint-gradient PM step (one forward + one adjoint step) against
    # its compulsory traffic (one read and one write per 3-D FFT, fused Fourier multipliers:
    # forward 48M + 60N, adjoint 104M + 120N bytes)
    comp_bytes = compulsory_bytes_per_pm_step(N, M)
    pass_bytes = sum(alg.values()) / n
    traffic = _ncu_traffic_step()
    achieved = comp_bytes / (ms_pm_step / 1e3) / 1e9
    # the dominant kernel category on its own per-pass bytes
    cats = {k: v for k, v in prof.items() if k in alg}
    dom = max(cats, key=lambda k: cats[k][0])
    dom_ms, dom_launches = cats[dom]
    dom_achieved = alg[dom] * args.steps / (dom_ms / 1e3) / 1e9
    launches_total = int(sum(v[1] for v in prof.values()))
    out = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_eval, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(world, args.workload),
        "pm_steps_per_bench_step": n, "ms_per_pm_step": ms_pm_step,
        "forward_steps_per_s": n / (ms_fwd / 1e3), "adjoint_steps_per_s": n / (ms_adj / 1e3),
        "ms_per_eval_forward": ms_fwd, "ms_per_eval_adjoint": ms_adj,
        "tuning": tuning, "autotuned": not args.no_autotune,
        "particle_updates_per_s": 2 * N * value,
        "roofline": {"bound": "hbm", "kernel": "whole adjoint-gradient PM step (forward step + adjoint step, "
                                                "every kernel)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} copy bandwidth", "alg_bytes": comp_bytes,
                     "alg_bytes_kind": "compulsory: one read + one write per 3-D FFT, multipliers fused",
                     "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "traffic": traffic, "traffic_source": TRAFFIC_NOTE if traffic else None,
                     "per": "PM step", "per_pass_bytes": pass_bytes,
                     "per_pass_frac": pass_bytes / (ms_pm_step / 1e3) / 1e9 / peak},
        "roofline_dominant_kernel": {"kernel": dom, "achieved": dom_achieved, "peak": peak, "unit": "GB/s",
                                     "frac": dom_achieved / peak, "alg_bytes": alg[dom] / (n + 1),
                                     "per": "force chain pair (one forward + one adjoint force evaluation)",
                                     "launches": dom_launches},
        "kernels_ms_per_eval": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": launches_total,
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": 4 * (N + M),
                "d2h_bytes_per_step": 4 * N + 8 * 5 + 8},
        "clocks": clk,
        "loss": loss_val,
    }
    if world == 1 and not args.no_extras:
        # the other configurations of the workload set, measured in the same run: the
        # batched ensemble against 16 sequential runs, and the memory and time of
        # checkpoints against reverse time integration
        torch.cuda.empty_cache()
        out["batched_ensemble"] = batched_ensemble(1, 2)
        torch.cuda.empty_cache()
        out["checkpoint_memory"] = ckpt_compare()
        torch.cuda.empty_cache()
        out["smaller_workloads"] = {w: workload_rate(w) for w in ("small", "medium")}
        torch.cuda.empty_cache()
        # the reduced-precision form on the main workload (accuracy: --precision-study)
        rp = workload_rate(args.workload, 3, 2, half_force=True)
        out["reduced_precision"] = {"form": "FP16 force meshes with a power-of-two scale per row and field "
                                            "(pm_config.half_force); FFTs, deposit and particles FP32", **rp,
                                    "speedup_vs_fp32": rp["steps_per_s"] / value}
    if not args.no_cpu_baseline:
        procs = host_cores()
        wall, per = oracle_pool_round(procs)
        out["cpu_baseline"] = {"value": procs / SAMPLE_SCALE / wall, "unit": "steps/s", "cores": procs,
                               "kind": "oracle",
                               "sample": SAMPLE_TEXT.replace("1 thread", "1 thread per process") +
                               f"; {procs} processes in parallel, one per host core; round of "
                               f"{wall:.2f} s wall, {np.mean(per):.2f} s per sample"}
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def run_op_case(args):
    """The force and force-VJP operators at the final state of a full forward run of the
    chosen workload (late-time clustering), for ncu captures: a warm-up pair, then one pair
    between cudaProfilerStart/Stop (one forward and one adjoint force chain)."""
    import torch
    from paper_2211_09815_gb300 import build, inputs, pm
    build.build()
    box, nm, npc, n = WORKLOADS[args.workload]
    N = npc ** 3
    om = torch.from_numpy(inputs.white_noise(npc, 1)).to("cuda")
    ctx = pm.PMContext(box, nm, npc, n, [THETA], om)
    # the deposit and x pass as separate kernels, the form the autotuner picks at 1024^3
    ctx.set_tuning({"fused_x": args.fused_x})
    disp = torch.empty(3 * N, device="cuda")
    ctx.forward(disp=disp)
    pi = torch.ones(3 * N, device="cuda") * 1e-3
    acc = torch.empty(3 * N, device="cuda")
    alpha = torch.empty(3 * N, device="cuda")
    ctx.op_force(disp, acc)
    ctx.op_force_vjp(disp, pi, acc, alpha)
    torch.cuda.synchronize()
    # the second pair is bracketed for `ncu --profile-from-start off`
    torch.cuda.profiler.start()
    ctx.op_force(disp, acc)
    ctx.op_force_vjp(disp, pi, acc, alpha)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ctx.close()
    print(json.dumps({"op_case": args.workload, "acc_rms": float(acc.pow(2).mean().sqrt()),
                      "alpha_rms": float(alpha.pow(2).mean().sqrt())}))


def run_fft_compare(args):
    """The hand-written 3-D R2C and C2R of a 1024^3 FP32 mesh (pm_op_fft: x, y and z passes
    plus the conversion to the standard [n][n][n/2+1] layout) timed beside cuFFT through
    torch.fft (a reference point, not part of the path), same input, CUDA events."""
    import torch
    from paper_2211_09815_gb300 import build, inputs, pm
    build.build()
    nm = 1024 if args.workload == "large" else WORKLOADS[args.workload][1]
    npc = 64
    om = torch.from_numpy(inputs.white_noise(npc, 1)).to("cuda")
    ctx = pm.PMContext(1000.0, nm, npc, 1, [THETA], om)
    x = torch.randn(nm, nm, nm, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    spec = torch.empty(nm, nm, nm // 2 + 1, 2, device="cuda")
    back = torch.empty(nm, nm, nm, device="cuda")

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            t.append(a.elapsed_time(b))
        return sorted(t)[len(t) // 2]

    ours_r2c = timed(lambda: ctx.op_fft(-1, x, spec))
    ours_c2r = timed(lambda: ctx.op_fft(+1, spec, back))
    ref = torch.fft.rfftn(x)
    got = torch.view_as_complex(spec)
    err = float((got - ref).abs().max() / ref.abs().max())
    del ref, got
    ctx.close()
    torch.cuda.empty_cache()
    cufft_r2c = timed(lambda: torch.fft.rfftn(x))
    X = torch.fft.rfftn(x)
    cufft_c2r = timed(lambda: torch.fft.irfftn(X, s=(nm, nm, nm)))
    gb = (4 * nm ** 3 + 8 * nm * nm * (nm // 2 + 1)) / 1e9
    print(json.dumps({"mode": "fft_compare", "mesh": nm, "dtype": "f32",
                      "ours_ms": {"r2c": ours_r2c, "c2r": ours_c2r},
                      "cufft_ms": {"r2c": cufft_r2c, "c2r": cufft_c2r},
                      "io_GB_per_transform": gb,
                      "ours_note": "x, y, z passes + layout conversion to [n][n][n/2+1]",
                      "max_rel_diff_vs_cufft": err}))


def workload_rate(name, warmup=3, steps=3, half_force=False):
    """Gradient steps/s of a single-instance configuration of the workload set (with
    `half_force`, the FP16 force-mesh form), timed like the main line: autotuned on the
    final forward state, CUDA events on the launching stream around `steps` evaluations
    after `warmup`, the error flag checked after."""
    import torch
    from paper_2211_09815_gb300 import inputs, pm
    box, nm, npc, n = WORKLOADS[name]
    N, M = npc ** 3, nm ** 3
    om2 = torch.from_numpy(inputs.white_noise(npc, 2)).to("cuda")
    c = pm.PMContext(box, nm, npc, n, [THETA], om2)
    target = torch.empty(M, device="cuda")
    c.forward(dens=target)
    c.close()
    om = torch.from_numpy(inputs.white_noise(npc, 1)).to("cuda")
    ctx = pm.PMContext(box, nm, npc, n, [THETA], om, check_errors=False, half_force=half_force)
    ctx.forward()
    ctx.autotune()
    djdd = torch.empty(M, device="cuda")
    gw = torch.empty(N, device="cuda")
    gt = torch.zeros(5, dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def evaluation():
        ctx.forward()
        ctx.loss_mse(target, djdd, loss)
        ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)

    for _ in range(warmup):
        evaluation()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        evaluation()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ctx.close()
    ms = e0.elapsed_time(e1) / steps
    peak, kind = _peaks()
    frac = compulsory_bytes_per_pm_step(N, M) * n / (ms * 1e-3) / 1e9 / peak
    return {"workload": f"{npc}^3 particles, {nm}^3 mesh, {box:g} Mpc/h, {n} steps", "steps_per_s": n / (ms * 1e-3),
            "ms_per_eval": ms, "timed_evals": steps, "warmup": warmup,
            "roofline_frac_compulsory": frac, "peak_kind": kind}


def run_batched(args):
    print(json.dumps(batched_ensemble(args.warmup, args.steps)))


def batched_ensemble(warmup, steps):
    """Batched ensemble: 16 instances of 128^3 particles on 256^3 meshes (200 Mpc/h), own
    seed and theta each, 32 steps, forward + adjoint.  The batched context runs every
    kernel once for all instances and replays a captured CUDA graph; it is compared with 16
    sequential single-instance FP32 contexts (eager launches) on the same inputs."""
    import torch
    from paper_2211_09815_gb300 import build, inputs, pm
    build.build()
    B, box, nm, npc, n = 16, 200.0, 256, 128, 32
    N, M = npc ** 3, nm ** 3
    theta = inputs.ensemble_theta(B)
    stream = torch.cuda.Stream()
    out = {"mode": "batched", "batch": B, "workload": "16 x 128^3 particles, 256^3 mesh, 200 Mpc/h, 32 steps"}
    with torch.cuda.stream(stream):
        om = torch.from_numpy(np.stack([inputs.white_noise(npc, 1 + b) for b in range(B)])).cuda()
        om_t = torch.from_numpy(np.stack([inputs.white_noise(npc, 101 + b) for b in range(B)])).cuda()
        ctx = pm.PMContext(box, nm, npc, n, theta.tolist(), om_t, batch=B, stream=stream, check_errors=False)
        tgt = torch.empty(B * M, device="cuda")
        ctx.forward(dens=tgt)
        # launch shapes from the autotuner, timed on the final (clustered) state
        out["tuning"], out["tuned_ms"] = ctx.autotune()
        ctx.set_inputs(omega=om)
        loss = torch.zeros(B, dtype=torch.float64, device="cuda")
        gw = torch.empty(B * N, device="cuda")
        gt = torch.zeros(5 * B, dtype=torch.float64, device="cuda")
        for _ in range(max(warmup, 1)):
            ctx.gradient_graph(tgt, loss=loss, grad_omega=gw, grad_theta=gt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.gradient_graph(tgt, loss=loss, grad_omega=gw, grad_theta=gt)
        e1.record(stream)
        stream.synchronize()
        ctx.check()
        t_batched = e0.elapsed_time(e1) / steps
        gw_b = gw.cpu().numpy().reshape(B, N)
        ctx.close()
        # 16 sequential single-instance contexts, eager launches
        t_single = 0.0
        max_diff = 0.0
        for b in range(B):
            c1 = pm.PMContext(box, nm, npc, n, [theta[b].tolist()], om[b].contiguous(), stream=stream,
                              check_errors=False)
            c1.set_tuning(out["tuning"])   # the same launch shapes: results comparable bit for bit
            djdd = torch.empty(M, device="cuda")
            g1 = torch.empty(N, device="cuda")
            t1 = tgt[b * M:(b + 1) * M]
            c1.forward(); c1.loss_mse(t1, djdd); c1.adjoint(djdd=djdd, grad_omega=g1)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            c1.forward(); c1.loss_mse(t1, djdd); c1.adjoint(djdd=djdd, grad_omega=g1)
            f1.record(stream)
            stream.synchronize()
            c1.check()
            t_single += f0.elapsed_time(f1)
            max_diff = max(max_diff, float(np.max(np.abs(g1.cpu().numpy() - gw_b[b]))))
            c1.close()
    out.update({"ms_per_batched_eval": t_batched, "ms_16_sequential_evals": t_single,
                "speedup": t_single / t_batched,
                "batched_instance_steps_per_s": B * n / (t_batched / 1e3),
                "sequential_instance_steps_per_s": B * n / (t_single / 1e3),
                "max_abs_grad_diff_batched_vs_single": max_diff})
    return out


def run_ckpt_compare(args):
    print(json.dumps(ckpt_compare()))


def ckpt_compare():
    """Reverse-time recomputation vs checkpoints every 8 steps vs every step (the stored
    trajectory) at 256^3 particles / 512^3 mesh / 400 Mpc/h / 63 steps: device memory,
    time per gradient evaluation and the gradient differences."""
    import torch
    from paper_2211_09815_gb300 import build, inputs, pm
    build.build()
    box, nm, npc, n = 400.0, 512, 256, 63
    N, M = npc ** 3, nm ** 3
    om = torch.from_numpy(inputs.white_noise(npc, 1)).cuda()
    om2 = torch.from_numpy(inputs.white_noise(npc, 2)).cuda()
    c0 = pm.PMContext(box, nm, npc, n, [THETA], om2)
    tgt = torch.empty(M, device="cuda")
    c0.forward(dens=tgt)
    c0.close()
    res, grads = {}, {}
    for k in (0, 8, 1):
        torch.cuda.synchronize()
        ctx = pm.PMContext(box, nm, npc, n, [THETA], om, ckpt_every=k, check_errors=False)
        djdd = torch.empty(M, device="cuda")
        gw = torch.empty(N, device="cuda")
        gt = torch.zeros(5, dtype=torch.float64, device="cuda")
        for _ in range(2):
            ctx.forward(); ctx.loss_mse(tgt, djdd); ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.forward(); ctx.loss_mse(tgt, djdd); ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
        e1.record()
        torch.cuda.synchronize()
        ctx.check()
        res[f"ckpt_every_{k}"] = {"ms_per_eval": e0.elapsed_time(e1), "scratch_GB": ctx.scratch_bytes / 1e9}
        grads[k] = (gw.cpu().numpy().astype(np.float64), gt.cpu().numpy())
        ctx.close()
    g0, g8, g1 = grads[0][0], grads[8][0], grads[1][0]
    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    def cos(a, b):
        return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
    res["grad_omega_reverse_vs_stored"] = {"rel_l2": rel(g0, g1), "cosine": cos(g0, g1)}
    res["grad_omega_ckpt8_vs_stored"] = {"rel_l2": rel(g8, g1), "cosine": cos(g8, g1)}
    res["grad_theta"] = {str(k): grads[k][1].tolist() for k in grads}
    return {"mode": "ckpt_compare", "workload": "256^3 particles, 512^3 mesh, 400 Mpc/h, 63 steps", **res}


def run_precision_study(args):
    """FP32 against an FP64 GPU run of the same workload, per output: final displacement
    RMS (in cells), momentum relative L2, per-shell P(k) relative error, dJ/domega cosine
    and relative L2, dJ/dtheta relative error; the FP32 gradient with reverse time
    integration, with checkpoints every 8 steps and with the exactly reversible fixed-point
    state (fixed_state).  Control: the FP64 run again with every
    omega value moved by one FP32 ulp (seeded signs), whose gradient difference from the
    FP64 run measures how much of the FP32 gradient error is the problem's own
    sensitivity (particles crossing cell faces, where the CIC weight gradient jumps)."""
    import torch
    from paper_2211_09815_gb300 import build, inputs, pm
    build.build()
    box, nm, npc, n = WORKLOADS[args.workload]
    N, M = npc ** 3, nm ** 3
    out = {}
    tgt_np = None
    for prec, ck, pert, fix, hf in ((0, 0, False, False, False), (0, 8, False, False, False),
                                    (0, 0, False, True, False), (0, 0, False, False, True),
                                    (1, 0, False, False, False), (1, 0, True, False, False)):
        dt = torch.float32 if prec == 0 else torch.float64
        if tgt_np is None:
            om2 = torch.from_numpy(inputs.white_noise(npc, 2)).cuda()
            c0 = pm.PMContext(box, nm, npc, n, [THETA], om2)
            t = torch.empty(M, device="cuda")
            c0.forward(dens=t)
            tgt_np = t.cpu().numpy()
            c0.close()
            del om2, t
        om_np = inputs.white_noise(npc, 1)
        if pert:
            sign = np.where(inputs.uniform01(77, om_np.size).reshape(om_np.shape) < 0.5, -1.0, 1.0)
            om_np = om_np.astype(np.float64) + sign * np.spacing(np.abs(om_np)).astype(np.float64)
        om = torch.from_numpy(np.ascontiguousarray(om_np)).to("cuda", dt)
        ctx = pm.PMContext(box, nm, npc, n, [THETA], om, precision=prec, ckpt_every=ck, fixed_state=fix,
                           half_force=hf)
        disp = torch.empty(3 * N, device="cuda", dtype=dt)
        mom = torch.empty_like(disp)
        ctx.forward(disp=disp, mom=mom)
        km, pk, nmodes = ctx.power_spectrum()
        tgt = torch.from_numpy(tgt_np).to("cuda", dt)
        djdd = torch.empty(M, device="cuda", dtype=dt)
        ctx.loss_mse(tgt, djdd)
        gw = torch.empty(N, device="cuda", dtype=dt)
        gt = torch.zeros(5, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
        torch.cuda.synchronize()
        out[(prec, ck, pert, fix, hf)] = dict(s=disp.cpu().numpy().astype(np.float64), p=mom.cpu().numpy().astype(np.float64),
                         pk=pk[0], nmodes=nmodes, gw=gw.cpu().numpy().astype(np.float64), gt=gt.cpu().numpy(),
                         adj_s=time.perf_counter() - t0)
        ctx.close()
        del om, disp, mom, tgt, djdd, gw, gt
        torch.cuda.empty_cache()
    a, b, a8 = out[(0, 0, False, False, False)], out[(1, 0, False, False, False)], out[(0, 8, False, False, False)]
    bp, af = out[(1, 0, True, False, False)], out[(0, 0, False, True, False)]
    ah = out[(0, 0, False, False, True)]
    cell = box / nm
    ok = b["nmodes"] > 0
    ok[0] = False
    res = {
        "mode": "precision_study", "workload": f"{npc}^3 particles, {nm}^3 mesh, {box:g} Mpc/h, {n} steps",
        "disp_rms_cells": float(np.sqrt(np.mean((a["s"] - b["s"]) ** 2)) / cell),
        "mom_rel_l2": float(np.linalg.norm(a["p"] - b["p"]) / np.linalg.norm(b["p"])),
        "pk_max_rel": float(np.max(np.abs(a["pk"][ok] / b["pk"][ok] - 1))),
        "grad_omega_cosine": float(a["gw"] @ b["gw"] / (np.linalg.norm(a["gw"]) * np.linalg.norm(b["gw"]))),
        "grad_omega_rel_l2": float(np.linalg.norm(a["gw"] - b["gw"]) / np.linalg.norm(b["gw"])),
        "grad_theta_rel": (np.abs(a["gt"] / b["gt"] - 1)).tolist(),
        "grad_theta_fp64": b["gt"].tolist(),
        "ckpt8_f32": {"grad_omega_cosine": float(a8["gw"] @ b["gw"] / (np.linalg.norm(a8["gw"]) * np.linalg.norm(b["gw"]))),
                      "grad_omega_rel_l2": float(np.linalg.norm(a8["gw"] - b["gw"]) / np.linalg.norm(b["gw"])),
                      "grad_theta_rel": (np.abs(a8["gt"] / b["gt"] - 1)).tolist()},
        "adjoint_seconds": {"f32": a["adj_s"], "f32_ckpt8": a8["adj_s"], "f64": b["adj_s"]},
        "f32_half_force": {
            "disp_rms_cells": float(np.sqrt(np.mean((ah["s"] - b["s"]) ** 2)) / cell),
            "mom_rel_l2": float(np.linalg.norm(ah["p"] - b["p"]) / np.linalg.norm(b["p"])),
            "pk_max_rel": float(np.max(np.abs(ah["pk"][ok] / b["pk"][ok] - 1))),
            "grad_omega_cosine": float(ah["gw"] @ b["gw"] / (np.linalg.norm(ah["gw"]) * np.linalg.norm(b["gw"]))),
            "grad_omega_rel_l2": float(np.linalg.norm(ah["gw"] - b["gw"]) / np.linalg.norm(b["gw"])),
            "grad_theta_rel": (np.abs(ah["gt"] / b["gt"] - 1)).tolist()},
        "f32_fixed_state": {
            "disp_rms_cells": float(np.sqrt(np.mean((af["s"] - b["s"]) ** 2)) / cell),
            "grad_omega_cosine": float(af["gw"] @ b["gw"] / (np.linalg.norm(af["gw"]) * np.linalg.norm(b["gw"]))),
            "grad_omega_rel_l2": float(np.linalg.norm(af["gw"] - b["gw"]) / np.linalg.norm(b["gw"])),
            "grad_theta_rel": (np.abs(af["gt"] / b["gt"] - 1)).tolist()},
        "control_f64_omega_moved_1_f32_ulp": {
            "disp_rms_cells": float(np.sqrt(np.mean((bp["s"] - b["s"]) ** 2)) / cell),
            "grad_omega_cosine": float(bp["gw"] @ b["gw"] / (np.linalg.norm(bp["gw"]) * np.linalg.norm(b["gw"]))),
            "grad_omega_rel_l2": float(np.linalg.norm(bp["gw"] - b["gw"]) / np.linalg.norm(b["gw"])),
            "grad_theta_rel": (np.abs(bp["gt"] / b["gt"] - 1)).tolist()},
    }
    print(json.dumps(res))


TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "ncu_traffic_medium_force_chains.md")
TRAFFIC_NOTE = ("ncu DRAM read + write bytes of every kernel of one forward and one adjoint force chain at "
                "256^3/512^3, scaled x8 to 512^3/1024^3 (profiles/ncu_traffic_medium_force_chains.md)")


def _ncu_traffic_table():
    """{category: DRAM bytes per PM step at the large workload} from the committed ncu
    summary of the current kernel build (measured at 256^3/512^3 and scaled by the 8x
    larger M and N), or {} when the summary is absent."""
    out = {}
    try:
        with open(TRAFFIC_SUMMARY) as f:
            for line in f:
                cells = [c.strip() for c in line.strip().strip("|").split("|")]
                if len(cells) == 6 and cells[0] not in ("category", "---"):
                    try:
                        out[cells[0]] = float(cells[5])
                    except ValueError:
                        pass
    except OSError:
        return {}
    return out


def _ncu_traffic(category):
    return _ncu_traffic_table().get(category)


def _ncu_traffic_step():
    """DRAM bytes of a whole PM step (every category), or None without a summary."""
    t = _ncu_traffic_table()
    return sum(t.values()) if t else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed evaluations with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-ensemble, checkpoint-memory and smaller-workload measurements of the main line")
    ap.add_argument("--batched", action="store_true", help="16-instance batched graph vs sequential runs")
    ap.add_argument("--fft-compare", action="store_true", help="hand-written 3-D FFT beside cuFFT (torch.fft)")
    ap.add_argument("--compare-ckpt", action="store_true", help="reverse time vs checkpoints: memory/time")
    ap.add_argument("--precision-study", action="store_true", help="FP32 vs FP64 GPU run, errors per output")
    ap.add_argument("--oracle-full", action="store_true",
                    help="time the oracle's whole gradient on the host cores (1 process and one per core)")
    ap.add_argument("--oracle-steps", type=int, default=2, help="steps of the 128^3 case of --oracle-full")
    ap.add_argument("--fused-x", type=int, default=0, help="--op-case: pm_tuning.fused_x (0: separate passes)")
    ap.add_argument("--op-case", action="store_true",
                    help="run one force and one force-VJP operator call (no timing), for profilers")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.fft_compare:
        run_fft_compare(args)
    elif args.batched:
        run_batched(args)
    elif args.compare_ckpt:
        run_ckpt_compare(args)
    elif args.precision_study:
        run_precision_study(args)
    elif args.op_case:
        run_op_case(args)
    elif args.oracle_full:
        run_oracle_full(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
