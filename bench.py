#!/usr/bin/env python
"""Benchmark of the DBH hot path on GB300: monomer-timesteps/s and accepted
double-bridging moves/s, with the step kernel's fraction of HBM roofline.

One bench step = 50 MD steps + one double-bridging sweep at the paper's rate
R_MC = 1e-3 per monomer per tau (Sec. II.B), i.e. M * 50 * dt * 1e-3 attempts.
Default workload: 1000 chains x N = 1600 (1.6M monomers), kappa = 3.5,
rho = 0.85, T = 1, Gamma = 1, mixed precision, stage n = 12 (WCA) at dt = 0.01
after a short dt-ramped walk through the softening stages.  Its working set is
larger than the 129 MB L2, so every MD step streams from HBM.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (one MD step and 1/50 of a sweep per bench step), on this host.
Under torchrun every rank advances an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MD_PER_STEP = 50
DT = 0.01
DB_BUDGET = 0.1          # attempts per monomer per sweep for the double-bridging metric
DB_SWEEPS = 5
# FENE continuation beyond r* = R0 sqrt(1 - q) for the soft stages of long
# runs (the log term of Eq. 3 is kept below r*; see kg_params.fene_qmin)
FENE_QMIN = 0.01
_T0 = time.time()


def log(msg):
    """Timestamped progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.time() - _T0:8.2f}s] {msg}", file=sys.stderr, flush=True)
# Algorithmic HBM bytes per monomer per step of the fused step kernel at the
# reference skin 0.3 (10.3 Verlet-list neighbours of 4 bytes):
#   positions read + written in binary64   48
#   velocities read + written              24 (binary32) / 48 (binary64)
#   binary32 float4 gather mirror w + r    32
#   Verlet list                            41
# = 145 B (mixed) and 170 B (binary64).  Gathers of neighbour positions are
# L1/L2 hits in cell order and count 0.  The roofline fraction is taken on
# this fixed model; the same model with the list at the skin in use is
# reported beside it.
ALGO_BYTES = {"mixed": 145.0, "fp64": 170.0}


def nb_mean(skin):
    return 0.85 * 4.0 / 3.0 * np.pi * (2 ** (1 / 6) + skin) ** 3


def bytes_per_monomer_at_skin(precision, skin):
    return (48 + 24 + 32 if precision == "mixed" else 48 + 48 + 32) + 4 * nb_mean(skin)


# DRAM bytes per monomer of the mixed step kernel from ncu captures of the
# 1.6M-monomer case, by skin, and the hash of the step kernel's source
# (kg_step.cu) they were taken on (reported as null for another skin or once
# the source changes)
NCU_TRAFFIC = {"bytes_per_monomer": {0.5: 196.8, 0.6: 213.9}, "src_sha1": "e627455da1f4382bbc2b14cf2e2c30d8d440a189"}

WORKLOADS = {
    "cfg5": dict(index=5, desc="1000 chains x N=1600 (1.6M monomers), kappa=3.5, rho=0.85"),
    "cfg4": dict(index=4, desc="500 chains x N=800 (400k monomers), kappa=3.0, rho=0.85"),
    "cfg2": dict(index=2, desc="200 chains x N=400 (80k monomers), kappa=2.5, rho=0.85"),
    "cfg1": dict(index=1, desc="20 chains x N=50 (1000 monomers), kappa=1.5, rho=0.85"),
}


def prelude_stages(kg):
    """dt ramp through the exponent set Xi (Eq. 11) to the n = 12 stage; the
    soft stages get small steps (their k_n bonds are weak, Sec. II.B)."""
    s = [(2.0, 300, 0.0005), (2.0, 300, 0.001), (3.0, 300, 0.001), (4.0, 300, 0.0015), (5.0, 300, 0.002),
         (5.75, 300, 0.002), (6.5, 300, 0.0025), (7.0, 300, 0.003), (8.0, 300, 0.003), (9.0, 300, 0.004),
         (10.0, 300, 0.004), (11.0, 300, 0.005), (12.0, 300, 0.005), (12.0, 300, 0.0075)]
    stages = [kg.stage(n, k, dt) for n, k, dt in s]
    return stages + [kg.stage(12.0, 10 ** 15, DT)], sum(k for _, k, _ in s)


def src_sha1():
    with open(os.path.join(ROOT, "paper_2109_11001_gb300", "csrc", "kg_step.cu"), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.path = os.path.join("/tmp", f"kg_clocks_{os.getpid()}.csv")
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_melt(wl, rank):
    import kg_inputs as KI
    d = KI.config(WORKLOADS[wl]["index"])
    return KI.random_walk_melt(d["n_chains"], d["chain_len"], d["rho"], d["kappa"], d["seed"] + 1000 * rank)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name and its core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        import platform
        name = platform.processor() or platform.machine()
    return name, os.cpu_count() or 1


def _oracle_job(job):
    """One oracle sample in a worker process: md_steps MD steps and db_attempts
    DB attempts from the state stored at job["path"]; returns the seconds of
    each part (the processes run concurrently, one per host core)."""
    import oracle as O
    d = np.load(job["path"])
    x, u = np.ascontiguousarray(d["x"]), np.ascontiguousarray(d["u"])
    p = O.params(job["n_chains"], job["chain_len"], job["box"], job["kappa"], n_exp=job["n_exp"], dt=job["dt"],
                 seed=3 + job["worker"], fene_qmin=job["fene_qmin"])
    t0 = time.perf_counter()
    O.run(p, x, u, 0, job["md_steps"])
    t1 = time.perf_counter()
    pid = np.arange(x.shape[1], dtype=np.int32)
    O.db_sweep(p, x, u, pid, job["worker"], job["db_attempts"])
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(job["db_attempts"], 1)


class OraclePool:
    """The oracle timed as it stands on the host's cores: one process per core,
    each advancing its own replica of the same state (independent melts are
    the method's natural parallel unit), started with the spawn method."""

    def __init__(self, m, x, u, n_exp, dt, fene_qmin, workers=None):
        import multiprocessing as mp
        import tempfile
        self.m = m
        self.workers = workers or (os.cpu_count() or 1)
        fd, self.path = tempfile.mkstemp(suffix=".npz", prefix="kg_oracle_state_")
        os.close(fd)
        np.savez(self.path, x=x, u=u)
        self.base = dict(path=self.path, n_chains=m.n_chains, chain_len=m.chain_len, box=m.box, kappa=m.kappa,
                         n_exp=n_exp, dt=dt, fene_qmin=fene_qmin)
        self.pool = mp.get_context("spawn").Pool(self.workers) if self.workers > 1 else None

    def sample(self, md_steps, db_attempts, concurrent=True):
        """(seconds per MD step, seconds per DB attempt, processes) averaged over
        the processes that ran at the same time."""
        n = self.workers if concurrent else 1
        jobs = [dict(self.base, md_steps=md_steps, db_attempts=db_attempts, worker=w) for w in range(n)]
        res = self.pool.map(_oracle_job, jobs, chunksize=1) if (self.pool and n > 1) else [_oracle_job(jobs[0])]
        t_md = sum(r[0] for r in res) / len(res) / md_steps
        t_db = sum(r[1] for r in res) / len(res)
        return t_md, t_db, n

    def close(self):
        if self.pool:
            self.pool.close()
            self.pool.join()
        try:
            os.unlink(self.path)
        except OSError:
            pass


def step_units(m):
    """(monomer-steps, DB attempts) of one bench step at the paper's rate."""
    return m.M * MD_PER_STEP, m.M * MD_PER_STEP * DT * 1e-3


def per_step_rate(m, t_md, t_db, procs):
    """Monomer-steps/s of `procs` concurrent oracle replicas, each doing one
    bench step (MD_PER_STEP MD steps + the DB attempts of the paper's rate)."""
    units, att = step_units(m)
    return procs * units / (MD_PER_STEP * t_md + att * t_db)


# The reference arm cannot relax the benchmark melt (the oracle needs ~1 s per
# MD step of 1.6M monomers and thousands of soft steps): it times the oracle
# on the generated melt in the soft first stage, n = 2 at dt = 0.001, where a
# step from the generated state is well defined (WCA at dt = 0.01 overstretches
# bonds of the unrelaxed melt within two steps).  The oracle's cost per step
# does not depend on n (every pair term is one pow) or on dt.
REF_STAGE = dict(n_exp=2.0, dt=0.001, fene_qmin=0.0)


def run_reference(args, world, rank):
    if rank != 0:
        return
    m = make_melt(args.workload, 0)
    units, att = step_units(m)
    att_sample = max(1, int(round(att / MD_PER_STEP)))
    pool = OraclePool(m, m.x, m.v, **REF_STAGE)
    try:
        for _ in range(args.warmup):
            pool.sample(1, att_sample)
        t = []
        for _ in range(args.steps):
            t_md, t_db, procs = pool.sample(1, att_sample)
            # one bench step of work spread over the concurrent replicas
            t.append((MD_PER_STEP * t_md + att * t_db) / procs)
    finally:
        pool.close()
    total = sum(t)
    value = m.M * MD_PER_STEP * args.steps / total
    name, ncpu = cpu_model()
    sample = (f"per step: {procs} concurrent processes (one per host core), each 1 MD step of all {m.M} monomers "
              f"+ {att_sample} DB attempts from the generated melt at n = 2, dt = 0.001, scaled to 50 MD steps + "
              f"{att:g} attempts; host CPU {name}")
    line = {"metric": "monomer-timesteps/s", "value": value, "unit": "monomer-steps/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]['desc']}", "sample": sample},
            "cpu_baseline": {"value": value, "unit": "monomer-steps/s", "cores": procs, "kind": "oracle",
                             "sample": sample, "cpu_model": name, "host_cores": ncpu},
            "e2e": {"value": value, "unit": "monomer-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import torch

    import paper_2109_11001_gb300 as kg
    from paper_2109_11001_gb300 import build as B

    if rank == 0 or world == 1:
        B.build()
    barrier(world)
    torch.cuda.set_device(local)
    log("generating melt")
    m = make_melt(args.workload, rank)
    log(f"melt M={m.M}")
    prec = kg.KG_MIXED if args.precision == "mixed" else kg.KG_FP64
    params = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=prec, seed=11 + rank,
                            fene_qmin=FENE_QMIN, skin=args.skin, sort_interval=args.sort_interval)
    stream = torch.cuda.current_stream()
    ctx = kg.kg_create(params, local, stream.cuda_stream, kg.torch_allocator())
    stages, n_pre = prelude_stages(kg)
    kg.kg_set_potential_schedule(ctx, stages)
    kg.kg_load_config(ctx, 0, m.x, m.v)
    log("context ready; prelude")
    kg.kg_step(ctx, n_pre)
    log(f"prelude done ({n_pre} steps)")
    tuning = None
    if args.autotune:
        # pick skin / cell size and step-kernel block size on the relaxed state
        xs, vs = np.zeros_like(m.x), np.zeros_like(m.v)
        kg.kg_get_config(ctx, 0, xs, vs)
        step0, sweep0 = kg.kg_get_counters(ctx)
        best = kg.kg_autotune(params, [xs], [vs], kg.stage(12.0, -1, DT), 200, local, stream.cuda_stream,
                              kg.torch_allocator())
        tuning = {"skin": best.skin, "block_size": best.block_size,
                  "threads_per_monomer": best.threads_per_monomer, "cell_scale": best.cell_scale,
                  "trials": best.trials, "ms_per_md_step": best.ms_per_step}
        log(f"autotune: {tuning}")
        kg.kg_destroy(ctx)
        params = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=prec, seed=11 + rank,
                                fene_qmin=FENE_QMIN, skin=best.skin, block_size=best.block_size,
                                threads_per_monomer=best.threads_per_monomer, sort_interval=args.sort_interval,
                                cell_scale=best.cell_scale)
        ctx = kg.kg_create(params, local, stream.cuda_stream, kg.torch_allocator())
        kg.kg_set_potential_schedule(ctx, [kg.stage(12.0, 10 ** 15, DT)])
        kg.kg_load_config(ctx, 0, xs, vs)
        kg.kg_set_counters(ctx, step0, sweep0)

    def bench_step():
        kg.kg_step(ctx, MD_PER_STEP)
        return kg.kg_db_sweep(ctx, -1.0)

    for i in range(args.warmup):
        st = bench_step()
        log(f"warmup step {i}: attempted {st.attempted} accepted {st.accepted} reevaluated {st.reevaluated}")
    # the state the timed region starts from: the CPU baseline times the oracle on it
    x_t0, u_t0 = np.zeros_like(m.x), np.zeros_like(m.v)
    kg.kg_get_config(ctx, 0, x_t0, u_t0)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    _, _, l0 = kg.kg_profile_read(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc = att = 0
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            st = bench_step()
            acc += st.accepted
            att += st.attempted
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, _, l1 = kg.kg_profile_read(ctx)
    log(f"timed region {ms:.1f} ms, {l1 - l0} kernel launches")
    # the step kernel's own launch time: CUDA events around each launch over
    # a window of the same bench steps (direct launches; the timed region
    # above replays captured graphs, which hold no host events)
    kg.kg_profile(ctx, 1)
    if args.profile_window:
        torch.cuda.cudart().cudaProfilerStart()
    for _ in range(min(args.steps, 5)):
        bench_step()
    if args.profile_window:
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
    step_ms, n_launch, _ = kg.kg_profile_read(ctx)
    kg.kg_profile(ctx, 0)
    log(f"step kernel: {n_launch} launches, {step_ms / max(n_launch, 1):.4f} ms each")
    barrier(world)
    t_max = allmax(world, ms / 1e3)
    units = allsum(world, float(m.M * MD_PER_STEP * args.steps))
    acc_all = allsum(world, float(acc))

    # end to end through the public API: state in from pinned host memory,
    # 50 MD steps + one sweep, positions back to pinned host memory
    hx = torch.from_numpy(m.x).pin_memory()
    hv = torch.from_numpy(m.v).pin_memory()
    hout = torch.empty_like(hx).pin_memory()
    kg.kg_get_config(ctx, 0, hx, hv)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        kg.kg_load_config(ctx, 0, hx, hv)
        bench_step()
        kg.kg_get_config(ctx, 0, hout)
    torch.cuda.synchronize()
    t_e2e = allmax(world, time.perf_counter() - t0)
    log(f"e2e {t_e2e:.3f} s")

    # double-bridging throughput at a fixed attempt budget: M/10 attempts per
    # sweep on the equilibrated melt (uniform proposal), sweeps back to back
    kg.kg_db_sweep(ctx, DB_BUDGET)
    torch.cuda.synchronize()
    barrier(world)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    db_acc = db_att = db_re = db_empty = 0
    d0.record(stream)
    for _ in range(DB_SWEEPS):
        st = kg.kg_db_sweep(ctx, DB_BUDGET)
        db_acc += st.accepted
        db_att += st.attempted
        db_re += st.reevaluated
        db_empty += st.empty
    d1.record(stream)
    torch.cuda.synchronize()
    t_sweeps = allmax(world, d0.elapsed_time(d1) / 1e3)
    db_acc_all = allsum(world, float(db_acc))
    db_att_all = allsum(world, float(db_att))
    db_empty_all = allsum(world, float(db_empty))
    log(f"db budget: {DB_SWEEPS} sweeps, {db_att} attempts, {db_acc} accepted, {db_re} re-evaluated, {t_sweeps * 1e3:.1f} ms")

    # secondary: the same step in plain binary64 on this GPU (single rank), and
    # the learned double-bridging proposal against the uniform one
    sec = lsec = bsec = psec = esec = ssec = None
    if world == 1 and args.secondary:
        psec = ppa_secondary(kg, torch, ctx, m)
        ssec = schedule_secondary(kg, torch, ctx, m)
        if os.path.exists(N1_REF):
            esec = equilibration_secondary(kg, torch, args, local)
        sec = secondary(kg, torch, args, local)
        bsec = batched_secondary(kg, torch, args, local)
        lsec = learned_secondary(kg, torch, args, local)
    kg.kg_destroy(ctx)
    if rank != 0:
        return
    avg_ms = step_ms / max(n_launch, 1)
    run_skin = tuning["skin"] if tuning else args.skin
    bpm = ALGO_BYTES[args.precision]
    achieved = bpm * m.M / (avg_ms * 1e-3) / 1e9
    bpm_skin = bytes_per_monomer_at_skin(args.precision, run_skin)
    peak, src = peaks()
    traffic = None
    bpm_ncu = {round(k, 6): v for k, v in NCU_TRAFFIC["bytes_per_monomer"].items()}.get(round(run_skin, 6))
    if bpm_ncu and NCU_TRAFFIC["src_sha1"] == src_sha1() and args.precision == "mixed":
        traffic = bpm_ncu * m.M
    # the oracle on the same state and stage as the timed region (n = 12,
    # dt = DT): one host core alone, then one process per host core at once
    log("oracle sample")
    pool = OraclePool(m, x_t0, u_t0, n_exp=12.0, dt=DT, fene_qmin=FENE_QMIN)
    try:
        t1_md, t1_db, _ = pool.sample(2, 8, concurrent=False)
        tn_md, tn_db, procs = pool.sample(1, 8, concurrent=True)
    finally:
        pool.close()
    cpu_one = per_step_rate(m, t1_md, t1_db, 1)
    cpu_all = per_step_rate(m, tn_md, tn_db, procs)
    cpu_name, ncpu = cpu_model()
    log(f"oracle: one core {t1_md:.3f} s per MD step, {t1_db:.4f} s per DB attempt; "
        f"{procs} processes {tn_md:.3f} s per MD step each")
    db_admissible = db_att_all - db_empty_all
    line = {
        "metric": "monomer-timesteps/s", "value": units / t_max, "unit": "monomer-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 forces, f64 state" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]['desc']}",
                   "step": f"{MD_PER_STEP} MD steps (n=12, dt={DT}) + 1 DB sweep at R_MC=1e-3/monomer/tau",
                   "precision": args.precision, "replicas": world, "autotuned": tuning,
                   "skin": tuning["skin"] if tuning else args.skin,
                   "l2": "inputs larger than L2 (working set > 129 MB), no flush"},
        "accepted_db_moves_per_s": db_acc_all / t_sweeps,
        "db": {"attempts_per_sweep": int(round(DB_BUDGET * m.M)), "sweeps": DB_SWEEPS * world,
               "attempted": int(db_att_all), "empty": int(db_att_all - db_admissible),
               "admissible": int(db_admissible), "accepted": int(db_acc_all), "reevaluated": int(db_re),
               "acceptance_per_attempt": db_acc_all / max(db_att_all, 1),
               "acceptance_per_admissible": db_acc_all / max(db_admissible, 1),
               "accepted_per_s": db_acc_all / t_sweeps, "attempts_per_s": db_att_all / t_sweeps,
               "ms_per_sweep": t_sweeps * 1e3 / DB_SWEEPS, "proposal": "uniform",
               "stage": f"n = 12, dt = {DT}",
               "timing": "CUDA events around back-to-back sweeps, stats read after each"},
        "accepted_db_moves_per_s_in_step": acc_all / t_max,
        "db_attempts_per_step": att / args.steps,
        "roofline": {"bound": "hbm", "kernel": "k_step32" if args.precision == "mixed" else "k_step_f64", "achieved": achieved, "peak": peak,
                     "timing": "CUDA events around each step-kernel launch, bench steps after the timed region",
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": src, "bytes_per_monomer": bpm,
                     "bytes_model": "145 B (mixed) / 170 B (binary64) per monomer-step: list at skin 0.3",
                     "bytes_per_monomer_at_skin": bpm_skin,
                     "frac_at_skin": bpm_skin * m.M / (avg_ms * 1e-3) / 1e9 / peak, "skin": run_skin,
                     "avg_launch_ms": avg_ms},
        "cpu_baseline": {"value": cpu_all, "unit": "monomer-steps/s", "cores": procs, "kind": "oracle",
                         "sample": f"one process per host core, each 1 MD step + 8 DB attempts of the full "
                                   f"{m.M}-monomer melt from the timed region's starting state at n = 12, "
                                   f"dt = {DT}, scaled to one bench step",
                         "single_core": {"value": cpu_one, "cores": 1,
                                         "sample": "2 MD steps + 8 DB attempts, one process"},
                         "cpu_model": cpu_name, "host_cores": ncpu},
        "e2e": {"value": units / t_e2e, "unit": "monomer-steps/s",
                "h2d_bytes_per_step": int(hx.numel() * 8 + hv.numel() * 8),
                "d2h_bytes_per_step": int(hout.numel() * 8)},
        "gpu_launches": int(l1 - l0),
        "clocks": clk.summary(),
    }
    if sec:
        line["secondary"] = sec
    if bsec:
        line["batched"] = bsec
    if lsec:
        line["learned_db"] = lsec
    if psec:
        line["ppa"] = psec
    if esec:
        line["equilibration"] = esec
    if ssec:
        line["schedule"] = ssec
    print(json.dumps(line))


SCHED_DT = 0.008          # tau / 125, the protocol's time step (Sec. II.B)


def schedule_secondary(kg, torch, ctx, m):
    """Throughput over the paper's whole schedule for this melt: every stage
    of Xi (Eq. 11) with the scheme of Eqs. 16-20 (scheme 2 above kappa = 2.5)
    timed for 4 x (50 MD steps + one DB sweep at R_MC) at dt = tau/125 on
    the benchmark melt, stages taken from n = 12 down (each switch softens
    the potential), and the stage rates combined with the weights of the
    schedule's step counts: total steps / sum(steps_i / rate_i)."""
    stream = torch.cuda.current_stream()
    plan = kg.kg_schedule_paper(m.kappa, m.chain_len, SCHED_DT, 1.0)
    rates = []
    for st in sorted(plan, key=lambda t: -t.n_exp):
        kg.kg_set_potential_schedule(ctx, [kg.stage(st.n_exp, 10 ** 15, SCHED_DT)])
        for _ in range(2):                                   # warm-up: graph capture, list at the new cut
            kg.kg_step(ctx, MD_PER_STEP)
            kg.kg_db_sweep(ctx, -1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(4):
            kg.kg_step(ctx, MD_PER_STEP)
            kg.kg_db_sweep(ctx, -1.0)
        e1.record(stream)
        torch.cuda.synchronize()
        rates.append((st.n_exp, int(st.n_steps), m.M * MD_PER_STEP * 4 / (e0.elapsed_time(e1) / 1e3)))
    steps = sum(k for _, k, _ in rates)
    weighted = steps / sum(k / r for _, k, r in rates)
    log(f"schedule-weighted: {weighted:.3e} monomer-steps/s over {len(rates)} stages")
    return {"workload": f"{m.n_chains} chains x N={m.chain_len}, kappa={m.kappa}",
            "dt": SCHED_DT, "monomer_steps_per_s": weighted,
            "stages": [{"n": n, "steps": k, "monomer_steps_per_s": r} for n, k, r in sorted(rates)],
            "timing": "CUDA events over 4 x (50 MD steps + 1 DB sweep at R_MC) per stage; weights = the "
                      "schedule's steps per stage"}


PPA_ITERS = 2000


def ppa_secondary(kg, torch, ctx, m):
    """Primitive-path analysis of the equilibrated benchmark melt: calls of 0
    and PPA_ITERS minimisation steps, each timed with CUDA events on the
    library's stream; the per-step time is their difference over PPA_ITERS,
    so the copy of the state, the work-space allocation and the first list
    cancel.  A throughput figure over the contraction phase, where most list
    builds fall."""
    stream = torch.cuda.current_stream()
    kw = dict(dt=0.005, gamma=1.0, skin=0.3)
    kg.kg_primitive_path(ctx, 0, m.n_chains, 2, **kw)            # warm-up
    ms = {}
    for n in (0, PPA_ITERS):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lpp, res = kg.kg_primitive_path(ctx, 0, m.n_chains, n, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[n] = e0.elapsed_time(e1)
    per = (ms[PPA_ITERS] - ms[0]) / PPA_ITERS
    log(f"ppa: {per * 1e3:.1f} us per step, L_pp {res['lpp_mean']:.2f} after {PPA_ITERS} steps, "
        f"{res['builds']} list builds")
    return {"workload": f"{m.n_chains} chains x N={m.chain_len}, the equilibrated benchmark melt",
            "steps": PPA_ITERS, "ms_per_step": per, "monomer_steps_per_s": m.M / (per * 1e-3),
            "setup_ms": ms[0], "lpp_mean": res["lpp_mean"], "fmax": res["fmax"], "list_builds": res["builds"],
            "mean_list_length": res["mean_neighbours"],
            "precision": "mixed",
            "timing": f"CUDA events: (call with {PPA_ITERS} steps - call with 0 steps) / {PPA_ITERS}"}


# kappa scan of eight melts of uneven size (kappa, N, chains): 485k monomers
KAPPA_SCAN = [(0.0, 100, 200), (0.5, 200, 150), (1.0, 400, 100), (1.5, 800, 50), (2.0, 100, 250),
              (2.5, 200, 250), (3.0, 400, 200), (3.5, 800, 250)]


def batched_secondary(kg, torch, args, local):
    """Eight melts of a kappa scan (20k-200k monomers each) advanced by the
    same launches in one context (graphs of separate launches, and persistent
    cooperative launches), against the same melts run one context at a time;
    4 x (50 MD steps + one DB sweep at R_MC) after the dt-ramped prelude."""
    import kg_inputs as KI
    melts = [KI.random_walk_melt(nch, n, 0.85, kap, 2109110013 + 100 * i)
             for i, (kap, n, nch) in enumerate(KAPPA_SCAN)]
    s = torch.cuda.current_stream()

    def run(ms, flags=0):
        p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa) for m in ms], precision=kg.KG_MIXED,
                           seed=19, fene_qmin=FENE_QMIN, skin=0.5, block_size=64, flags=flags)
        ctx = kg.kg_create(p, local, s.cuda_stream, kg.torch_allocator())
        stages, n_pre = prelude_stages(kg)
        kg.kg_set_potential_schedule(ctx, stages)
        for i, m in enumerate(ms):
            kg.kg_load_config(ctx, i, m.x, m.v)
        kg.kg_step(ctx, n_pre)
        kg.kg_step(ctx, MD_PER_STEP)
        kg.kg_db_sweep(ctx, -1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(4):
            kg.kg_step(ctx, MD_PER_STEP)
            kg.kg_db_sweep(ctx, -1.0)
        e1.record(s)
        torch.cuda.synchronize()
        kg.kg_destroy(ctx)
        return e0.elapsed_time(e1) / 1e3

    M = sum(m.M for m in melts)
    t_batched = run(melts)
    log(f"batched kappa scan: {M} monomers, {t_batched * 1e3:.1f} ms")
    t_persist = run(melts, kg.KG_FLAG_PERSISTENT)
    log(f"batched kappa scan, persistent launches: {t_persist * 1e3:.1f} ms")
    t_seq = sum(run([m]) for m in melts)
    log(f"kappa scan one melt at a time: {t_seq * 1e3:.1f} ms")
    units = M * MD_PER_STEP * 4
    return {"workload": "kappa scan: 8 melts, kappa 0-3.5, N 100-800, 50-250 chains, "
                        f"{M} monomers, rho=0.85, skin 0.5, block 64",
            "batched_monomer_steps_per_s": units / t_batched,
            "batched_persistent_monomer_steps_per_s": units / t_persist,
            "persistent": "one cooperative launch per 50 MD steps of all eight melts (KG_FLAG_PERSISTENT)",
            "one_melt_at_a_time_monomer_steps_per_s": units / t_seq}


N1_REF = os.path.join(ROOT, "tests", "golden", "n1_reference.json")


def run_protocol(kg, torch, ref, melts, precision, seeds_from=0, sample=True):
    """The scaled paper protocol of `ref` (stages, sweeps at R_MC with the
    fractional attempts carried over) on `melts` in one context; returns
    (seconds, per-melt <R^2(n)> averaged over the final stage's window,
    end-to-end vectors sampled in the final stage).  Melt i takes the noise
    stream of melt seeds_from + i."""
    S = ref["settings"]
    s = torch.cuda.current_stream()
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa) for m in melts], precision=precision,
                       seed=S["seed"], fene_qmin=S["fene_qmin"])
    ctx = kg.kg_create(p, 0, s.cuda_stream, kg.torch_allocator())
    nm = len(melts)
    N = melts[0].chain_len
    r2 = np.zeros((nm, N))
    buf = np.zeros(N)
    ree = []
    ns = 0
    try:
        stages = [tuple(x) for x in ref["stages"]]
        kg.kg_set_potential_schedule(ctx, [kg.stage(n, k, dt) for n, k, dt in stages])
        for i, m in enumerate(melts):
            kg.kg_load_config(ctx, i, m.x, m.v)
        kg.kg_set_counters(ctx, 0, 0)
        x = np.zeros_like(melts[0].x)
        carry = 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for si, (n, k, dt) in enumerate(stages):
            done = 0
            while done < k:
                q = min(S["sweep_every"], k - done)
                kg.kg_step(ctx, q)
                done += q
                want = S["r_mc"] * melts[0].M * q * dt + carry
                K = int(np.floor(want))
                carry = want - K
                kg.kg_db_sweep_k(ctx, [K] * nm)
                if sample and si == len(stages) - 1 and done % S["sample_every"] == 0:
                    if done > (1 - S["window_frac"]) * k:
                        for i in range(nm):
                            kg.kg_observables(ctx, i, buf)
                            r2[i] += buf
                        ns += 1
                    kg.kg_get_config(ctx, 0, x)
                    c = x.reshape(3, melts[0].n_chains, N)
                    ree.append(c[:, :, -1] - c[:, :, 0])
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
    finally:
        kg.kg_destroy(ctx)
    return sec, (r2 / max(ns, 1)), np.array(ree)


def _r2_mid(r2n):
    N = len(r2n)
    n = np.arange(N // 4, N // 2 + 1)
    return float(np.mean(r2n[n] / n))


def _ree_acf(ree, lags):
    """<R_ee(t) . R_ee(t + lag)> / <R_ee^2> over chains and time origins."""
    v = np.transpose(ree, (0, 2, 1))            # (samples, chains, 3)
    norm = float((v * v).sum(axis=2).mean())
    return [float((v[:-L or None] * v[L:]).sum(axis=2).mean() / norm) if L < len(v) else None for L in lags]


def equilibration_secondary(kg, torch, args, local):
    """Equilibrated melts per hour: the scaled paper protocol (dt ramp, the
    twelve stages of Eqs. 16-20 for kappa = 1.5, N = 50, DB at R_MC) on 16
    melts of 20 x 50, (a) all in one mixed-precision context, (b) in plain
    binary64, one melt per context (two melts timed, the rate per melt
    extrapolated).  Each form's final <R^2(n)>/n over N/4 <= n <= N/2
    (time average over the last 40% of the n = 12 stage, mean over melts) is
    compared with the oracle's value on the same melts and protocol
    (tests/golden/n1_reference.json, written by an oracle-only script); the
    criterion is agreement within 1%."""
    import kg_inputs as KI
    with open(N1_REF) as f:
        ref = json.load(f)
    S = ref["settings"]
    base = KI.config(1)["seed"]
    melts = [KI.random_walk_melt(S["n_chains"], S["chain_len"], S["rho"], S["kappa"], base + 100 * i)
             for i in range(S["n_melts"])]
    oracle_mid = np.array([_r2_mid(np.array(r)) for r in ref["r2n_protocol_end"]])
    t_mix, r2_mix, ree_mix = run_protocol(kg, torch, ref, melts, kg.KG_MIXED)
    mid_mix = np.array([_r2_mid(r) for r in r2_mix])
    log(f"equilibration: mixed batched {len(melts)} melts in {t_mix:.1f} s")
    fp = []
    for i in range(2):
        t, r2, _ = run_protocol(kg, torch, ref, [melts[i]], kg.KG_FP64, sample=True)
        fp.append((t, _r2_mid(r2[0])))
    t_fp = sum(t for t, _ in fp) / len(fp)
    log(f"equilibration: binary64 one melt per context {t_fp:.1f} s per melt")
    d = mid_mix - oracle_mid
    sample_dt = S["sample_every"] * S["dt"]
    lags_tau = [50, 100, 200, 400]
    acf = _ree_acf(ree_mix, [int(round(L / sample_dt)) for L in lags_tau])
    mph_mix = 3600.0 * len(melts) / t_mix
    mph_fp = 3600.0 / t_fp
    return {"workload": f"{len(melts)} melts of {S['n_chains']} chains x N={S['chain_len']}, kappa={S['kappa']}, "
                        f"rho={S['rho']}",
            "protocol": f"dt ramp in n = 2, then the paper's 12 stages (scheme 1) scaled by {S['scale']} at "
                        f"dt = {S['dt']}; {sum(int(x[1]) for x in ref['stages'])} steps; DB at R_MC",
            "criterion": "<R^2(n)>/n over N/4..N/2 within 1% of the oracle's value on the same melts and protocol",
            "oracle_r2_mid": float(oracle_mid.mean()),
            "mixed_batched": {"melts": len(melts), "wall_s": t_mix, "melts_per_hour": mph_mix,
                              "r2_mid": float(mid_mix.mean()),
                              "rel_to_oracle": float(mid_mix.mean() / oracle_mid.mean() - 1.0),
                              "paired_z": float(d.mean() / (d.std(ddof=1) / np.sqrt(len(d)))),
                              "paired_sem_rel": float(d.std(ddof=1) / np.sqrt(len(d)) / oracle_mid.mean()),
                              "within_1pct": bool(abs(mid_mix.mean() / oracle_mid.mean() - 1.0) < 0.01),
                              "within_2_sem": bool(abs(d.mean()) < 2 * d.std(ddof=1) / np.sqrt(len(d)))},
            "fp64_plain": {"melts_timed": len(fp), "wall_s_per_melt": t_fp, "melts_per_hour": mph_fp,
                           "r2_mid_melts_0_1": [m for _, m in fp],
                           "oracle_r2_mid_melts_0_1": oracle_mid[:2].tolist()},
            "melts_per_hour_ratio": mph_mix / mph_fp,
            "ree_autocorrelation": {"lag_tau": lags_tau, "C": acf,
                                    "wall_s_per_tau_mixed_batched_per_melt": t_mix / len(melts) /
                                    (sum(int(x[1]) * x[2] for x in ref["stages"])),
                                    "wall_s_per_tau_fp64_plain": t_fp / (sum(int(x[1]) * x[2] for x in ref["stages"]))}}


def secondary(kg, torch, args, local):
    """80k-monomer melt: mixed vs plain binary64 step rate on this GPU."""
    import kg_inputs as KI
    m = KI.make(2)
    out = {"workload": "cfg2: " + WORKLOADS["cfg2"]["desc"]}
    for name, prec in (("mixed", kg.KG_MIXED), ("fp64", kg.KG_FP64)):
        p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=prec, seed=13,
                           fene_qmin=FENE_QMIN)
        s = torch.cuda.current_stream()
        ctx = kg.kg_create(p, local, s.cuda_stream, kg.torch_allocator())
        stages, n_pre = prelude_stages(kg)
        kg.kg_set_potential_schedule(ctx, stages)
        kg.kg_load_config(ctx, 0, m.x, m.v)
        kg.kg_step(ctx, n_pre)
        log(f"secondary {name}: prelude done")
        for _ in range(2):
            kg.kg_step(ctx, MD_PER_STEP)
            kg.kg_db_sweep(ctx, -1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 10
        e0.record(s)
        for _ in range(n):
            kg.kg_step(ctx, MD_PER_STEP)
            kg.kg_db_sweep(ctx, -1.0)
        e1.record(s)
        torch.cuda.synchronize()
        out[name + "_monomer_steps_per_s"] = m.M * MD_PER_STEP * n / (e0.elapsed_time(e1) / 1e3)
        kg.kg_destroy(ctx)
    return out


LEARNED_STAGES = [(2.0, 300, 0.0005), (2.0, 300, 0.001), (2.0, 300, 0.002), (2.0, 10 ** 15, 0.005)]


def learned_secondary(kg, torch, args, local):
    """400k-monomer melt in the softest stage (n = 2, where the schedule spends
    most of its swaps): double-bridging sweeps with the paper's uniform partner
    draw against the learned proposal (lambda = 0.1) after online training on
    logged uniform sweeps; sweeps alternate between 50-step MD runs so both see
    the same kind of states."""
    import kg_inputs as KI
    m = KI.make(4)
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=kg.KG_MIXED, seed=17,
                       fene_qmin=FENE_QMIN)
    s = torch.cuda.current_stream()
    ctx = kg.kg_create(p, local, s.cuda_stream, kg.torch_allocator())
    kg.kg_set_potential_schedule(ctx, [kg.stage(n, k, dt) for n, k, dt in LEARNED_STAGES])
    kg.kg_load_config(ctx, 0, m.x, m.v)
    kg.kg_step(ctx, 1200)
    K = m.M // 5                                  # ~0.3% of draws are admissible at N = 800: ~20 swaps a sweep
    lam = 0.1
    kg.kg_mlp_log(ctx, 4_000_000)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(6):                          # log: uniform proposal through the learned path
        kg.kg_step(ctx, MD_PER_STEP)
        kg.kg_db_sweep_learned_k(ctx, [K], 1.0)
    kg.kg_mlp_set_weights(ctx, _init_weights())
    iters, batch = 400, 2048
    e0, e1 = ev(), ev()
    e0.record(s)
    loss = kg.kg_mlp_train(ctx, iters, batch, 2e-3)
    e1.record(s)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    log(f"learned: trained {iters} x {batch} rows in {train_ms:.1f} ms, loss {loss:.4f}")
    kg.kg_mlp_log(ctx, 0)
    res = {"uniform": [0, 0, 0.0], "learned": [0, 0, 0.0]}
    for _ in range(4):
        for name in ("uniform", "learned"):
            kg.kg_step(ctx, MD_PER_STEP)
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(s)
            st = kg.kg_db_sweep_k(ctx, [K]) if name == "uniform" else kg.kg_db_sweep_learned_k(ctx, [K], lam)
            b.record(s)
            torch.cuda.synchronize()
            r = res[name]
            r[0] += st.attempted
            r[1] += st.accepted
            r[2] += a.elapsed_time(b)
    kg.kg_destroy(ctx)
    out = {"workload": "cfg4: " + WORKLOADS["cfg4"]["desc"], "stage": "n = 2, k_2, dt = 0.005",
           "attempts_per_sweep": K, "lambda": lam,
           "train": {"iters": iters, "batch": batch, "ms": train_ms, "final_loss": loss}}
    for name, (att, acc, ms) in res.items():
        out[name] = {"acceptance": acc / att, "attempts_per_s": att / (ms / 1e3),
                     "accepted_per_s": acc / (ms / 1e3), "sweep_ms": ms / 4}
    return out


def _init_weights(seed=0):
    """He-style random start for the proposal network (zero biases)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2 / 24), (64, 24))
    W2 = rng.normal(0, np.sqrt(2 / 64), (64, 64))
    w3 = rng.normal(0, np.sqrt(1 / 64), 64) * 0.1
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]])


DBS_KAPPAS = [1.0, 1.5, 2.0, 2.5, 3.0, 3.5]
DBS_STAGES = [2.0, 3.0, 4.0, 5.0, 5.75, 6.5, 7.0, 8.0, 9.0]


def measure_db_success(kg, torch, kappas, stages, rounds=30, flags=0, n_chains=50, N=400):
    """Success rate per admissible double-bridging attempt (Sec. II.B, Fig. 3):
    melts of n_chains x N at each kappa share one mixed context; after a dt
    ramp each stage n relaxes for 2000 steps, then `rounds` rounds of 100 MD
    steps and one sweep of M attempts per melt count admissible attempts (a
    drawn bond with a non-empty partner set) and accepted swaps.  Returns the
    table and the weighted least-squares fit of ln S = ln a - b kappa - d n
    (weights: accepted counts), the form of Eq. 15."""
    import kg_inputs as KI
    s = torch.cuda.current_stream()
    base = KI.SEED_BASE + 7
    melts = [KI.random_walk_melt(n_chains, N, 0.85, k, base + 100 * i) for i, k in enumerate(kappas)]
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa) for m in melts], precision=kg.KG_MIXED,
                       seed=29, fene_qmin=FENE_QMIN, flags=flags, skin=0.4)
    ctx = kg.kg_create(p, 0, s.cuda_stream, kg.torch_allocator())
    table = []
    try:
        kg.kg_set_potential_schedule(ctx, [kg.stage(2.0, 300, 0.0005), kg.stage(2.0, 300, 0.001),
                                           kg.stage(2.0, 300, 0.002), kg.stage(2.0, 10 ** 15, 0.005)])
        for i, m in enumerate(melts):
            kg.kg_load_config(ctx, i, m.x, m.v)
        kg.kg_step(ctx, 900)
        for n in stages:
            dt = 0.005 if n < 5 else 0.008
            kg.kg_set_potential_schedule(ctx, [kg.stage(n, 10 ** 15, dt)])
            kg.kg_step(ctx, 2000)
            adm = np.zeros(len(melts), dtype=np.int64)
            acc = np.zeros(len(melts), dtype=np.int64)
            for _ in range(rounds):
                kg.kg_step(ctx, 100)
                for i, m in enumerate(melts):
                    st = kg.kg_db_sweep_k(ctx, [m.M if j == i else 0 for j in range(len(melts))])
                    adm[i] += st.attempted - st.empty
                    acc[i] += st.accepted
            for i, k in enumerate(kappas):
                table.append({"kappa": k, "n": n, "admissible": int(adm[i]), "accepted": int(acc[i]),
                              "S": float(acc[i] / max(adm[i], 1)),
                              "S_eq15": 1.6 * float(np.exp(-0.77 * k - 0.35 * n))})
    finally:
        kg.kg_destroy(ctx)
    rows = [t for t in table if t["accepted"] > 0]
    A = np.array([[1.0, -t["kappa"], -t["n"]] for t in rows])
    y = np.array([np.log(t["S"]) for t in rows])
    w = np.sqrt(np.array([t["accepted"] for t in rows], dtype=np.float64))
    coef, *_ = np.linalg.lstsq(A * w[:, None], y * w, rcond=None)
    return table, {"a": float(np.exp(coef[0])), "b": float(coef[1]), "d": float(coef[2])}


def db_success(args):
    """Double-bridging success rate per admissible attempt against Eq. 15,
    S = 1.6 exp(-0.77 kappa - 0.35 n), over kappa = 1 ... 3.5 and the stages
    of Xi up to n = 9, with the exact Metropolis-Hastings acceptance and with
    the paper's plain Metropolis (KG_FLAG_PAPER_METROPOLIS)."""
    import torch

    import paper_2109_11001_gb300 as kg
    out = {"workload": "6 melts of 50 chains x N=400 (20k monomers each), kappa 1-3.5, rho=0.85, mixed",
           "rounds": 30, "attempts_per_round": "M per melt", "eq15": "S = 1.6 exp(-0.77 kappa - 0.35 n)"}
    for name, flags in (("hastings", 0), ("paper_metropolis", kg.KG_FLAG_PAPER_METROPOLIS)):
        table, fit = measure_db_success(kg, torch, DBS_KAPPAS, DBS_STAGES, 30, flags)
        out[name] = {"table": table, "fit": fit}
        log(f"db success {name}: fit a {fit['a']:.3f} b {fit['b']:.3f} d {fit['d']:.3f}")
    print(json.dumps({"db_success": out}))


def ncu_case(args):
    """A short run for kernel captures: the 1.6M-monomer melt, no prelude,
    seven steps at dt = 0.001 of the stage --ncu-n (default n = 2).  The
    first step after the load runs alone and is followed by the re-sort into
    its cell order, so the second step's binning, list build and step kernel
    (launches 4-6 of those three kernels) run on the sorted state with few
    launches before them; the inputs stay larger than L2."""
    import torch

    import paper_2109_11001_gb300 as kg
    m = make_melt(args.workload, 0)
    prec = kg.KG_MIXED if args.precision == "mixed" else kg.KG_FP64
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=prec, seed=11,
                       fene_qmin=FENE_QMIN, sort_interval=3, skin=args.skin)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    kg.kg_set_potential_schedule(ctx, [kg.stage(args.ncu_n, 10 ** 9, 0.001)])
    kg.kg_load_config(ctx, 0, m.x, m.v)
    kg.kg_step(ctx, 7)          # step 1 alone, the re-sort, then a build on the sorted state
    st = kg.kg_db_sweep(ctx, args.ncu_db_budget)
    torch.cuda.synchronize()
    kg.kg_destroy(ctx)
    print(json.dumps({"ncu_case": args.workload, "M": m.M, "db_accepted": st.accepted}))


def ppa_case(args):
    """A run for primitive-path captures: the 1.6M-monomer melt relaxed
    through the prelude walk, then kg_primitive_path (mixed) of 0 and
    --ppa-case steps, the second between cudaProfilerStart/Stop (for ncu
    --profile-from-start off); below 50 steps every launch is direct."""
    import torch

    import paper_2109_11001_gb300 as kg
    m = make_melt(args.workload, 0)
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=kg.KG_MIXED, seed=11,
                       fene_qmin=FENE_QMIN, skin=0.5)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    stages, n_prelude = prelude_stages(kg)
    kg.kg_set_potential_schedule(ctx, stages)
    kg.kg_load_config(ctx, 0, m.x, m.v)
    kg.kg_step(ctx, n_prelude)
    kg.kg_primitive_path(ctx, 0, m.n_chains, 0, dt=0.005, gamma=1.0, skin=0.3)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    lpp, res = kg.kg_primitive_path(ctx, 0, m.n_chains, args.ppa_case, dt=0.005, gamma=1.0, skin=0.3)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    kg.kg_destroy(ctx)
    print(json.dumps({"ppa_case": args.workload, "M": m.M, "steps": args.ppa_case, **res}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg5", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-secondary", dest="secondary", action="store_false")
    ap.add_argument("--skin", type=float, default=0.3, help="skin when not autotuned")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--sort-interval", type=int, default=0, help="MD steps between re-sorts (0: library default)")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the direct-launch window (same bench steps, no graphs) with cudaProfilerStart/Stop, for ncu --profile-from-start off")
    ap.add_argument("--ncu-case", action="store_true")
    ap.add_argument("--ncu-db-budget", type=float, default=1e-3, help="DB attempts per monomer in the --ncu-case sweep")
    ap.add_argument("--ncu-n", type=float, default=2.0, help="stage exponent n of the --ncu-case steps")
    ap.add_argument("--ppa-case", type=int, default=0, help="primitive-path steps of a capture run (0: off)")
    ap.add_argument("--batched", action="store_true", help="run only the batched kappa-scan comparison")
    ap.add_argument("--equilibration", action="store_true",
                    help="run only the equilibrated-melts-per-hour comparison and print its JSON")
    ap.add_argument("--db-success", action="store_true",
                    help="measure the DB success rate per admissible attempt over kappa and n against Eq. 15")
    args = ap.parse_args()
    if args.ncu_case:
        ncu_case(args)
        return
    if args.ppa_case:
        ppa_case(args)
        return
    if args.db_success:
        db_success(args)
        return
    if args.batched:
        import torch

        import paper_2109_11001_gb300 as kg
        print(json.dumps({"batched": batched_secondary(kg, torch, args, 0)}))
        return
    if args.equilibration:
        import torch

        import paper_2109_11001_gb300 as kg
        print(json.dumps({"equilibration": equilibration_secondary(kg, torch, args, 0)}))
        return
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
