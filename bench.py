#!/usr/bin/env python3
"""Benchmark: pairwise interactions/s of the direct-summation force path.

Workload: two Plummer spheres of 524 288 particles each (N = 1 048 576) on a
head-on approach (centres at x = -5 and +5, relative speed 0.5), Henon units,
eps = 1e-3, FP32-compensated pairwise arithmetic with FP64 positions and
velocities.  One bench step is one full kick-drift-kick leapfrog step through
``nbody_step`` (replayed CUDA graph): kick + drift, Morton reordering, tile
packing, the force kernel with the fused closing kick, and the per-step energy
and momentum diagnostics.  Every step evaluates N^2 pairwise interactions.

Output: one JSON line on rank 0.  ``value`` is N^2 * steps * ranks / device
time of the timed steps (each step bracketed by CUDA events on the launching
stream, L2 flushed between steps by writing a 512 MiB buffer outside the timed
events).  ``roofline`` reports the force kernel against the FP32-pipe bound
(13 FP32 operations per pair on 128 FP32 lanes per SM, at the maximum SM
clock).  ``cpu_baseline`` times the FP64 oracle on a bounded sample of rows on
the host cores.  ``e2e`` repeats the steps through the same C ABI call with
pinned host buffers (host<->device copies inside the timed region).

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(bounded row samples per step), since the paper ships no runnable code.

With torchrun (N > 1) every rank integrates its own independent copy of the
workload (replicas; the force path has no data exchange between systems), the
steps are bracketed by a barrier, and the slowest rank's time is used.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("pairwise interactions/s and % of FP32/rsqrt roofline at N=1M, "
          "vs FP64 GPU at stated error")
UNIT = "interactions/s"
N_EACH = 524288
EPS = 1.0e-3
DT = 1.0e-4
SEED = 5
FP32_OPS_PER_PAIR = 13      # 3 add (dx), 3 fma (r^2), 3 mul, 1 add (phi), 3 fma (a)
JERK_OPS_PER_PAIR = 27      # + 3 add (u), 3 (r.u), 2 mul (beta), 6 fma (jerk)
PAPER_N = 102400            # the paper's run: 102 400 particles, ten time cycles (Sec. 4)
PAPER_SECONDS = {"wormhole_n300": 301.40, "cpu_2x_epyc_9124_32_threads": 672.90}
FP32_LANES_PER_SM = 128
MUFU_PER_SM = 16
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "force_kernel_traffic.json")
FORCE_SRC = os.path.join(ROOT, "paper_2509_19294_gb300", "csrc", "forces_f32c.cuh")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_name(n: int) -> str:
    return (f"two Plummer spheres head-on, N={n} (2x{n // 2}), eps=1e-3, KDK dt=1e-4, "
            "Morton reorder + pack + force + kick + diagnostics per step")


def workload(n_each=N_EACH):
    from paper_2509_19294_gb300 import ic
    return ic.two_plummer(n_each, seed=SEED)


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's value (the bench times every rank and keeps the max)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, seconds: float) -> float:
    """Units processed by all ranks over the timed steps / the slowest rank's time."""
    return units_per_rank_step * steps * world / seconds


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle_rows(pos, mass, budget_s, seed):
    """FP64 oracle on random rows against all j, sized to ~budget_s of CPU."""
    import oracle
    from paper_2509_19294_gb300 import ic
    n = mass.shape[0]
    rows = ic.sample_rows(n, 64, seed)
    t0 = time.perf_counter()
    oracle.forces_rows(pos, mass, EPS, rows)
    t1 = time.perf_counter()
    per_row = (t1 - t0) / len(rows)
    k = int(max(64, min(n, budget_s / max(per_row, 1e-9))))
    rows = ic.sample_rows(n, k, seed + 1)
    t0 = time.perf_counter()
    oracle.forces_rows(pos, mass, EPS, rows)
    t1 = time.perf_counter()
    return len(rows) * n / (t1 - t0), len(rows), t1 - t0, oracle.num_threads()


def host_cpu():
    """CPU model and usable cores of this host (for the CPU-baseline record)."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:  # Arm hosts: /proc/cpuinfo has no model name, lscpu does
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    return {"model": model or platform.processor() or platform.machine(), "arch": platform.machine(),
            "cores_usable": cores}


def time_oracle_configs():
    """One full FP64 oracle evaluation at the smaller workloads (C1 N=1024,
    C2 N=16384 uniform sphere with log-uniform masses, C3 N=131072), as
    context for the sampled rate at N=1M."""
    import oracle
    from paper_2509_19294_gb300 import ic
    out = {}
    cases = [("C1 Plummer N=1024", lambda: (ic.plummer(1024, seed=1)[0], np.full(1024, 1.0 / 1024), 0.01)),
             ("C2 uniform sphere N=16384, log-uniform masses",
              lambda: (ic.uniform_sphere(16384, seed=2)[0], ic.log_uniform_masses(16384, seed=2), 0.005)),
             ("C3 Plummer N=131072", lambda: (ic.plummer(131072, seed=3)[0], np.full(131072, 1.0 / 131072),
                                               1e-3))]
    for name, make in cases:
        pos, mass, eps = make()
        n = mass.shape[0]
        t0 = time.perf_counter()
        oracle.forces(pos, mass, eps)
        sec = time.perf_counter() - t0
        out[name] = {"seconds": sec, "interactions_per_s": float(n) * n / sec}
    return out


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                try:
                    pw.append(float(parts[2]))
                except ValueError:
                    pass
                for name, val in zip(self.NAMES, parts[4:8]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_mean": statistics.fmean(pw) if pw else None,
                "power_w_max": max(pw) if pw else None}


def traffic_for_current_kernel(tiles):
    """DRAM bytes per force launch from the committed ncu summary, if it was
    taken on the kernel source as it is now and with the same tile shape and
    split (else null)."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
        with open(FORCE_SRC, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        for r in rec.get("records", [rec]):
            if r.get("source_sha256") == sha and list(r.get("tiles", [])) == list(tiles):
                return r.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


# ----------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import paper_2509_19294_gb300 as nb
    from paper_2509_19294_gb300 import build as nbuild

    rank, world, local = dist_env()
    if rank == 0 and not nbuild.up_to_date():
        nbuild.build()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
        pg.barrier()            # the other ranks wait for rank 0's build
    nb.load()

    pos, vel, mass = workload(args.n_each)
    n = mass.shape[0]
    pairs_per_step = float(n) * n
    stream = torch.cuda.current_stream()

    flags = nb.NBODY_FLAG_PROFILE
    forced = tuple(int(x) for x in args.tiles.split(",")) if args.tiles else None
    if forced is None:
        flags |= nb.NBODY_FLAG_AUTOTUNE
    ctx = nb.nbody_init(n, EPS, mode=nb.NBODY_F32C, reorder_every=1, flags=flags, tiles=forced)
    tiles = nb.nbody_get_tiles(ctx)
    p = torch.from_numpy(pos).cuda()
    v = torch.from_numpy(vel).cuda()
    m = torch.from_numpy(mass).cuda()
    acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    diag = torch.empty((1, 1, 9), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    nb.nbody_forces(ctx, p, m, acc, pot)
    for _ in range(args.warmup):
        nb.nbody_step(ctx, p, v, m, acc, pot, DT, 1, diag)
    torch.cuda.synchronize()
    e_first = nb.nbody_energy(ctx, p, v, m, pot)[0]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    nb.nbody_profile_read(ctx, reset=True)
    launches0 = nb.nbody_kernel_launches(ctx)
    visible = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    sampler = ClockSampler(visible[local] if local < len(visible) else local)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                                   # L2 flush, outside the events
        ev[k][0].record(stream)
        nb.nbody_step(ctx, p, v, m, acc, pot, DT, 1, diag)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    wall1 = time.perf_counter()
    clocks = sampler.stop()
    launches = nb.nbody_kernel_launches(ctx) - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_total = float(sum(step_ms))
    kern_ms, kern_n = nb.nbody_profile_read(ctx, reset=True)
    e_last = nb.nbody_energy(ctx, p, v, m, pot)[0]
    ms_total = max_over_ranks(ms_total, pg, device="cuda")

    # accuracy of the timed configuration: sampled rows against the FP64 oracle
    # (the state after the timed steps; rows computed one by one on the host)
    accuracy = None
    cpu = None
    if rank == 0:
        import oracle
        from paper_2509_19294_gb300 import ic
        ph = p.cpu().numpy()
        mh = m.cpu().numpy()
        nb.nbody_forces(ctx, p, m, acc, pot)
        ah = acc.cpu().numpy()
        poth = pot.cpu().numpy()
        rows = ic.sample_rows(n, 512, 99)
        ra, rp = oracle.forces_rows(ph, mh, EPS, rows)
        ga = ah[:, rows]
        rel = np.linalg.norm(ga - ra, axis=0) / np.linalg.norm(ra, axis=0)
        typical = math.sqrt(float(np.mean(np.sum(ra ** 2, axis=0))))
        own = np.linalg.norm(ra, axis=0)
        accuracy = {
            "rows": int(len(rows)),
            "median_rel_acc_err": float(np.median(rel)),
            "max_rel_acc_err": float(rel.max()),
            "paper_metric_component_over_own_norm": float((np.abs(ga - ra).max(axis=0) / own).max()),
            "paper_metric_component_over_rms": float(np.abs(ga - ra).max() / typical),
            "max_rel_pot_err": float((np.abs(poth[rows] - rp) / np.abs(rp)).max()),
            "dE_over_E_timed_steps": float(abs(e_last[2] - e_first[2]) / abs(e_first[2])),
        }
        if not args.no_cpu_baseline:
            val, nrows, secs, thr = time_oracle_rows(ph, mh, args.cpu_seconds, 7)
            cpu = {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle",
                   "sample": f"{nrows} random rows x all {n} particles of the same state "
                             f"(FP64, {secs:.1f} s on {thr} threads)",
                   "full_evaluations": time_oracle_configs(), "host": host_cpu()}

    # plain FP64 GPU kernel on the same GPU and the same state: one full
    # evaluation of the timed workload (N = 1M: about 48 s), and the F32C
    # result of that state against it on every row
    fp64 = None
    if rank == 0 and not args.no_fp64:
        fp64 = fp64_comparison(nb, torch, p, m, ah, poth, args.fp64_n)

    # |dE/E| drift of the FP32C path against the FP64 GPU path over the same
    # steps: C4 (512 clusters, 100 steps, per cluster) and C3 (N = 131072,
    # 1000 steps; about 12 minutes of FP64 work)
    drift = None
    if rank == 0 and world == 1 and not args.no_drift:
        drift = {"c4": c4_drift(nb, torch)}
        if not args.no_c3_drift:
            drift["c3"] = c3_drift(nb, torch, args.c3_steps)

    # F32C force evaluations across the workloads' sizes (autotuned tiles)
    sweep = None
    if rank == 0 and world == 1 and not args.no_sweep:
        sweep = force_sweep(nb, torch)

    # batched ensemble: 512 independent Plummer clusters, one persistent launch per step
    ensemble = None
    if rank == 0 and not args.no_ensemble:
        from paper_2509_19294_gb300 import ic
        ens = ic.ensemble(512, seed=4)
        ne = ens.mass.shape[0]
        pairs_e = float((ens.sizes.astype(np.float64) ** 2).sum())
        with nb.nbody_init(ne, ens.eps, cluster_offsets=ens.offsets, reorder_every=10,
                           flags=nb.NBODY_FLAG_PROFILE | nb.NBODY_FLAG_AUTOTUNE) as ce:
            pe, ve, me = (torch.from_numpy(x.copy()).cuda() for x in (ens.pos, ens.vel, ens.mass))
            ae = torch.empty((3, ne), dtype=torch.float64, device="cuda")
            poe = torch.empty(ne, dtype=torch.float64, device="cuda")
            de = torch.empty((100, 512, 9), dtype=torch.float64, device="cuda")
            nb.nbody_forces(ce, pe, me, ae, poe)
            nb.nbody_step(ce, pe, ve, me, ae, poe, 1e-3, 5)
            torch.cuda.synchronize()
            nb.nbody_profile_read(ce, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nb.nbody_step(ce, pe, ve, me, ae, poe, 1e-3, 100, de)
            e1.record(stream)
            torch.cuda.synchronize()
            ems = e0.elapsed_time(e1)
            kms, kn = nb.nbody_profile_read(ce, reset=True)
            et = nb.nbody_get_tiles(ce)
        ensemble = {"workload": "512 Plummer clusters, N_c ~ U{256..8192} (seed 4), "
                                "eps_c = 0.01 N_c^(-1/3), 100 KDK steps dt=1e-3, reorder every 10",
                    "n_total": int(ne), "pairs_per_step": pairs_e,
                    "value": pairs_e * 100 / (ems / 1e3), "unit": UNIT,
                    "ms_per_step": ems / 100, "force_kernel_ms": kms / max(kn, 1),
                    "tiles": {"block": et[0], "p": et[1], "tj": et[2], "split": et[3],
                              "ctas_per_sm": et[4]}}

    # the paper's workload size with its force payload (acceleration + jerk):
    # N = 102 400 Plummer sphere, ten fourth-order Hermite steps
    paper_scale = None
    if rank == 0 and not args.no_paper_scale:
        from paper_2509_19294_gb300 import ic
        pp_, pv_, pm_ = ic.plummer(PAPER_N, seed=6)
        with nb.nbody_init(PAPER_N, 1e-3, mode=nb.NBODY_F32C, reorder_every=1,
                           flags=nb.NBODY_FLAG_PROFILE) as cj:
            p_, v_, m_ = (torch.from_numpy(x.copy()).cuda() for x in (pp_, pv_, pm_))
            a_ = torch.empty((3, PAPER_N), dtype=torch.float64, device="cuda")
            j_ = torch.empty((3, PAPER_N), dtype=torch.float64, device="cuda")
            po_ = torch.empty(PAPER_N, dtype=torch.float64, device="cuda")
            nb.nbody_forces_jerk(cj, p_, v_, m_, a_, j_, po_)
            nb.nbody_step_hermite(cj, p_, v_, m_, a_, j_, po_, 1e-4, 3)   # warm-up, graph capture
            torch.cuda.synchronize()
            nb.nbody_profile_read(cj, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nb.nbody_step_hermite(cj, p_, v_, m_, a_, j_, po_, 1e-4, 10)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            jms, jn = nb.nbody_profile_read(cj, reset=True)
            jt = nb.nbody_get_jerk_tiles(cj)
        pairs_j = float(PAPER_N) ** 2
        paper_scale = {
            "workload": "Plummer sphere N=102400 (seed 6), eps=1e-3, 10 Hermite steps dt=1e-4, "
                        "acceleration + jerk each step (Morton reorder, pack, predictor, "
                        "force+jerk kernel, corrector)",
            "seconds_10_steps": sec, "interactions_per_s": pairs_j * 10 / sec,
            "force_jerk_kernel_ms": jms / max(jn, 1),
            "tiles": {"block": jt[0], "p": jt[1], "tj": jt[2], "split": jt[3], "ctas_per_sm": jt[4]},
            "paper_time_to_solution_s": PAPER_SECONDS,
            "note": "context only: the paper's times are whole-application runs of its own code "
                    "and initial conditions on other hardware (Sec. 4)"}

    # individual (block) time steps on the paper's particle count: timed without
    # profiling events (steps then replay several to a graph), and run again
    # with them for the force-pass time (the same deterministic trajectory)
    block = None
    if rank == 0 and not args.no_block_steps:
        from paper_2509_19294_gb300 import ic
        bp_, bv_, bm_ = ic.plummer(PAPER_N, seed=7)

        def block_run(flags):
            with nb.nbody_init(PAPER_N, 1e-3, mode=nb.NBODY_F32C, reorder_every=4, flags=flags) as cb:
                p_, v_, m_ = (torch.from_numpy(x.copy()).cuda() for x in (bp_, bv_, bm_))
                a_ = torch.empty((3, PAPER_N), dtype=torch.float64, device="cuda")
                j_ = torch.empty((3, PAPER_N), dtype=torch.float64, device="cuda")
                po_ = torch.empty(PAPER_N, dtype=torch.float64, device="cuda")
                nb.nbody_block_start(cb, p_, v_, m_, a_, j_, po_, 2.0 ** -7, 2.0 ** -22, 0.02, 0.01)
                b0, e0_ = nb.nbody_block_advance(cb, p_, v_, m_, a_, j_, po_, 2.0 ** -7)  # warm-up
                torch.cuda.synchronize()
                if flags:
                    nb.nbody_profile_read(cb, reset=True)
                t0 = time.perf_counter()
                b1, e1_ = nb.nbody_block_advance(cb, p_, v_, m_, a_, j_, po_, 2.0 ** -4)
                torch.cuda.synchronize()
                sec = time.perf_counter() - t0
                kms = nb.nbody_profile_read(cb, reset=True)[0] if flags & nb.NBODY_FLAG_PROFILE else None
                trace = nb.nbody_block_trace(cb, b0 + 1, b1) if flags & nb.NBODY_FLAG_TRACE else None
                _, dts = nb.nbody_block_state(cb)
            return b1 - b0, e1_ - e0_, sec, kms, dts, trace

        # the timed run records each step's start and size on the device (one
        # thread's timer read and two stores a step)
        blocks, evals, sec, _, dts, trace = block_run(nb.NBODY_FLAG_TRACE)
        blocks_p, evals_p, sec_p, kms, _, _ = block_run(nb.NBODY_FLAG_PROFILE)
        step_s, step_n = trace
        regimes = {}
        for name, lo, hi in (("few_particle_le_32", 1, 32), ("small_set_33_511", 33, 511),
                             ("large_set_ge_512", 512, 1 << 62), ("one_active", 1, 1)):
            sel = (step_n >= lo) & (step_n <= hi)
            if sel.any():
                regimes[name] = {"steps": int(sel.sum()), "seconds": float(step_s[sel].sum()),
                                 "median_step_us": float(np.median(step_s[sel]) * 1e6),
                                 "interactions_per_s": float(step_n[sel].sum() * float(PAPER_N)
                                                             / step_s[sel].sum())}
        block = {"workload": "Plummer sphere N=102400 (seed 7), eps=1e-3, Hermite with individual "
                             "power-of-two steps (dt_max 2^-7, Aarseth eta 0.02) from t=2^-7 to 2^-4",
                 "block_steps": int(blocks), "particle_evaluations": int(evals),
                 "mean_active": evals / max(blocks, 1), "seconds": sec,
                 "interactions_per_s": evals * float(PAPER_N) / sec,
                 "subset_kernel_ms_total": kms,
                 "per_regime": regimes,
                 "per_regime_scope": "device trace (NBODY_FLAG_TRACE) of the timed run: a step runs "
                                     "from its pack's start to the next one's; by active particles "
                                     "(few-particle pass <= 32, small-set kernel < 512, large-set)",
                 "profiled_run": {"seconds": sec_p, "same_schedule": bool(blocks_p == blocks and
                                                                          evals_p == evals)},
                 "steps_histogram": {f"2^{int(round(np.log2(v)))}": int(c)
                                     for v, c in zip(*np.unique(dts, return_counts=True))},
                 "shared_step_equivalent_evaluations": int(blocks) * PAPER_N,
                 "subset_kernel_scope": "CUDA events around each step's force pass (in the profiled "
                                        "run): the few-particle or subset kernels, the split reduction "
                                        "and, fused into their epilogues, the Hermite corrector"}

    # end to end through the same C ABI call with pinned host buffers
    e2e = None
    if not args.no_e2e:
        ph = torch.from_numpy(pos.copy()).pin_memory()
        vh = torch.from_numpy(vel.copy()).pin_memory()
        mh = torch.from_numpy(mass.copy()).pin_memory()
        ah = torch.empty((3, n), dtype=torch.float64).pin_memory()
        poth = torch.empty(n, dtype=torch.float64).pin_memory()
        dh = torch.empty((1, 1, 9), dtype=torch.float64).pin_memory()
        with nb.nbody_init(n, EPS, mode=nb.NBODY_F32C, reorder_every=1,
                           tiles=tiles) as ce:
            nb.nbody_forces(ce, ph, mh, ah, poth)
            nb.nbody_step(ce, ph, vh, mh, ah, poth, DT, 1, dh)
            if pg:
                pg.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                nb.nbody_step(ce, ph, vh, mh, ah, poth, DT, 1, dh)   # H2D, step, D2H, sync
            torch.cuda.synchronize()
            t1 = time.perf_counter()
        secs = max_over_ranks(t1 - t0, pg, device="cuda")
        bi = 8 * (3 * n + 3 * n + n + 3 * n + n)
        bo = 8 * (3 * n + 3 * n + 3 * n + n + 9)
        e2e = {"value": whole_job_rate(pairs_per_step, args.steps, world, secs), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo}

    nb.nbody_destroy(ctx)
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    try:
        from paper_2509_19294_gb300 import probe
        rates = probe.measure_pipes()
    except RuntimeError:
        rates = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            sm_max = float(json.load(f).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        sm_max = 2070.0
    value = whole_job_rate(pairs_per_step, args.steps, world, ms_total / 1e3)
    kern_avg_s = kern_ms / max(kern_n, 1) / 1e3
    achieved = pairs_per_step / kern_avg_s / 1e9
    peak_fp32 = FP32_LANES_PER_SM * sms * sm_max * 1e6 / FP32_OPS_PER_PAIR / 1e9
    peak_mufu = MUFU_PER_SM * sms * sm_max * 1e6 / 1e9
    peak = min(peak_fp32, peak_mufu)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Ginteractions/s",
            "frac": achieved / peak, "traffic": traffic_for_current_kernel(tiles),
            "kernel": "forces_f32c_kernel", "avg_launch_ms": kern_avg_s * 1e3,
            "launches": kern_n,
            "peak_basis": f"FP32 pipe: {FP32_LANES_PER_SM} lanes/SM x {sms} SMs x {sm_max:.0f} MHz "
                          f"/ {FP32_OPS_PER_PAIR} FP32 ops per pair (MUFU bound "
                          f"{peak_mufu:.0f} G/s is looser); derived, not measured"}
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / sm_max)
    if rates:
        # measured per-SM-per-clock rates (clock64 cycles, one CTA of 1024 threads per SM)
        roof["measured_rates"] = rates
        roof["pair_arith_ceiling_frac"] = (rates["pair_arith_pairs_per_clk_sm"]
                                           / (FP32_LANES_PER_SM / FP32_OPS_PER_PAIR))
    if fp64 is not None:
        fp64["ratio_f32c_over_f64"] = value / fp64["value"]
    if sweep is not None:
        for rec in sweep:
            rec["roofline_frac"] = rec["kernel_interactions_per_s"] / 1e9 / peak
            rec["call_roofline_frac"] = rec["call_interactions_per_s"] / 1e9 / peak
    # energy to solution (the paper's second metric): GPU board power sampled by
    # nvidia-smi every 200 ms during the timed steps, times the timed wall time
    energy = None
    if clocks and clocks.get("power_w_mean"):
        joules = clocks["power_w_mean"] * (wall1 - wall0)
        energy = {"gpu_power_w_mean": clocks["power_w_mean"], "gpu_power_w_max": clocks["power_w_max"],
                  "joules_per_step": joules / args.steps,
                  "interactions_per_joule": pairs_per_step * args.steps / joules,
                  "scope": "GPU board power only (nvidia-smi power.draw), host excluded"}
    if paper_scale is not None:
        jpeak = FP32_LANES_PER_SM * sms * sm_max * 1e6 / JERK_OPS_PER_PAIR / 1e9
        jach = float(PAPER_N) ** 2 / (paper_scale["force_jerk_kernel_ms"] / 1e3) / 1e9
        paper_scale["jerk_roofline"] = {"achieved": jach, "peak": jpeak, "unit": "Ginteractions/s",
                                        "frac": jach / jpeak,
                                        "basis": f"{JERK_OPS_PER_PAIR} FP32 ops per pair"}
    if block is not None:
        jpeak = FP32_LANES_PER_SM * sms * sm_max * 1e6 / JERK_OPS_PER_PAIR / 1e9
        bk = block["particle_evaluations"] * float(PAPER_N) / (block["subset_kernel_ms_total"] / 1e3) / 1e9
        block["subset_kernel_roofline_frac"] = bk / jpeak
    if ensemble is not None:
        ek = ensemble["pairs_per_step"] / (ensemble["force_kernel_ms"] / 1e3) / 1e9
        ensemble["roofline_frac"] = ek / peak
        ensemble["step_frac"] = ensemble["value"] / 1e9 / peak
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
        "ms_per_step_median": float(np.median(step_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(n),
                   "n": n, "eps": EPS, "dt": DT, "seed": SEED,
                   "precision": "FP32 pairwise (MUFU rsqrt), Kahan-compensated FP32 tile sums, "
                                "FP64 positions/velocities/reduction",
                   "tiles": {"block": tiles[0], "p": tiles[1], "tj": tiles[2], "split": tiles[3],
                             "ctas_per_sm": tiles[4]},
                   "l2": "flushed between steps (512 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "fp64_gpu": fp64,
        "drift": drift,
        "sweep": sweep,
        "ensemble": ensemble,
        "paper_scale": paper_scale,
        "block_steps": block,
        "energy": energy,
        "accuracy": accuracy,
        "clocks": clocks,
        "wall_s_timed": wall1 - wall0,
    }
    print(json.dumps(out), flush=True)
    if pg:
        pg.destroy_process_group()


# ----------------------------------------------------------------- comparisons

def fp64_comparison(nb, torch, p, m, a32, p32, n64=0):
    """The plain FP64 GPU kernel on the timed workload's state (all N rows; n64 > 0
    evaluates only the first n64 particles as their own system instead), its
    interactions/s, and the F32C acceleration/potential of that state (a32, p32,
    host arrays) against it row by row."""
    n = int(m.shape[0]) if not n64 else int(n64)
    pp = p if not n64 else p[:, :n].contiguous()
    mm = m if not n64 else m[:n].contiguous()
    with nb.nbody_init(n, EPS, mode=nb.NBODY_F64, flags=nb.NBODY_FLAG_PROFILE) as c64:
        aa = torch.empty((3, n), dtype=torch.float64, device="cuda")
        po = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_profile_read(c64, reset=True)
        nb.nbody_forces(c64, pp, mm, aa, po)
        ms64, _ = nb.nbody_profile_read(c64, reset=True)
        a64, q64 = aa.cpu().numpy(), po.cpu().numpy()
    out = {"value": float(n) * n / (ms64 / 1e3), "unit": UNIT, "kernel_ms": ms64,
           "sample": f"one full FP64 evaluation of the timed workload's state, N={n}",
           "ratio_f32c_over_f64": None}
    if not n64:
        rel = np.linalg.norm(a32 - a64, axis=0) / np.linalg.norm(a64, axis=0)
        typical = math.sqrt(float(np.mean(np.sum(a64 ** 2, axis=0))))
        prel = np.abs(p32 - q64) / np.abs(q64)
        out["f32c_vs_f64_all_rows"] = {
            "rows": n, "median_rel_acc_err": float(np.median(rel)), "max_rel_acc_err": float(rel.max()),
            "paper_metric_component_over_own_norm": float(
                (np.abs(a32 - a64).max(axis=0) / np.linalg.norm(a64, axis=0)).max()),
            "paper_metric_component_over_rms": float(np.abs(a32 - a64).max() / typical),
            "median_rel_pot_err": float(np.median(prel)), "max_rel_pot_err": float(prel.max())}
    return out


def _run_with_diag(nb, torch, pos, vel, mass, eps, dt, nsteps, mode, offsets=None, reorder=10):
    """Energies of every cluster at t = 0 and after each of nsteps graph-replayed
    KDK steps ([nsteps + 1, clusters, 9]) and the device seconds of the steps."""
    n = mass.shape[0]
    with nb.nbody_init(n, eps, mode=mode, cluster_offsets=offsets, reorder_every=reorder) as ctx:
        pt, vt, mt = (torch.from_numpy(x.copy()).cuda() for x in (pos, vel, mass))
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, pt, mt, acc, pot)
        e0 = nb.nbody_energy(ctx, pt, vt, mt, pot)
        d = torch.empty((nsteps, ctx.n_clusters, 9), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        nb.nbody_step(ctx, pt, vt, mt, acc, pot, dt, nsteps, d)
        ev1.record(stream)
        torch.cuda.synchronize()
        return np.concatenate([e0[None], d.cpu().numpy()]), ev0.elapsed_time(ev1) / 1e3


def _drift(e):
    """max over steps of |E(t) - E(0)| / |E(0)| per cluster, E with each path's own phi."""
    return np.abs(e[:, :, 2] - e[0, :, 2]).max(axis=0) / np.abs(e[0, :, 2])


def c4_drift(nb, torch):
    from paper_2509_19294_gb300 import ic
    ens = ic.ensemble(512, seed=4)
    res = {}
    for name, mode in (("f32c", nb.NBODY_F32C), ("f64", nb.NBODY_F64)):
        e, sec = _run_with_diag(nb, torch, ens.pos, ens.vel, ens.mass, ens.eps, 1e-3, 100, mode,
                                offsets=ens.offsets)
        res[name] = (_drift(e), sec, np.abs(e[:, :, 3:6] - e[0, :, 3:6]).max(axis=(0, 2)))
    ratio = res["f32c"][0] / res["f64"][0]
    worst = int(np.argmax(ratio))
    return {"workload": "C4 ensemble, 512 clusters (seed 4), 100 KDK steps dt=1e-3, both paths "
                        "from the same initial state, E with each path's own potential",
            "per_cluster_ratio": {"max": float(ratio.max()), "median": float(np.median(ratio)),
                                  "clusters_above_2": int((ratio > 2).sum())},
            "worst_cluster": {"cluster": worst, "n_c": int(ens.sizes[worst]),
                              "f32c": float(res["f32c"][0][worst]), "f64": float(res["f64"][0][worst])},
            "f32c_max_abs_dE_over_E": float(res["f32c"][0].max()),
            "f64_max_abs_dE_over_E": float(res["f64"][0].max()),
            "f64_median_abs_dE_over_E": float(np.median(res["f64"][0])),
            "max_abs_dP": {"f32c": float(res["f32c"][2].max()), "f64": float(res["f64"][2].max())},
            "seconds": {"f32c": res["f32c"][1], "f64": res["f64"][1]}}


def c3_drift(nb, torch, nsteps=1000):
    from paper_2509_19294_gb300 import ic
    pos, vel, mass = ic.plummer(131072, seed=3)
    res = {}
    for name, mode in (("f32c", nb.NBODY_F32C), ("f64", nb.NBODY_F64)):
        e, sec = _run_with_diag(nb, torch, pos, vel, mass, 1e-3, 1e-4, nsteps, mode)
        res[name] = {"max_abs_dE_over_E": float(_drift(e)[0]),
                     "max_abs_dP": float(np.abs(e[:, 0, 3:6] - e[0, 0, 3:6]).max()),
                     "max_abs_dL": float(np.abs(e[:, 0, 6:9] - e[0, 0, 6:9]).max()),
                     "seconds": sec}
    return {"workload": f"C3 Plummer N=131072 (seed 3), eps=1e-3, {nsteps} graph-replayed KDK steps "
                        "dt=1e-4, Morton re-sort every 10, both paths from the same initial state, "
                        "E with each path's own potential",
            "steps": nsteps, "f32c": res["f32c"], "f64": res["f64"],
            "ratio_f32c_over_f64": res["f32c"]["max_abs_dE_over_E"] / res["f64"]["max_abs_dE_over_E"]}


def force_sweep(nb, torch):
    """nbody_forces (F32C, autotuned tiles) at the workloads' sizes: kernel-only
    and whole-call (pack + queue reset + force kernel) interactions/s."""
    from paper_2509_19294_gb300 import ic
    cases = [("C1 Plummer N=1024, eps=0.01", lambda: ic.plummer(1024, seed=1), 0.01),
             ("C2 uniform sphere N=16384, log-uniform masses, eps=0.005",
              lambda: ic.uniform_sphere(16384, seed=2, masses=ic.log_uniform_masses(16384, seed=2)), 0.005),
             ("C2 Plummer N=16384, log-uniform masses, eps=0.005",
              lambda: ic.plummer(16384, seed=2, masses=ic.log_uniform_masses(16384, seed=2)), 0.005),
             ("C3 Plummer N=131072, eps=1e-3", lambda: ic.plummer(131072, seed=3), 1e-3),
             ("C5 two Plummer spheres N=1048576, eps=1e-3", lambda: ic.two_plummer(N_EACH, seed=SEED), 1e-3)]
    out = []
    stream = torch.cuda.current_stream()
    for name, make, eps in cases:
        pos, _, mass = make()
        n = mass.shape[0]
        reps = int(min(200, max(3, 2e12 / (float(n) * n))))
        with nb.nbody_init(n, eps, flags=nb.NBODY_FLAG_PROFILE | nb.NBODY_FLAG_AUTOTUNE) as ctx:
            pt, mt = torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda()
            acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
            pot = torch.empty(n, dtype=torch.float64, device="cuda")
            for _ in range(3):
                nb.nbody_forces(ctx, pt, mt, acc, pot)
            torch.cuda.synchronize()
            nb.nbody_profile_read(ctx, reset=True)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(reps):
                nb.nbody_forces(ctx, pt, mt, acc, pot)
            ev1.record(stream)
            torch.cuda.synchronize()
            call_s = ev0.elapsed_time(ev1) / 1e3 / reps
            kms, kn = nb.nbody_profile_read(ctx, reset=True)
            t = nb.nbody_get_tiles(ctx)
        kern_s = kms / max(kn, 1) / 1e3
        out.append({"workload": name, "n": int(n), "evaluations": reps,
                    "kernel_ms": kern_s * 1e3, "call_ms": call_s * 1e3,
                    "kernel_interactions_per_s": float(n) * n / kern_s,
                    "call_interactions_per_s": float(n) * n / call_s,
                    "tiles": {"block": t[0], "p": t[1], "tj": t[2], "split": t[3], "ctas_per_sm": t[4]},
                    "l2": "inputs resident (j-set 16 B/particle); no flush between evaluations"})
    return out


# ----------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2509_19294_gb300 import ic
    oracle.build()
    pos, vel, mass = workload()
    n = mass.shape[0]
    # each step: the oracle's force rows on a bounded sample (sized so that
    # warmup + steps stay within a few minutes on the host cores)
    per_step_s = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    val0, nrows, _, thr = time_oracle_rows(pos, mass, per_step_s, 11)
    for w in range(args.warmup):
        oracle.forces_rows(pos, mass, EPS, ic.sample_rows(n, nrows, 100 + w))
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.forces_rows(pos, mass, EPS, ic.sample_rows(n, nrows, 200 + k))
    secs = time.perf_counter() - t0
    value = nrows * n * args.steps / secs
    sample = f"{nrows} random rows x all {n} particles per step (FP64 oracle, {thr} threads)"
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(n), "n": n, "eps": EPS, "dt": DT, "seed": SEED,
                   "parallelism": "host cores",
                   "reference_step": "FP64 oracle forces of a bounded random sample of rows "
                                     "against all N particles (the full O(N^2) step would take "
                                     "~11 minutes on the host cores)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_block_drift(n, t_end):
    """Energy drift of block steps, F32C against the FP64 path: a Plummer sphere
    of n (seed 8), eps 1e-3, dt_max 2^-7, advanced dt_max per call to t_end,
    E from nbody_energy after every call with each path's own potential, and
    with an FP64 potential of the same states (separating the integration from
    the potential's rounding).  Prints one JSON line."""
    import torch
    import paper_2509_19294_gb300 as nb
    from paper_2509_19294_gb300 import build as nbuild
    from paper_2509_19294_gb300 import ic
    if not nbuild.up_to_date():
        nbuild.build()
    pos, vel, mass = ic.plummer(n, seed=8)
    dt_max = 2.0 ** -7
    res = {}
    c64 = nb.nbody_init(n, 1e-3, mode=nb.NBODY_F64)  # the same states' energy with an FP64 potential
    a64 = torch.empty((3, n), dtype=torch.float64, device="cuda")
    p64 = torch.empty(n, dtype=torch.float64, device="cuda")

    def energy_fp64(p_, v_, m_):
        nb.nbody_forces(c64, p_, m_, a64, p64)
        return nb.nbody_energy(c64, p_, v_, m_, p64)[0][2]

    for name, mode in (("f32c", nb.NBODY_F32C), ("f64", nb.NBODY_F64)):
        with nb.nbody_init(n, 1e-3, mode=mode, reorder_every=4) as cb:
            p_, v_, m_ = (torch.from_numpy(x.copy()).cuda() for x in (pos, vel, mass))
            a_ = torch.empty((3, n), dtype=torch.float64, device="cuda")
            j_ = torch.empty((3, n), dtype=torch.float64, device="cuda")
            po_ = torch.empty(n, dtype=torch.float64, device="cuda")
            nb.nbody_block_start(cb, p_, v_, m_, a_, j_, po_, dt_max, 2.0 ** -22, 0.02, 0.01)
            e0 = nb.nbody_energy(cb, p_, v_, m_, po_)[0][2]
            f0 = energy_fp64(p_, v_, m_)
            worst, worst64, k, blocks, evals, sec = 0.0, 0.0, 0, 0, 0, 0.0
            while (k + 1) * dt_max <= t_end:
                k += 1
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                blocks, evals = nb.nbody_block_advance(cb, p_, v_, m_, a_, j_, po_, k * dt_max)
                e = nb.nbody_energy(cb, p_, v_, m_, po_)[0][2]
                sec += time.perf_counter() - t0
                worst = max(worst, abs(e - e0) / abs(e0))
                worst64 = max(worst64, abs(energy_fp64(p_, v_, m_) - f0) / abs(f0))
            res[name] = {"block_steps": int(blocks), "particle_evaluations": int(evals),
                         "max_abs_dE_over_E": worst, "max_abs_dE_over_E_fp64_potential": worst64,
                         "seconds": sec, "pos": p_.cpu().numpy()}
    nb.nbody_destroy(c64)
    dx = np.abs(res["f32c"].pop("pos") - res["f64"].pop("pos")).max(axis=0)
    print(json.dumps({"block_drift": {
        "workload": f"Plummer sphere N={n} (seed 8), eps=1e-3, block steps dt_max 2^-7 (eta 0.02), "
                    f"t=0..{t_end}, one advance call per dt_max, re-sort every 4 dt_max",
        "f32c": res["f32c"], "f64": res["f64"],
        "drift_ratio_f32c_over_f64": res["f32c"]["max_abs_dE_over_E"] / res["f64"]["max_abs_dE_over_E"],
        "drift_ratio_fp64_potential": (res["f32c"]["max_abs_dE_over_E_fp64_potential"] /
                                       res["f64"]["max_abs_dE_over_E_fp64_potential"]),
        "final_position_difference": {"median": float(np.median(dx)), "max": float(dx.max())}}}))


def run_c5_drift(nsteps):
    """C5 over nsteps KDK steps, F32C against the plain FP64 GPU path from the
    same initial state: |dE/E| (each path's own potential), |dP|, and the final
    positions' difference.  Prints one JSON line (10 steps take ~9 minutes of
    FP64 work)."""
    import torch
    import paper_2509_19294_gb300 as nb
    from paper_2509_19294_gb300 import build as nbuild
    if not nbuild.up_to_date():
        nbuild.build()
    pos, vel, mass = workload()
    n = mass.shape[0]
    res = {}
    for name, mode in (("f32c", nb.NBODY_F32C), ("f64", nb.NBODY_F64)):
        with nb.nbody_init(n, EPS, mode=mode, reorder_every=1) as ctx:
            p_, v_, m_ = (torch.from_numpy(x.copy()).cuda() for x in (pos, vel, mass))
            a_ = torch.empty((3, n), dtype=torch.float64, device="cuda")
            po_ = torch.empty(n, dtype=torch.float64, device="cuda")
            t0 = time.perf_counter()
            nb.nbody_forces(ctx, p_, m_, a_, po_)
            e0 = nb.nbody_energy(ctx, p_, v_, m_, po_)
            d = torch.empty((nsteps, 1, 9), dtype=torch.float64, device="cuda")
            nb.nbody_step(ctx, p_, v_, m_, a_, po_, DT, nsteps, d)
            e = np.concatenate([e0[None], d.cpu().numpy()])[:, 0]
            res[name] = {"max_abs_dE_over_E": float(np.abs(e[:, 2] - e[0, 2]).max() / abs(e[0, 2])),
                         "max_abs_dP": float(np.abs(e[:, 3:6] - e[0, 3:6]).max()),
                         "E": e[:, 2].tolist(), "seconds": time.perf_counter() - t0,
                         "pos": p_.cpu().numpy()}
    dx = np.abs(res["f32c"].pop("pos") - res["f64"].pop("pos")).max(axis=0)
    e32, e64 = np.array(res["f32c"]["E"]), np.array(res["f64"]["E"])
    print(json.dumps({"c5_drift": {
        "workload": f"{workload_name(n)}; {nsteps} KDK steps, both paths from the same initial state",
        "f32c": res["f32c"], "f64": res["f64"],
        "ratio_f32c_over_f64": res["f32c"]["max_abs_dE_over_E"] / res["f64"]["max_abs_dE_over_E"],
        "max_abs_E_f32c_minus_E_f64_over_E": float(np.abs(e32 - e64).max() / abs(e64[0])),
        "final_position_difference": {"median": float(np.median(dx)), "max": float(dx.max())}}}))


def ablation_child(lib):
    """One library's accuracy at C5 (1024 sampled rows against the FP64 oracle)
    and at C3 (every row of one evaluation, and 10 KDK steps, against the FP64
    GPU path); prints one JSON line."""
    import torch
    import oracle
    import paper_2509_19294_gb300 as nb
    from paper_2509_19294_gb300 import ic
    nb.load(lib)
    out = {"library": os.path.basename(lib)}
    pos, _, mass = workload()
    n = mass.shape[0]
    tiles = (128, 2, 256, 4, 4)     # one shape and split for both libraries
    with nb.nbody_init(n, EPS, tiles=tiles) as ctx:
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), acc, pot)
        a, q = acc.cpu().numpy(), pot.cpu().numpy()
    rows = ic.sample_rows(n, 1024, 77)
    ra, rp = oracle.forces_rows(pos, mass, EPS, rows)
    rel = np.linalg.norm(a[:, rows] - ra, axis=0) / np.linalg.norm(ra, axis=0)
    prel = np.abs(q[rows] - rp) / np.abs(rp)
    out["c5_rows_vs_oracle"] = {"rows": len(rows), "median_rel_acc_err": float(np.median(rel)),
                                "max_rel_acc_err": float(rel.max()), "median_rel_pot_err": float(np.median(prel)),
                                "max_rel_pot_err": float(prel.max()), "tiles": list(tiles)}
    cpos, cvel, cmass = ic.plummer(131072, seed=3)
    evals, tracks = {}, {}
    for name, mode in (("f32c", nb.NBODY_F32C), ("f64", nb.NBODY_F64)):
        e, _ = _run_with_diag(nb, torch, cpos, cvel, cmass, 1e-3, 1e-4, 10, mode)
        tracks[name] = e[:, 0]
        with nb.nbody_init(131072, 1e-3, mode=mode) as ctx:
            acc = torch.empty((3, 131072), dtype=torch.float64, device="cuda")
            pot = torch.empty(131072, dtype=torch.float64, device="cuda")
            nb.nbody_forces(ctx, torch.from_numpy(cpos).cuda(), torch.from_numpy(cmass).cuda(), acc, pot)
            evals[name] = (acc.cpu().numpy(), pot.cpu().numpy())
    (a32, p32), (a64, p64) = evals["f32c"], evals["f64"]
    rel = np.linalg.norm(a32 - a64, axis=0) / np.linalg.norm(a64, axis=0)
    prel = np.abs(p32 - p64) / np.abs(p64)
    e32, e64 = tracks["f32c"], tracks["f64"]
    out["c3_all_rows_vs_fp64"] = {"median_rel_acc_err": float(np.median(rel)), "max_rel_acc_err": float(rel.max()),
                                  "median_rel_pot_err": float(np.median(prel)), "max_rel_pot_err": float(prel.max())}
    out["c3_10_steps"] = {"f32c_max_abs_dE_over_E": float(np.abs(e32[:, 2] - e32[0, 2]).max() / abs(e32[0, 2])),
                          "f64_max_abs_dE_over_E": float(np.abs(e64[:, 2] - e64[0, 2]).max() / abs(e64[0, 2])),
                          "max_abs_E_f32c_minus_E_f64_over_E": float(np.abs(e32[:, 2] - e64[:, 2]).max() / abs(e64[0, 2]))}
    print(json.dumps(out), flush=True)


def run_tile_sum_ablation():
    """Accuracy with and without the cross-tile Kahan compensation of the F32C
    kernels (the ablation library is built on request only); one JSON line."""
    from paper_2509_19294_gb300 import build as nbuild
    nbuild.build()
    libs = [nbuild.LIB, nbuild.build_ablation()]
    res = []
    for lib in libs:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--ablation-child", lib],
                           capture_output=True, text=True, check=True)
        res.append(json.loads(r.stdout.strip().splitlines()[-1]))
    print(json.dumps({"tile_sum_compensation_ablation": {"with_compensation": res[0],
                                                         "without_compensation": res[1]}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--fp64-n", type=int, default=0,
                    help="FP64 comparator on the first N particles only (0 = the whole timed state)")
    ap.add_argument("--no-drift", action="store_true", help="skip the C4 and C3 drift comparisons")
    ap.add_argument("--no-c3-drift", action="store_true", help="skip the 1000-step C3 drift comparison")
    ap.add_argument("--c3-steps", type=int, default=1000)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-paper-scale", action="store_true")
    ap.add_argument("--no-block-steps", action="store_true")
    ap.add_argument("--n-each", type=int, default=N_EACH,
                    help="particles per sphere (default 524288: the N=1M workload)")
    ap.add_argument("--tiles", default=None,
                    help="force the tile shape block,p,tj,split instead of autotuning")
    ap.add_argument("--block-drift", default=None, metavar="N,T",
                    help="only the block-step energy drift, F32C vs FP64 path (e.g. 16384,0.5; "
                         "the FP64 path takes minutes)")
    ap.add_argument("--c5-drift", type=int, default=0, metavar="STEPS",
                    help="only the C5 energy drift over STEPS steps, F32C vs the FP64 path "
                         "(10 steps: ~9 minutes of FP64 work)")
    ap.add_argument("--ablation-tile-sums", action="store_true",
                    help="only the accuracy with and without the cross-tile Kahan compensation")
    ap.add_argument("--ablation-child", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.ablation_child:
        ablation_child(args.ablation_child)
        return
    if args.ablation_tile_sums:
        run_tile_sum_ablation()
        return
    if args.c5_drift:
        run_c5_drift(args.c5_drift)
        return
    if args.block_drift:
        n, t = args.block_drift.split(",")
        run_block_drift(int(n), float(t))
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
