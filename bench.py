"""Benchmark: pruned trajectories/s at n = 12 vs full on the same B300, with
p50/p99 query latency.

Workload: qubit encoding (phase-kickback fetch between two Hadamard walls),
n = 12 (4096 cells), k = 4 data qubits per cell with i.i.d. random bits, the
data-loading input (one branch per address, zero bus), gamma log-uniform in
[1e-5, 1e-2] per batch of 1000 trajectories, 1e5 trajectories, complex FP64.
A step is one pruned launch over the whole 1e5-trajectory batch (every row
of the hot path: sampling, marking, explicit evolution with the joint
sampler, closed-form good branches, final measurement).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank simulates its own 1e5 trajectories (weak scaling,
replicas by trajectory range; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "pruned trajectories/s at n=12 vs full on same B300; p50/p99 query latency"
N, K, NTRAJ, BATCH = 12, 4, 100_000, 1000
G_LO, G_HI = 1e-5, 1e-2
SEED = 4001
WORKLOAD = ("qubit encoding n=12 (4096 cells), k=4 i.i.d. data bits, data-loading input, "
            "gamma log-uniform [1e-5,1e-2] per batch of 1000 trajectories, 1e5 trajectories, complex FP64")


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def trajectory_base(rank: int) -> int:
    """First trajectory index of a rank: ranks simulate disjoint ranges (weak
    scaling; trajectories are independent given (seed, index))."""
    return rank * 1_000_000_000


def world_throughput(t_local: float, steps: int, ntraj: int, dist=None) -> tuple:
    """Whole-job trajectories/s: every rank ran `steps` x `ntraj`; the job
    takes as long as the slowest rank (max over ranks, the only exchange)."""
    import torch
    world = 1
    t = t_local
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        tt = torch.tensor([t_local], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt[0])
    return world * steps * ntraj / t, t


# INT32 operations per unit of counted work: a fault-stream draw is half a
# Philox4x32-10 call (10 rounds of 2 wide multiplies, 4 xors, 2 key adds)
# plus the 13-step fixed-point gap search; a component-slice is the path-word
# gate arithmetic; a branch-epoch is the closed-form exposure (4 table
# lookups and adds), the hit test and a histogram count; a component-epoch
# is the pack/unpack, mask and histogram bookkeeping of an explicit pass
OPS_PER_UNIT = {"draws": 140, "comp_slices": 12, "branch_epochs": 12, "comp_epochs": 30}
# 32-bit integer add/logic lanes per SM per clock (the unified FP32/INT32
# cores; qram_measure_peaks measures 92 % of SMs x 128 x 2032 MHz)
INT32_LANES = 128
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "traj_kernel_qubit_n12k4_traffic.json")


def _kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2609_34935_b300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".h")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    with open(os.path.join(ROOT, "include", "qram_sim.h"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def _traffic_per_step():
    """DRAM bytes of one step launch: the committed ncu record of the small
    mix case (--profile-mix: 592 trajectories with the bench's mix of damping
    rates, one launch) scaled per trajectory to the 1e5 trajectories of a
    step; only if it was taken on the kernel sources of this tree."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("sources_sha256") != _kernel_sources_hash() or "dram_bytes_per_trajectory" not in rec:
        return None
    return rec["dram_bytes_per_trajectory"] * NTRAJ


def _problem():
    return W.data_loading(W.QUBIT, N, K, seed=SEED)


def _gammas():
    return W.gamma_batches(NTRAJ, BATCH, G_LO, G_HI, seed=SEED)


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        # the raw samples are kept in QRAM_CLOCKS_DIR (default: the system's temporary directory)
        import tempfile
        d = os.environ.get("QRAM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_bench_{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_baseline(p, gam, budget_s=15.0):
    """The oracle (plain CPU full evolution) on the host cores, on a bounded
    sample: trajectories spread over the gamma batches of the workload."""
    cores = os.cpu_count() or 1
    idx = np.arange(0, NTRAJ, BATCH // 2)            # 2 per gamma batch, 200 in total
    done, t0 = 0, time.perf_counter()
    for start in range(0, len(idx), cores):
        sel = idx[start:start + cores]
        _oracle_chunk(p, gam, sel, cores)
        done += len(sel)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} trajectories of the workload (every {BATCH // 2}th index, spanning the gamma "
                      f"batches), full evolution, one trajectory per host thread"}


def _oracle_chunk(p, gam, sel, cores):
    """Run the given trajectory indices on `cores` threads (each trajectory
    keeps its own index and damping rate)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import core
    with ThreadPoolExecutor(max_workers=cores) as ex:
        return list(ex.map(lambda t: core.run(p, SEED, int(t), gam[t:t + 1], nthreads=1), sel))


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    p = _problem()
    gam = _gammas()
    from oracle import core
    core.build()
    cores = os.cpu_count() or 1
    per_step = max(cores, 16)
    idx = np.arange(0, NTRAJ, NTRAJ // per_step)[:per_step]
    for _ in range(args.warmup):
        _oracle_chunk(p, gam, idx[:cores], cores)
    times = []
    for s in range(args.steps):
        sel = (idx + s) % NTRAJ
        t0 = time.perf_counter()
        _oracle_chunk(p, gam, sel, cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * per_step / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trajectories/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": "oracle full evolution (CPU)"},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} trajectories per step spread over the gamma batches"},
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", action="store_true", help="run the serving-stream benchmark instead")
    ap.add_argument("--requests", type=int, default=2000, help="--serving: number of requests")
    ap.add_argument("--traj-lo", type=float, default=1e3, help="--serving: trajectories per request, log-uniform from")
    ap.add_argument("--traj-hi", type=float, default=1e5, help="--serving: ... to")
    ap.add_argument("--scan", action="store_true",
                    help="fidelity vs n (qubit, k=3, 500-branch random input, 200 trajectories per point)")
    ap.add_argument("--profile-case", type=float, default=None, metavar="GAMMA",
                    help="one launch of 592 trajectories (296 CTAs of 512 threads) at this gamma, for ncu")
    ap.add_argument("--profile-mix", action="store_true",
                    help="one launch of 592 trajectories with the bench workload's rates (every 168th index; "
                         "296 CTAs of 512 threads), for ncu: the small case whose traffic scales to a step")
    ap.add_argument("--configs", action="store_true",
                    help="the other workload configurations (qutrit n=3, qubit n=6, qutrit n=10): throughput, "
                         "work and measured peaks")
    ap.add_argument("--only", type=int, default=None, help="with --configs: run only this configuration index")
    ap.add_argument("--variants", action="store_true",
                    help="pruned throughput of each launch variant (128/256/512 threads per CTA) over encoding, "
                         "n = 4..14, k = 1, 2, 4 and gamma 3e-4, 3e-3, each launch filling the device")
    ap.add_argument("--rate-scan", action="store_true",
                    help="pruned and full over n = 4..12 and gamma 0..1e-2 (qubit, k=3, the shape of Tab. V), "
                         "damping only")
    args = ap.parse_args()
    if args.rate_scan:
        return run_rate_scan(args)
    if args.variants:
        return run_variants(args)
    if args.profile_case is not None or args.profile_mix:
        return run_profile_case(args.profile_case)
    if args.configs:
        return run_configs(args)
    if args.scan:
        return run_scan(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)

    import torch
    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_2609_34935_b300 import QramSim

    p = _problem()
    gam_h = _gammas()
    stream = torch.cuda.Stream(device=dev)
    sim = QramSim(p, seed=SEED, device=local, stream=stream)
    sim.set_gamma_bound(G_HI)
    with torch.cuda.stream(stream):
        variant = sim.autotune("pruned", 3e-3, 2000)                     # threads per CTA for this problem
    gam = torch.tensor(gam_h, dtype=torch.float64, device=dev)
    out = torch.empty((NTRAJ, 48), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)      # > 126 MB L2
    base = trajectory_base(rank)                                          # disjoint trajectory ranges
    traj0 = torch.zeros(1, dtype=torch.int64, device=dev)
    graph = sim.graph("pruned", gam, out, traj0)          # per step: launch-order score and sort, one persistent launch

    def step(j):
        traj0.fill_(base + j * NTRAJ)
        graph()

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for j in range(args.warmup):
            step(j)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    sim.work_counters(reset=True)
    l0 = sim.launch_count
    ev = []
    barrier()
    for j in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(j & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(args.warmup + j)
            e1.record(stream)
        ev.append((e0, e1))
    barrier()
    launches = sim.launch_count - l0
    ms = [a.elapsed_time(b) for a, b in ev]
    work = sim.work_counters(reset=True)
    cl = clocks.stop()
    res = sim.results(out)
    value, t_dev = world_throughput(sum(ms) / 1e3, args.steps, NTRAJ, dist)

    def timed(fn, reps=1):
        with torch.cuda.stream(stream):
            fn()
            stream.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    # ---- full evolution on the whole workload, same trajectories ------------
    # One graph-captured full-mode launch per step over the same 1e5
    # trajectories as the pruned steps (the same trajectory indices, damping
    # rates and noise histories), timed like them; then the pruned step of
    # the last index range is replayed to compare the two modes trajectory by
    # trajectory.
    out_f = torch.empty((NTRAJ, 48), dtype=torch.uint8, device=dev)
    graph_f = sim.graph("full", gam, out_f, traj0)
    full_steps = max(2, min(args.steps, 3))
    with torch.cuda.stream(stream):
        traj0.fill_(base + args.warmup * NTRAJ)
        graph_f()
    barrier()
    evf = []
    for j in range(full_steps):
        with torch.cuda.stream(stream):
            flush.fill_(j & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            traj0.fill_(base + (args.warmup + j) * NTRAJ)
            a.record(stream)
            graph_f()
            b.record(stream)
        evf.append((a, b))
    barrier()
    t_full_step = sum(a.elapsed_time(b) for a, b in evf) / 1e3 / full_steps
    full_res = sim.results(out_f)
    with torch.cuda.stream(stream):
        graph()                                   # pruned, same traj0 as the last full step
    barrier()
    pr_res = sim.results(out)
    agree = float(np.max(np.abs(full_res["fidelity"] - pr_res["fidelity"])))
    same_int = bool(all(np.array_equal(full_res[f], pr_res[f]) for f in ("ncand", "bad", "ref", "jumps",
                                                                           "first_jump_slice", "q_ground")))
    graph_f.close()

    # ---- pruned vs full per gamma decade (the shape of the paper's Tab. V) ---
    per_decade = {}
    nd = 20_000
    gd = torch.empty(nd, dtype=torch.float64, device=dev)
    od = torch.empty((nd, 48), dtype=torch.uint8, device=dev)
    for dg in (1e-5, 1e-4, 1e-3, 1e-2):
        gd.fill_(dg)
        tp = timed(lambda: sim.run_pruned(base + 8_000_000, gd, od))
        rp = sim.results(od)
        tf = timed(lambda: sim.run_full(base + 8_000_000, gd, od))
        rf = sim.results(od)
        per_decade[f"{dg:g}"] = {"pruned_traj_per_s": nd / tp, "full_traj_per_s": nd / tf, "speedup": tf / tp,
                                 "evolved_fraction": float(np.mean(rp["explicit_comps"]) / np.mean(rf["explicit_comps"])),
                                 "max_abs_fidelity_diff": float(np.max(np.abs(rp["fidelity"] - rf["fidelity"]))),
                                 "trajectories": nd}

    # ---- the paper's mixed setting, depolarizing faults with eps = gamma ------
    # Every branch is explicit in both modes and every tree site takes faults
    # (the placement the paper leaves open), so stray excitations pile up in
    # every component; a trajectory whose strays exceed the per-component
    # capacity (32 off-path sites) reports QRAM_E_CAP.  The mean fidelity and
    # the rate are over the completed trajectories, with the failed count.
    mixed = {}
    nm = 2000
    pm = W.data_loading(W.QUBIT, 8, 3, seed=SEED + 8)
    simm = QramSim(pm, seed=SEED + 8, device=local, stream=stream)
    simm.set_gamma_bound(1e-3)
    simm.set_depolarizing(0.0, eps_equals_gamma=True)
    gm = torch.empty(nm, dtype=torch.float64, device=dev)
    om = torch.empty((nm, 48), dtype=torch.uint8, device=dev)
    for dg in (1e-5, 1e-4, 1e-3):
        gm.fill_(dg)
        tm_ = timed(lambda: simm.run_pruned(base + 6_000_000, gm, om))
        rm = QramSim.results(om)
        okm = rm["status"] == 0
        mixed[f"{dg:g}"] = {"completed_traj_per_s": int(okm.sum()) / tm_,
                            "mean_fidelity_completed": float(rm["fidelity"][okm].mean()) if okm.any() else None,
                            "completed": int(okm.sum()), "failed_capacity": int(np.sum(rm["status"] == 6)),
                            "failed_other": int(np.sum(~okm & (rm["status"] != 6)))}
    simm.close()

    # ---- mixed persistent launch: three workloads in one graph launch -------
    mixed_launch = _mixed_launch_row(dev, stream, variant)

    # ---- per-query latency: one gamma batch (1000 trajectories) alone -----
    lat = []
    gb = torch.empty(BATCH, dtype=torch.float64, device=dev)
    ob = torch.empty((BATCH, 48), dtype=torch.uint8, device=dev)
    for b in range(0, NTRAJ, BATCH * 4):
        gb.copy_(gam[b:b + BATCH])
        lat.append(1e3 * timed(lambda: sim.run_pruned(base + 9_000_000 + b, gb, ob)))
    lat_tp = np.array(lat)
    # the same queries on the latency variant: 1024 threads, one trajectory
    # per SM (a query ends with its slowest trajectory, which then has a
    # whole SM's threads for its explicit components)
    lsim = QramSim(p, seed=SEED, device=local, stream=stream)
    lsim.set_gamma_bound(G_HI)
    lsim.set_variant(1024)
    lat = []
    for b in range(0, NTRAJ, BATCH * 4):
        gb.copy_(gam[b:b + BATCH])
        lat.append(1e3 * timed(lambda: lsim.run_pruned(base + 9_000_000 + b, gb, ob)))
    lat = np.array(lat)
    lsim.close()

    # ---- end to end through the C ABI with host buffers --------------------
    g_pin = torch.tensor(gam_h, dtype=torch.float64).pin_memory()
    o_pin = torch.empty((NTRAJ, 48), dtype=torch.uint8).pin_memory()
    e2e_t = []
    for j in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            gam.copy_(g_pin, non_blocking=True)
            sim.run_pruned(base + 5_000_000 + j * NTRAJ, gam, out)
            o_pin.copy_(out, non_blocking=True)
        stream.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = world * NTRAJ / float(np.mean(e2e_t))

    # ---- roofline of the trajectory kernel ---------------------------------
    # algorithmic INT32 work counted by the kernel itself over the timed steps
    ops = sum(work[k] * OPS_PER_UNIT[k] for k in OPS_PER_UNIT) / args.steps
    sm_mhz = cl.get("sm_mhz") or 2032.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_int = nsm * INT32_LANES * sm_mhz * 1e6 / 1e12  # Tops/s
    launch_s = t_dev / args.steps
    achieved = ops / launch_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_int, "unit": "Tops/s (INT32)",
            "frac": achieved / peak_int, "traffic": _traffic_per_step(),
            "note": "algorithmic INT32 ops per step launch from the kernel's work counters x ops per unit "
                    f"{OPS_PER_UNIT} / launch time from CUDA events; peak derived: SMs x {INT32_LANES} INT32 "
                    "lanes/clock x median SM clock under load (measured_peaks: the measured add/logic rate); "
                    "traffic: DRAM read+write bytes per trajectory of the small mix case (ncu, one launch of 592 "
                    "trajectories on the step's 296 CTAs, same kernel sources) x the trajectories of a step, else null",
            "work_per_step": {k: v / args.steps for k, v in work.items()}, "variant_threads": variant}
    try:
        from paper_2609_34935_b300 import measure_peaks
        mp = measure_peaks(local)
        roof["measured_peaks"] = {"int32_tops": mp["int32_ops"] / 1e12, "fp64_tflops": mp["fp64_flops"] / 1e12,
                                  "frac_of_measured_int32": achieved / (mp["int32_ops"] / 1e12),
                                  "how": "qram_measure_peaks (independent add+xor / FP64 FMA chains on every SM)"}
    except Exception as e:               # pragma: no cover
        roof["measured_peaks"] = {"error": str(e)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = _cpu_baseline(p, gam_h)
        except Exception as e:           # pragma: no cover
            cpu = {"value": None, "error": str(e)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": "pruned", "trajectories_per_step": NTRAJ,
                       "l2": "256 MiB buffer written between timed steps",
                       "parallelism": f"replicas x{world} (trajectory ranges)"},
            "full": {"value": world * NTRAJ / t_full_step, "unit": "trajectories/s",
                     "ms_per_step": 1e3 * t_full_step, "steps": full_steps,
                     "speedup_pruned_over_full": t_full_step / (t_dev / args.steps),
                     "trajectories": f"the same {NTRAJ} trajectories per step as the pruned steps (same indices, "
                                     "damping rates and noise histories), one graph per step (launch-order score and sort, one persistent launch)",
                     "max_abs_fidelity_diff_pruned_vs_full": agree, "integer_outputs_equal": same_int},
            "per_gamma_decade": per_decade,
            "eps_eq_gamma_per_decade": {"note": "depolarizing faults of strength eps = gamma on top of the damping "
                                                "(the paper's benchmark setting; every tree site active, a reading "
                                                "the paper's Tab. IV does not pin), every branch explicit; qubit "
                                                "n=8, k=3, data-loading input, 2000 trajectories per decade; rate "
                                                "and mean fidelity over the completed trajectories", **mixed},
            "mixed_launch": mixed_launch,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "query": "one gamma batch of 1000 trajectories launched alone", "n": int(len(lat)),
                           "variant_threads": 1024,
                           "throughput_variant": {"threads": variant, "p50": float(np.percentile(lat_tp, 50)),
                                                  "p99": float(np.percentile(lat_tp, 99))}},
            "mean_fidelity": float(res["fidelity"].mean()), "status_ok": bool(np.all(res["status"] == 0)),
            "mean_bad_fraction": float(res["bad"].mean() / (1 << N)),
            "e2e": {"value": e2e_val, "unit": "trajectories/s", "h2d_bytes_per_step": int(g_pin.numel() * 8),
                    "d2h_bytes_per_step": int(o_pin.numel())},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": cl,
        }
        print(json.dumps(line), flush=True)
    graph.close()
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


def _mixed_launch_row(dev, stream, threads):
    """Qubit n=6 (3e4 trajectories, gamma cycling through 1e-4, 1e-3, 1e-2),
    qutrit n=10 (1e5 at 1e-3) and the bench workload (qubit n=12, k=4, 1e5)
    in one persistent graph-captured launch (qram_batch_create), against the
    three launched one after the other as their own graphs in the same
    variant; both timed with CUDA events, best of three."""
    import torch
    from paper_2609_34935_b300 import QramBatch, QramSim
    parts = [(W.data_loading(W.QUBIT, 6, 1, seed=2001), 2001, np.tile([1e-4, 1e-3, 1e-2], 10_000)),
             (W.data_loading(W.QUTRIT, 10, 1, seed=3001), 3001, np.full(NTRAJ, 1e-3)),
             (_problem(), SEED, _gammas())]
    sims, gams, outs, graphs, t0s = [], [], [], [], []
    for p, seed, g in parts:
        sim = QramSim(p, seed=seed, device=dev.index or 0, stream=stream)
        sim.set_gamma_bound(float(g.max()))
        sim.set_variant(threads)
        gams.append(torch.tensor(g, dtype=torch.float64, device=dev))
        outs.append(torch.empty((len(g), 48), dtype=torch.uint8, device=dev))
        t0s.append(torch.zeros(1, dtype=torch.int64, device=dev))
        sims.append(sim)
    for sim, g, o, t0 in zip(sims, gams, outs, t0s):
        graphs.append(sim.graph("pruned", g, o, t0))
    batch = QramBatch(sims, "pruned", [0, 0, 0], gams, outs, threads=threads)

    def best(fn):
        with torch.cuda.stream(stream):
            fn()
            stream.synchronize()
            b = float("inf")
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                b = min(b, e0.elapsed_time(e1) / 1e3)
        return b

    def separate():
        for gr in graphs:
            gr()
    t_sep = best(separate)
    sep = [sim.results(o).copy() for sim, o in zip(sims, outs)]
    t_mix = best(batch)
    same = all(np.array_equal(QramSim.results(o), r) for o, r in zip(outs, sep))
    ntot = sum(len(g) for _, _, g in parts)
    row = {"workloads": "qubit n=6 k=1 (3e4, gamma 1e-4/1e-3/1e-2), qutrit n=10 k=1 (1e5, gamma 1e-3), "
                        "qubit n=12 k=4 (1e5, the bench's gamma mix)",
           "threads": threads, "ctas": batch.grid, "trajectories": ntot,
           "mixed_traj_per_s": ntot / t_mix, "separate_graphs_traj_per_s": ntot / t_sep,
           "mixed_ms": 1e3 * t_mix, "separate_ms": 1e3 * t_sep, "results_equal_to_separate": bool(same)}
    batch.close()
    for gr in graphs:
        gr.close()
    for sim in sims:
        sim.close()
    return row


def run_scan(args):
    """Fidelity versus n for gamma in {1e-5, 1e-4, 1e-3} (the damping-only
    analog of the paper's Fig. 2), one JSON line with the table."""
    import torch
    from paper_2609_34935_b300.scan import fidelity_vs_n
    t0 = time.perf_counter()
    rows = fidelity_vs_n(W.QUBIT, range(3, 13), (1e-5, 1e-4, 1e-3), k=3, D=500, ntraj=200)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    # with every tree site active, stray excitations exceed the per-component
    # capacity beyond these sizes (reported as QRAM_E_CAP)
    rows_eps = fidelity_vs_n(W.QUBIT, range(3, 9), (1e-5, 1e-4), k=3, D=500, ntraj=200, eps_equals_gamma=True)
    rows_eps += fidelity_vs_n(W.QUBIT, range(3, 7), (1e-3,), k=3, D=500, ntraj=200, eps_equals_gamma=True)
    torch.cuda.synchronize()
    print(json.dumps({"scan": "mean fidelity vs n, qubit, k=3, 500-branch random input (one column per "
                              "address), 200 trajectories per point; damping only, and depolarizing faults "
                              "of the same strength (eps = gamma, every tree site active; n <= 8, n <= 6 at 1e-3)",
                      "seconds": t1 - t0, "rows": rows,
                      "seconds_eps_eq_gamma": time.perf_counter() - t1, "rows_eps_eq_gamma": rows_eps}), flush=True)
    return 0


# The workload configurations besides the bench's own (qubit n=12, k=4):
# (name, encoding, n, k, gammas, trajectories, seeds per gamma).  All use the
# data-loading input (every address, equal weights, zero bus) and i.i.d.
# random cell bits.
CONFIGS = [
    ("qutrit n=3 (8 cells), k=1, gamma 1e-3, 1000 trajectories", W.QUTRIT, 3, 1, [1e-3], 1000, [1001]),
    ("qubit n=6 (64 cells), k=1, gamma 1e-4 / 1e-3 / 1e-2, 1e4 trajectories each", W.QUBIT, 6, 1,
     [1e-4, 1e-3, 1e-2], 10_000, [2001, 2002, 2003]),
    ("qutrit n=10 (1024 cells), k=1, gamma 1e-3, 1e5 trajectories in one graph-captured launch", W.QUTRIT, 10, 1,
     [1e-3], 100_000, [3001]),
]


def run_configs(args):
    """Each configuration at each of its gammas: one graph-captured pruned
    launch over all its trajectories (best of three, CUDA events on the
    simulator's stream), full mode on up to 2e4 of the same trajectories,
    the kernel's work counters and the INT32 rate they give, against the
    derived INT32 peak and the measured integer and FP64 peaks."""
    import torch
    from paper_2609_34935_b300 import QramSim, measure_peaks
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    peaks = measure_peaks(0)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    rows = []
    for ci, (name, enc, n, k, gammas, ntraj, seeds) in enumerate(CONFIGS):
        if args.only is not None and ci != args.only:
            continue
        for g, seed in zip(gammas, seeds):
            stream = torch.cuda.Stream(device=dev)
            sim = QramSim(W.data_loading(enc, n, k, seed=seed), seed=seed, device=0, stream=stream)
            sim.set_gamma_bound(g)
            with torch.cuda.stream(stream):
                variant = sim.autotune("pruned", g, min(ntraj, 2000))
            gam = torch.full((ntraj,), g, dtype=torch.float64, device=dev)
            out = torch.empty((ntraj, 48), dtype=torch.uint8, device=dev)
            traj0 = torch.zeros(1, dtype=torch.int64, device=dev)
            graph = sim.graph("pruned", gam, out, traj0)

            def timed(fn, reps):
                with torch.cuda.stream(stream):
                    fn()
                    stream.synchronize()
                    best = float("inf")
                    for _ in range(reps):
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        fn()
                        b.record(stream)
                        b.synchronize()
                        best = min(best, a.elapsed_time(b) / 1e3)
                return best

            sim.work_counters(reset=True)
            t_p = timed(graph, 3)
            work = {kk: v / 4 for kk, v in sim.work_counters(reset=True).items()}   # warm-up + 3 timed launches
            rp = sim.results(out)
            nf = min(ntraj, 20_000)
            gf, of = gam[:nf], torch.empty((nf, 48), dtype=torch.uint8, device=dev)
            t_f = timed(lambda: sim.run_full(0, gf, of), 1)
            rf = sim.results(of)
            graph.close()
            sim.close()
            ops = sum(work[kk] * OPS_PER_UNIT[kk] for kk in OPS_PER_UNIT)
            achieved = ops / t_p
            peak_derived = nsm * INT32_LANES * 2032e6
            rows.append({
                "config": name, "gamma": g, "trajectories": ntraj, "variant_threads": variant,
                "pruned_traj_per_s": ntraj / t_p, "full_traj_per_s": nf / t_f, "speedup": (ntraj / t_p) / (nf / t_f),
                "mean_fidelity": float(rp["fidelity"].mean()),
                "bad_fraction_mean": float(np.mean(rp["bad"]) / (1 << n)),
                "max_abs_fidelity_diff_full": float(np.max(np.abs(rp["fidelity"][:nf] - rf["fidelity"]))),
                "status_ok": bool((rp["status"] == 0).all() and (rf["status"] == 0).all()),
                "work_per_launch": work,
                "int32": {"achieved_tops": achieved / 1e12, "frac_of_derived": achieved / peak_derived,
                          "frac_of_measured": achieved / peaks["int32_ops"]},
            })
    print(json.dumps({"configs": rows, "measured_peaks": {
        "fp64_tflops": peaks["fp64_flops"] / 1e12, "int32_tops": peaks["int32_ops"] / 1e12,
        "how": "qram_measure_peaks: 8 independent FMA (FP64) or add+xor (INT32) chains per thread on every SM, "
               "best of 5 launches"},
        "int32_peak_derived_tops": nsm * INT32_LANES * 2032e6 / 1e12}))
    return 0


PROFILE_TRAJ = 592          # two per CTA of a launch with the bench's 296 CTAs (2 per SM)
PROFILE_STRIDE = 168        # the mix case: trajectory indices 0, 168, ... (spans the 100 gamma batches)


def run_profile_case(gamma):
    """Small case of the bench kernel for a profiler capture: the bench
    problem in the bench's launch shape (512-thread CTAs, two per SM), one
    launch of two trajectories per CTA.  With a gamma, every trajectory has
    that rate.  Without (the mix case), trajectories 0..591 take the rates
    of every PROFILE_STRIDE-th index of the bench workload: about six per
    gamma batch, the bench's own mix of rates, with as many CTAs sharing L2
    as in a step, so per-trajectory counters (DRAM bytes, work) scale to a
    step."""
    import torch
    from paper_2609_34935_b300 import QramSim
    sim = QramSim(_problem(), seed=SEED, device=0)
    sim.set_variant(512)
    sim.set_launch_ctas(PROFILE_TRAJ // 2)
    sim.set_gamma_bound(G_HI)
    if gamma is None:
        idx = np.arange(PROFILE_TRAJ) * PROFILE_STRIDE
        gh = _gammas()[idx]
    else:
        gh = np.full(PROFILE_TRAJ, gamma)
    g = torch.tensor(gh, dtype=torch.float64, device="cuda:0")
    sim.work_counters(reset=True)
    raw = sim.run_pruned(0, g)
    torch.cuda.synchronize()
    r = sim.results(raw)
    w = sim.work_counters(reset=True)
    print(json.dumps({"profile_case": gamma if gamma is not None else "mix", "trajectories": PROFILE_TRAJ,
                      "status_max": int(r["status"].max()), "mean_fidelity": float(r["fidelity"].mean()),
                      "jumps": float(r["jumps"].mean()), "work": w}))
    sim.close()
    return 0


def run_variants(args):
    """Launch-variant table: for each (encoding, n, k, gamma) the pruned
    trajectories/s of the 128-, 256- and 512-thread variants, data-loading
    input, one launch over the whole device (best of three after one
    untimed), CUDA events on the simulator's stream."""
    import torch
    from paper_2609_34935_b300 import QramSim
    rank, world, local = _env_rank()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    rows = []
    for enc in (W.QUTRIT, W.QUBIT):
        for n in (4, 6, 8, 10, 12, 14):
            for k in (1, 2, 4):
                p = W.data_loading(enc, n, k, seed=7000 + n * 10 + k)
                sim = QramSim(p, seed=7000 + n, device=local)
                for gamma in (3e-4, 3e-3):
                    nt = 6000 if n <= 8 else 3000
                    g = torch.full((nt,), gamma, dtype=torch.float64, device=f"cuda:{local}")
                    row = {"encoding": "qubit" if enc == W.QUBIT else "qutrit", "n": n, "k": k, "gamma": gamma,
                           "trajectories": nt}
                    for th in (128, 256, 512):
                        sim.set_variant(th)
                        res = sim.run("pruned", 0, g)
                        sim.sync()
                        best = float("inf")
                        for _ in range(3):
                            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            sim.sync()
                            e0.record(sim.stream)
                            sim.run("pruned", 0, g, out=res)
                            e1.record(sim.stream)
                            e1.synchronize()
                            best = min(best, e0.elapsed_time(e1))
                        row[f"traj_per_s_{th}"] = nt / (best * 1e-3)
                        row["status_ok"] = bool(np.all(QramSim.results(res)["status"] == 0)) and row.get("status_ok", True)
                    row["best_threads"] = max((128, 256, 512), key=lambda t: row[f"traj_per_s_{t}"])
                    rows.append(row)
                sim.close()
    print(json.dumps({"metric": "pruned trajectories/s per launch variant", "unit": "trajectories/s",
                      "data": "synthetic", "rows": rows}), flush=True)


def run_rate_scan(args):
    """Pruned against full over address width and damping rate, in the shape
    of the paper's performance table (Tab. V: qubit encoding, k = 3,
    data-loading input, n = 4..12), damping only.  Per point: 4000
    trajectories, both modes on the same indices and rates, each mode on its
    fastest launch variant (one untimed launch, then one timed with CUDA
    events); the evolved fraction is the explicit components of the pruned
    mode over those of the full mode."""
    import torch
    from paper_2609_34935_b300 import QramSim
    rank, world, local = _env_rank()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    nt = 4000
    rows = []
    for n in (4, 6, 8, 10, 12):
        p = W.data_loading(W.QUBIT, n, 3, seed=6000 + n)
        sim = QramSim(p, seed=6000 + n, device=local)
        sim.set_gamma_bound(1e-2)
        g = torch.empty(nt, dtype=torch.float64, device=f"cuda:{local}")
        out = torch.empty((nt, 48), dtype=torch.uint8, device=f"cuda:{local}")
        for gamma in (0.0, 1e-5, 1e-4, 1e-3, 1e-2):
            g.fill_(gamma)
            row = {"n": n, "k": 3, "gamma": gamma, "trajectories": nt}
            res = {}
            for mode in ("pruned", "full"):
                best, bth = float("inf"), 0
                for th in (128, 256, 512):
                    sim.set_variant(th)
                    sim.run(mode, 0, g, out=out)
                    sim.sync()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(sim.stream)
                    sim.run(mode, 0, g, out=out)
                    e1.record(sim.stream)
                    e1.synchronize()
                    if e0.elapsed_time(e1) < best:
                        best, bth = e0.elapsed_time(e1), th
                res[mode] = QramSim.results(out)
                row[f"{mode}_traj_per_s"] = nt / (best * 1e-3)
                row[f"{mode}_threads"] = bth
            rp, rf = res["pruned"], res["full"]
            row["speedup"] = row["pruned_traj_per_s"] / row["full_traj_per_s"]
            row["evolved_fraction"] = float(np.mean(rp["explicit_comps"]) / np.mean(rf["explicit_comps"]))
            row["max_abs_fidelity_diff"] = float(np.max(np.abs(rp["fidelity"] - rf["fidelity"])))
            row["status_ok"] = bool(np.all(rp["status"] == 0) and np.all(rf["status"] == 0))
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
        sim.close()
    print(json.dumps({"metric": "pruned and full trajectories/s over n and damping rate", "unit": "trajectories/s",
                      "data": "synthetic", "config": {"workload": "qubit encoding, k=3, data-loading input, "
                                                                  "damping only, 4000 trajectories per point"},
                      "rows": rows}), flush=True)


def run_serving(args):
    """Serving stream: Poisson arrivals of requests, each drawing encoding
    (qutrit/qubit 50/50), n uniform in 4..14, data qubits 1..min(n, 4), gamma
    log-uniform in [1e-5, 1e-2], trajectories log-uniform in [lo, hi],
    seeded data; admitted by device-memory budget.  The arrival rate is set
    to a fraction (0.7 and 0.95) of the capacity measured on the same request
    mix submitted at once.  Reports p50/p99 latency and trajectories/s."""
    import torch
    from paper_2609_34935_b300 import QramServer
    rank, world, local = _env_rank()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    rng = np.random.default_rng(5001)
    lo, hi = args.traj_lo, args.traj_hi
    reqs = []
    for i in range(args.requests):
        enc = int(rng.integers(0, 2))
        n = int(rng.integers(4, 15))
        k = int(rng.integers(1, min(n, 4) + 1))
        g = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-2))))
        nt = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        reqs.append((W.data_loading(enc, n, k, seed=5001 * 1_000_000 + i), 5001 * 1_000_000 + i, 0,
                     np.full(nt, g), 0))
    free = torch.cuda.mem_get_info(local)[0]
    budget = int(free * 0.6)

    def run(rate):
        srv = QramServer(budget, device=local, max_active=8)
        t0 = time.perf_counter()
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs))) if rate else np.zeros(len(reqs))
        ids = []
        for (p, seed, traj0, g, mode), ta in zip(reqs, arrivals):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0005)
            ids.append(srv.submit(p, seed, traj0, g, mode))
        assert srv.drain(3600.0)
        wall = time.perf_counter() - t0
        comps = srv.poll(len(ids) + 16)
        srv.close()
        lat = np.array([c["t_finish"] - c["t_submit"] for c in comps])
        ok = all(c["status"] == 0 for c in comps)
        ntot = sum(c["ntraj"] for c in comps)
        return wall, lat, ok, ntot

    clocks = Clocks(local)
    clocks.start()
    wall0, _, ok0, ntot = run(0.0)                     # capacity: everything submitted at once
    cap_rps = len(reqs) / wall0
    lines = []
    for frac in (0.7, 0.95):
        wall, lat, ok, ntot = run(frac * cap_rps)
        lines.append({"load": frac, "rate_req_per_s": frac * cap_rps, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                      "p99_ms": 1e3 * float(np.percentile(lat, 99)), "trajectories_per_s": ntot / wall,
                      "status_ok": bool(ok)})
    cl = clocks.stop()
    print(json.dumps({"metric": "serving stream: p50/p99 query latency and trajectories/s", "unit": "ms",
                      "requests": len(reqs), "capacity_req_per_s": cap_rps, "capacity_traj_per_s": ntot / wall0,
                      "runs": lines, "data": "synthetic", "clocks": cl, "capacity_status_ok": bool(ok0),
                      "config": {"workload": f"Poisson arrivals of {len(reqs)} requests; encoding 50/50, n in 4..14, "
                                             f"k in 1..min(n,4), gamma log-uniform [1e-5,1e-2], trajectories "
                                             f"log-uniform [{lo:g},{hi:g}], data-loading input, pruned mode",
                                 "budget_bytes": budget, "max_active": 8}}), flush=True)


if __name__ == "__main__":
    main()
