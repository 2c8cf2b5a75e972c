"""Walker-steps/s of the stochastic SC-NEVPT2(s) local-estimator walk on GB300.

One "step" of this benchmark = one walk launch that advances every walker by `--inner`
continuous-time steps (each: local energy, reach-back overlaps, H_D numerator, rates,
accumulation, move) followed by the finalize kernels (E^(2) and jackknife errors).  Inputs
are the seeded synthetic 56-orbital CAS(10e,10o) system (6 core, 10 active, 40 virtual,
63,504-determinant reference) with 4,096 walkers, FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank walks its own independent walkers (different seeds),
there is no data-path collective (weak scaling); timing is barrier-bracketed, max over ranks.
The reference arm times the CPU oracle (the plain C implementation) on this host.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cas10_56o"
# DRAM bytes (read + write) per walker-step of k_walk on the 56-orbital workload, from one ncu
# capture of a steady-state 4,096-walker launch (46.95 MB); null for other workloads
TRAFFIC_PER_WALKER_STEP = {"cas10_56o": 46.953472e6 / 4096}
METRIC = "walker-steps/s"
# FP64 FMA pipe of GB300: 2 FMA per clock per SM, 152 SMs, 2.07 GHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# random 8-byte loads from an L2-resident table, measured on this machine's GB300 (loads/s)
L2_GATHER_PEAK = 3.14e11


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--walkers", type=int, default=4096)
    ap.add_argument("--system", default=WORKLOAD, help="named synthetic workload of the plain path")
    ap.add_argument("--inner", type=int, default=1, help="walker steps per walk launch")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="plain", choices=["plain", "batch", "serve"])
    ap.add_argument("--n-systems", type=int, default=64)
    ap.add_argument("--n-requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=20.0, help="request arrivals per second (served mode)")
    ap.add_argument("--target-sigma", type=float, default=1e-3)
    ap.add_argument("--req-walkers", type=int, default=512)
    ap.add_argument("--req-max-steps", type=int, default=400)
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=100.0)
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) > 8 for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def rank_seed(rank: int) -> int:
    """Each rank walks its own independent walkers: a different Philox key per rank."""
    return 1000 + rank


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The job's time is the slowest rank's (all ranks run the same number of walker-steps)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job walker-steps/s: all ranks' units over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(system, seconds: float, threads: int, orc=None):
    """Walker-steps/s of the plain C oracle's walk on a bounded sample of the same workload."""
    import oracle as O
    if orc is None:
        orc = O.Oracle.from_system(system)
    nw = max(threads, 1)
    t0 = time.perf_counter()
    acc = orc.sample(nw, 1, 0, seed=3, n_groups=1, threads=threads)
    t1 = time.perf_counter()
    steps = 1
    if (t1 - t0) < seconds / 3:
        steps = max(1, int(seconds / max(t1 - t0, 1e-3)) - 1)
        t0 = time.perf_counter()
        acc = orc.sample(nw, steps, 0, seed=3, n_groups=1, threads=threads)
        t1 = time.perf_counter()
    ws = nw * steps
    return ws / (t1 - t0), dict(walkers=nw, steps=steps, seconds=t1 - t0, type_steps=acc["type_steps"].tolist())


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    import synthetic as S
    system = S.workload(args.system)
    threads = os.cpu_count() or 1
    orc = O.Oracle.from_system(system)
    per_step = max(args.cpu_seconds / max(args.steps, 1), 1.0)
    rates = []
    meta = None
    for k in range(args.warmup + args.steps):
        r, meta = cpu_oracle_rate(system, per_step, threads, orc)
        if k >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * meta["walkers"] * meta["steps"] / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.system, "walkers_per_step": meta["walkers"], "steps_per_walker": meta["steps"]},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                         "sample": f"{meta['walkers']} walkers x {meta['steps']} steps per timed step"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import paper_1909_06935_gb300 as P
    import synthetic as S

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    system = S.workload(args.system)
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(local)
    ctx.set_stream(stream.cuda_stream)
    ctx.load_hamiltonian(system.n_core, system.n_act, system.n_virt, system.n_alpha, system.n_beta, system.h1,
                         system.eri, system.e_nuc)
    ctx.load_reference(system.dets, system.coeffs)
    ctx.set_coeffs(system.c)
    nw, inner = args.walkers, args.inner
    seed = rank_seed(rank)
    p = ctx.params(nw, args.warmup * inner, burn_in=0, seed=seed, n_groups=16)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize(dev)

    # warm-up
    ctx.walkers_init(p)
    res_w = None
    for _ in range(args.warmup):
        ctx.walkers_advance(inner)
        res_w = ctx.finalize()
        flush.zero_()
    snap0 = ctx.walkers(nw)[0]
    # timed region
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = None
    barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.walkers_advance(inner)
            res = ctx.finalize()
            flush.zero_()
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    # walk-kernel time of the timed launches (CUDA events recorded by the library on its stream)
    walk_s = res["seconds"] - (res_w["seconds"] if res_w else 0.0)
    walk_launches = res["walk_launches"] - (res_w["walk_launches"] if res_w else 0)
    snap1 = ctx.walkers(nw)[0]
    units = nw * inner * args.steps
    value = job_rate(units, world, ms)

    # algorithmic work per walker-step, counted exactly by the debug kernel on walker snapshots taken
    # before and after the timed region: every reach-back term H_mk phi0(k) is one FP64 FMA (2 flops),
    # every neighbour adds <n|H|m>, the ratio, the rate and three sums (8 flops)
    locs = [ctx.debug_local(snap)[0] for snap in (snap0, snap1)]
    terms = float(np.mean([np.mean(l["n_terms"]) for l in locs]))
    nbrs = float(np.mean([np.mean(l["n_neighbours"]) for l in locs]))
    gathers = float(np.mean([np.mean(l["n_gathers"] + l["n_probes"]) for l in locs]))
    flops_per_step = 2.0 * terms + 8.0 * nbrs
    launch_s = walk_s / max(walk_launches, 1)
    units_per_launch = nw * inner
    fp64_peak = FP64_PEAK_TFLOPS
    achieved = flops_per_step * units_per_launch / launch_s / 1e12
    peaks, peak_kind = load_peaks()
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak,
            "traffic": (TRAFFIC_PER_WALKER_STEP[args.system] * units_per_launch
                        if args.system in TRAFFIC_PER_WALKER_STEP else None),
            "kernel": "k_walk",
            "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (probe on this pool: 1.254 TFLOP/s)",
            "flops_per_walker_step": flops_per_step, "terms_per_walker_step": terms,
            "launch_seconds": launch_s, "launches_timed": int(walk_launches),
            "gathers_per_walker_step": gathers,
            "l2_gather_rate_per_s": gathers * units_per_launch / launch_s,
            "l2_gather_peak_per_s": L2_GATHER_PEAK, "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)),
            "hbm_peak_source": peak_kind}
    cand_per_step = float(np.mean([np.mean(l["n_candidates"]) for l in locs]))
    nb_per_step = nbrs

    # end to end through the public API with host buffers (inputs copied in every step)
    e2e = None
    if not args.no_e2e and rank == 0:
        h2d = system.h1.nbytes + system.eri.nbytes + system.dets.nbytes + system.coeffs.nbytes + system.c.nbytes
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
               dict(h1=system.h1, eri=system.eri, dets=system.dets.view(np.int64), co=system.coeffs,
                    c=system.c).items()}
        ctx2 = P.Context(local)
        ctx2.set_stream(stream.cuda_stream)
        k_e2e = max(inner, 4)   # walker steps per call: the cheap first step from the start determinant is one of k
        pe = ctx2.params(nw, k_e2e, burn_in=0, seed=seed, n_groups=16)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx2.load_hamiltonian(system.n_core, system.n_act, system.n_virt, system.n_alpha, system.n_beta,
                                  pin["h1"], pin["eri"], system.e_nuc)
            ctx2.load_reference(pin["dets"], pin["co"])
            ctx2.set_coeffs(pin["c"])
            ctx2.sample(pe)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        import ctypes
        d2h = ctypes.sizeof(P.Result)
        e2e = {"value": nw * k_e2e * args.steps / (t1 - t0), "unit": METRIC, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "walker_steps_per_call": nw * k_e2e,
               "call": "load_hamiltonian + load_reference + set_coeffs from pinned host memory, sample "
                       f"({k_e2e} steps from the start determinant), result read back"}
        ctx2.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, meta = cpu_oracle_rate(system, args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle",
               "sample": f"{meta['walkers']} walkers x {meta['steps']} steps of the same workload "
                         f"({meta['seconds']:.1f} s; class mix {meta['type_steps']})"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.system,
                       "orbitals": f"{system.n_core} core, {system.n_act} active, {system.n_virt} virtual",
                       "electrons": system.n_alpha + system.n_beta,
                       "reference_dets": int(len(system.coeffs)), "walkers_per_gpu": nw,
                       "walker_steps_per_launch": inner, "groups": 16, "method": "SC-NEVPT2(s) + E_L",
                       "l2": "256 MB buffer written between timed steps",
                       "neighbours_per_walker_step": nb_per_step, "candidates_per_walker_step": cand_per_step,
                       "class_mix": {P.TYPE_NAMES[t]: int(res["type_steps"][t]) for t in range(P.NTYPES)},
                       "e2": res["e2"], "e2_sigma": res["e2_sigma"]},
            "clocks": clk.summary(),
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": 3 * args.steps,        # per step: walk, finalize-labels, finalize-reduce
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batched(args):
    """Plain (one system per launch) against batched (all systems in one launch) on the batched
    workload: 64 seeded systems, 30-120 orbitals, CAS(6..10) references, walkers proportional to
    reference size (32,768 in total)."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import synthetic as S
    specs, walkers = S.batch_specs(args.n_systems)
    t0 = time.perf_counter()
    systems = S.make_systems(specs, processes=min(16, os.cpu_count() or 1))
    t_gen = time.perf_counter() - t0
    import torch
    import paper_1909_06935_gb300 as P
    dev = torch.device("cuda", 0)
    ctxs = [P.Context.from_system(s) for s in systems]
    params = [c.params(nw, 0, burn_in=0, seed=500 + k, n_groups=8) for k, (c, nw) in enumerate(zip(ctxs, walkers))]
    total = sum(walkers)

    R = max(1, args.inner)      # walker steps per reporting interval (one finalize per system)

    def plain_step():
        for c in ctxs:
            c.walkers_advance(R)
            c.finalize()

    def batched_step():
        P.batch_advance(ctxs, R)
        for c in ctxs:
            c.finalize()

    out, tune = {}, None
    for name, fn in (("plain", plain_step), ("batched", batched_step), ("batched_tuned", batched_step)):
        for c, p in zip(ctxs, params):
            c.walkers_init(p)
            c.set_launch()
        if name == "batched_tuned":     # autotune walkers/block and steps/launch, then graph replay
            tune = P.tune_batch(ctxs, trial_steps=min(R, 16))
            for c in ctxs:
                c.set_launch(tune["warps_per_block"], min(tune["steps_per_launch"], R), True)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        torch.cuda.synchronize(dev)
        out[name] = total * R * args.steps / (time.perf_counter() - t0)
    for c in ctxs:
        c.set_launch()
    line = {"metric": METRIC, "mode": "batched", "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "plain": out["plain"], "batched": out["batched"],
            "batched_tuned": out["batched_tuned"], "speedup": out["batched"] / out["plain"],
            "speedup_tuned": out["batched_tuned"] / out["plain"], "tuned_launch": tune,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batch{args.n_systems}", "systems": args.n_systems, "walkers": total,
                       "steps_per_report": R,
                       "orbitals": [s.n_orb for s in systems], "reference_dets": [len(s.coeffs) for s in systems],
                       "generation_seconds": t_gen}}
    print(json.dumps(line), flush=True)


def run_served(args):
    """Poisson stream of sampling requests through the request server (continuous batching):
    p50 / p99 time to the target error of E^(2), and throughput."""
    import synthetic as S
    import paper_1909_06935_gb300 as P
    rng = np.random.Generator(np.random.PCG64(77))
    base = dict(n_core=2, n_act=6, n_virt=16, n_alpha=5, n_beta=5, rank=72, seed=3301, chol_sigma=0.06)
    pool = [S.workload("tiny_12o_cas4")]
    pool += [S.make_system(2 + k % 3, 4 + 2 * (k % 2), 8 + 4 * k, 2 + k % 3 + (2 + k % 2), 2 + k % 3 + (2 + k % 2),
                           rank=40 + 8 * k, seed=3400 + k, chol_sigma=0.06) for k in range(6)]
    scan = S.scan_systems(base, n_points=10)
    reqs = [pool[int(rng.integers(len(pool)))] for _ in range(args.n_requests - len(scan))] + scan
    order = rng.permutation(len(reqs))
    srv = P.Server(max_active=args.max_active, hbm_budget_bytes=int(args.budget_gb * (1 << 30)), steps_per_round=2)
    srv.start()
    t0 = time.perf_counter()
    tickets = []
    for k in order:
        tickets.append(srv.submit(reqs[k], args.req_walkers, args.req_max_steps, target_sigma=args.target_sigma,
                                  burn_in=10, seed=900 + int(k), n_groups=16))
        time.sleep(rng.exponential(1.0 / args.rate))
    while not all(srv.poll(t)["state"] in ("done", "failed", "cancelled") for t in tickets):
        time.sleep(0.02)
    wall = time.perf_counter() - t0
    srv.stop()
    st = [srv.poll(t) for t in tickets]
    tt = np.array([x["total_seconds"] for x in st])
    reached = np.array([x["result"]["e2_sigma"] <= args.target_sigma for x in st])
    steps = sum(x["result"]["walker_steps"] for x in st)
    line = {"metric": "time-to-target", "mode": "served", "unit": "s", "p50": float(np.percentile(tt, 50)),
            "p99": float(np.percentile(tt, 99)), "requests": len(st), "reached_target": int(reached.sum()),
            "throughput_req_per_s": len(st) / wall, "walker_steps_per_s": srv.info()["walker_steps"] / wall,
            "accumulated_walker_steps": int(steps), "target_sigma": args.target_sigma, "arrival_rate": args.rate,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "served", "request_walkers": args.req_walkers, "max_steps": args.req_max_steps,
                       "max_active": args.max_active, "scan_points": len(scan)}}
    print(json.dumps(line), flush=True)
    srv.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batched(args)
    elif args.workload == "serve":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
