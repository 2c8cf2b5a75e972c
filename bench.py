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
# DRAM bytes (read + write) per walker-step of the walk kernel, from an ncu capture of one
# steady-state launch of the current kernel: dram__bytes_read.sum + dram__bytes_write.sum =
# 183.68 MB + 6630.77 MB for 4,096 walkers on the 56-orbital workload
TRAFFIC_PER_WALKER_STEP = {"cas10_56o": (183.676416e6 + 6630.774e6) / 4096}
METRIC = "walker-steps/s"
# FP64 FMA pipe of GB300: 2 FMA per clock per SM, 152 SMs, 2.07 GHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


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
    ap.add_argument("--ref-walkers", type=int, default=8, help="walkers moved per timed step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="plain", choices=["plain", "batch", "serve"])
    ap.add_argument("--n-systems", type=int, default=64)
    ap.add_argument("--n-requests", type=int, default=16)
    ap.add_argument("--rate", type=float, default=20.0, help="request arrivals per second (served mode)")
    ap.add_argument("--target-sigma", type=float, default=1e-4)
    ap.add_argument("--req-walkers", type=int, default=256)
    ap.add_argument("--req-max-steps", type=int, default=20000)
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=100.0)
    ap.add_argument("--no-batched", action="store_true", help="leave the batched sub-object out of the line")
    ap.add_argument("--no-served", action="store_true", help="leave the served sub-object out of the line")
    ap.add_argument("--batch-walkers", type=int, default=32768, help="walkers of the batched sub-object")
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


def groups_per_rank(world: int) -> int:
    """Walker groups of each rank: 16, fewer when all ranks' groups together would exceed the 64 a
    context can finalize."""
    return max(1, min(16, 64 // max(world, 1)))


def merge_rank_accumulators(accs):
    """Union of the ranks' walker groups (rank r's group g becomes group r G + g): the per-group
    sums are concatenated, the type counts and walker steps add up."""
    out = {k: np.concatenate([np.asarray(a[k]) for a in accs], 0)
           for k in ("N", "U", "W", "E", "A", "B") if all(a.get(k) is not None for a in accs)}
    out["type_steps"] = np.sum([np.asarray(a["type_steps"]) for a in accs], 0).astype(np.int64)
    out["total_steps"] = int(sum(int(a.get("total_steps", 0)) for a in accs))
    return out


def combine_ranks(ctx, groups: int, world: int, rank: int, total_steps: int):
    """Every rank's accumulators to rank 0, which finalizes their union (the cross-rank reduction
    of a multi-process run; one exchange after the timed region)."""
    acc = ctx.accumulators(groups)
    acc["A"], acc["B"] = ctx.gradient_sums(groups)
    acc["total_steps"] = total_steps
    if world <= 1:
        return None
    import torch.distributed as dist
    objs = [None] * world
    dist.all_gather_object(objs, acc)
    if rank != 0:
        return None
    merged = merge_rank_accumulators(objs)
    ctx.load_accumulators(merged, merged["total_steps"])
    res = ctx.finalize()
    return {"groups": groups * world, "walker_steps": merged["total_steps"], "e2": res["e2"],
            "e2_sigma": res["e2_sigma"], "e_var": res["e_var"], "e_var_sigma": res["e_var_sigma"]}


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job walker-steps/s: all ranks' units over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- CPU oracle

def type_mix(orc, dets):
    """Class mix (walkers per type 3h + p) of a set of determinants, by the oracle's labels."""
    mix = [0] * 9
    for d in dets:
        _, h, p = orc.label(d)
        mix[3 * h + p] += 1
    return mix


def cpu_oracle_steps(orc, dets, seconds: float, threads: int, seed: int = 3, step0: int = 0):
    """Walker-steps/s of the plain C oracle on walker determinants `dets`: each one is one walker
    step (local quantities of Eq. 5 and Eq. 16 with every reach-back overlap, then the move), the
    oracle's own code as it stands, on `threads` cores.  Stops after `seconds` (at least one step).
    Returns (rate, steps done, the moved determinants)."""
    import oracle as O
    O.set_threads(threads)
    moved = []
    t0 = time.perf_counter()
    for w, d in enumerate(dets):
        nxt, _, _ = orc.move(d, seed=seed, step=step0, walker=w)
        moved.append(nxt)
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    O.set_threads(0)
    return len(moved) / dt, len(moved), np.array(moved)


def oracle_steady_dets(orc, n_walkers: int, warm_steps: int, seed: int):
    """Walker determinants after `warm_steps` steps of the oracle's own walk from the start (the
    steady-state class mix, for a CPU arm that has no GPU walkers to copy)."""
    return np.array([orc.walk_one(w, warm_steps, seed)[-1] for w in range(n_walkers)])


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the benchmark's workload.  Each timed step
    moves a bounded sample of walkers once (from the steady state of a short untimed warm-up walk),
    on all of this host's cores."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    import synthetic as S
    system = S.workload(args.system)
    threads = os.cpu_count() or 1
    orc = O.Oracle.from_system(system)
    nw = args.ref_walkers
    dets = oracle_steady_dets(orc, nw, 3, seed=11)
    mix = type_mix(orc, dets)
    rates = []
    per_step = max(args.cpu_seconds / max(args.steps, 1), 1.0)
    for k in range(args.warmup + args.steps):
        r, done, moved = cpu_oracle_steps(orc, dets, per_step, threads, seed=11, step0=3 + k)
        dets = np.concatenate([moved, dets[done:]]) if done < len(dets) else moved
        if k >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * nw / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.system, "walkers_per_step": nw, "class_mix_at_start": mix},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                         "sample": f"{nw} walkers per timed step (at most {per_step:.0f} s each), one walker step "
                                   f"each, from the state after a 3-step untimed oracle walk (class mix {mix})"},
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
    groups = groups_per_rank(world)
    p = ctx.params(nw, args.warmup * inner, burn_in=0, seed=seed, n_groups=groups)
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
    combined = combine_ranks(ctx, groups, world, rank, int(res["total_steps"]))
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
    achieved = flops_per_step * units_per_launch / launch_s / 1e12
    peaks, peak_kind = load_peaks()
    probe = P.probe_peaks(local)
    sectors_per_s = gathers * units_per_launch / launch_s
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": (TRAFFIC_PER_WALKER_STEP[args.system] * units_per_launch
                        if args.system in TRAFFIC_PER_WALKER_STEP else None),
            "kernel": "k_walk2",
            "peak_source": "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (derived from unit counts and the "
                           "maximum SM clock)",
            "peak_measured": probe["fp64_flops"] / 1e12,
            "frac_of_measured": achieved / (probe["fp64_flops"] / 1e12),
            "flops_per_walker_step": flops_per_step, "terms_per_walker_step": terms,
            "neighbours_per_walker_step": nbrs, "launch_seconds": launch_s, "launches_timed": int(walk_launches),
            # the gather view of the same launches: every integral / table gather and hash-slot read is
            # one random 32-byte sector (the algorithmic sectors of the walk)
            "sectors_per_walker_step": gathers, "sectors_per_s": sectors_per_s,
            "l2_gather_peak_per_s": probe["l2_gathers_per_s"], "hbm_gather_peak_per_s": probe["hbm_gathers_per_s"],
            "l2_frac": sectors_per_s / probe["l2_gathers_per_s"],
            "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)), "hbm_peak_source": peak_kind}
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
        k_e2e = max(inner, 10)  # walker steps per call (the first, from the start determinant, is one of 10)
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
        # the oracle on the GPU walkers' own steady-state determinants (the same class mix), on all
        # host cores and on one core
        import oracle as O
        orc = O.Oracle.from_system(system)
        threads = os.cpu_count() or 1
        sample = snap1[:64]
        rate, done, _ = cpu_oracle_steps(orc, sample, args.cpu_seconds, threads)
        rate1, done1, _ = cpu_oracle_steps(orc, sample, args.cpu_seconds / 2, 1)
        mix = type_mix(orc, sample[:done])
        cpu = {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle",
               "one_core": {"value": rate1, "steps": done1},
               "sample": f"{done} walker steps of the oracle (local quantities with every reach-back overlap, "
                         f"then the move) from the GPU walkers' determinants after the timed region "
                         f"(class mix {mix}), at most {args.cpu_seconds:.0f} s; one core: {done1} steps"}

    # the metric's other half: batched and served against plain, on their own workloads
    batched = served = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = measure_batched(args.n_systems, args.batch_walkers, R=1, steps=1, warmup=1, tuned=False)
    if rank == 0 and world == 1 and not args.no_served:
        served = measure_served(args.n_requests, args.rate, args.target_sigma, args.req_walkers, args.req_max_steps,
                                args.max_active, args.budget_gb)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.system,
                       "orbitals": f"{system.n_core} core, {system.n_act} active, {system.n_virt} virtual",
                       "electrons": system.n_alpha + system.n_beta,
                       "reference_dets": int(len(system.coeffs)), "walkers_per_gpu": nw,
                       "walker_steps_per_launch": inner, "groups": groups, "method": "SC-NEVPT2(s) + E_L",
                       "l2": "256 MB buffer written between timed steps",
                       "neighbours_per_walker_step": nb_per_step, "candidates_per_walker_step": cand_per_step,
                       "class_mix": {P.TYPE_NAMES[t]: int(res["type_steps"][t]) for t in range(P.NTYPES)},
                       "e2": res["e2"], "e2_sigma": res["e2_sigma"],
                       # N > 1: the estimate of all ranks' walkers, finalized by rank 0 over the union
                       # of their groups
                       "all_ranks": combined},
            "clocks": clk.summary(),
            "roofline": roof,
            "e2e": e2e,
            # per step: slot keys, slot sort, walk, accumulate; finalize labels, finalize reduce
            "gpu_launches": 6 * args.steps,
            "cpu_baseline": cpu,
            "batched": batched,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_batched(n_systems: int, total_walkers: int, R: int, steps: int, warmup: int, max_act: int = 14,
                    tuned: bool = True):
    """Walker-steps/s of the batched workload (seeded systems of 30-120 orbitals, active spaces
    6-max_act, references of 400 to 5e5 determinants, walkers proportional to the reference size)
    run three ways with the same reporting interval of R walker steps (one finalize per system):
    plain (one system per launch, one after the other), batched (every system in one launch per
    determinant width and occupancy class) and batched with the autotuned launch configuration and
    CUDA-graph replay."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import synthetic as S
    specs, walkers = S.batch_specs(n_systems, total_walkers=total_walkers, max_act=max_act)
    t0 = time.perf_counter()
    systems = S.make_systems(specs, processes=min(16, os.cpu_count() or 1))
    t_gen = time.perf_counter() - t0
    import torch
    import paper_1909_06935_gb300 as P
    dev = torch.device("cuda", 0)
    ctxs = [P.Context.from_system(s) for s in systems]
    params = [c.params(nw, 0, burn_in=0, seed=500 + k, n_groups=8) for k, (c, nw) in enumerate(zip(ctxs, walkers))]
    total = sum(walkers)

    def plain_step():
        for c in ctxs:
            c.walkers_advance(R)
            c.finalize()

    def batched_step():
        P.batch_advance(ctxs, R)
        for c in ctxs:
            c.finalize()

    out, tune = {}, None
    modes = (("plain", plain_step), ("batched", batched_step)) + ((("batched_tuned", batched_step),) if tuned else ())
    for name, fn in modes:
        for c, p in zip(ctxs, params):
            c.walkers_init(p)
            c.set_launch()
        if name == "batched_tuned":     # autotune warps per walker and steps per launch, then graph replay
            tune = P.tune_batch(ctxs, trial_steps=min(R, 16))
            for c in ctxs:
                c.set_launch(tune["warps_per_walker"], min(tune["steps_per_launch"], R), True)
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize(dev)
        out[name] = total * R * steps / (time.perf_counter() - t0)
    for c in ctxs:
        c.set_launch()
        c.close()
    return {"plain": out["plain"], "batched": out["batched"], "batched_tuned": out.get("batched_tuned"),
            "speedup": out["batched"] / out["plain"],
            "speedup_tuned": out["batched_tuned"] / out["plain"] if "batched_tuned" in out else None,
            "unit": METRIC, "tuned_launch": tune, "steps": steps, "warmup": warmup, "steps_per_report": R,
            "config": {"workload": f"batch{n_systems}", "systems": n_systems, "walkers": total,
                       "active_orbitals": sorted({s.n_act for s in systems}),
                       "orbitals": [s.n_orb for s in systems], "reference_dets": [len(s.coeffs) for s in systems],
                       "generation_seconds": t_gen}}


def run_batched(args):
    """The batched workload at full size (64 systems, 32,768 walkers) as its own JSON line."""
    r = measure_batched(args.n_systems, 32768, max(1, args.inner), args.steps, args.warmup)
    line = {"metric": METRIC, "mode": "batched", "n_gpus": 1, "dtype": "f64", "data": "synthetic", **r}
    print(json.dumps(line), flush=True)


def served_pool(n_requests: int, seed: int = 77):
    """The served request stream: small seeded systems (12-18 orbitals, CAS(4e,4o) references) and a
    10-point geometry scan of one 16-orbital system (one orbital partition, L(lambda) = L0 + lambda dL),
    in a seeded random order.  Small enough that every request reaches sigma(E^(2)) <= 0.1 mHa within
    seconds on the GPU."""
    import synthetic as S
    rng = np.random.Generator(np.random.PCG64(seed))
    base = dict(n_core=2, n_act=4, n_virt=10, n_alpha=4, n_beta=4, rank=48, seed=3301, chol_sigma=0.06)
    pool = [S.workload("tiny_12o_cas4")]
    pool += [S.make_system(2, 4, 8 + 2 * k, 4, 4, rank=36 + 6 * k, seed=3400 + k, chol_sigma=0.06) for k in range(3)]
    scan = S.scan_systems(base, n_points=10)
    reqs = [pool[int(rng.integers(len(pool)))] for _ in range(max(0, n_requests - len(scan)))] + scan
    return [reqs[k] for k in rng.permutation(len(reqs))], len(scan)


def measure_served(n_requests: int, rate: float, target: float, req_walkers: int, max_steps: int,
                   max_active: int, budget_gb: float, steps_per_round: int = 20, seed: int = 77):
    """Time to a target sigma of E^(2) for a Poisson stream of requests, served (continuous batching,
    up to max_active requests resident) and plain (the same stream, one request resident at a time,
    first come first served).  Returns both with p50 / p99 time to target and throughput."""
    import paper_1909_06935_gb300 as P
    reqs, n_scan = served_pool(n_requests, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    gaps = rng.exponential(1.0 / rate, len(reqs))

    def one(active):
        srv = P.Server(max_active=active, hbm_budget_bytes=int(budget_gb * (1 << 30)), steps_per_round=steps_per_round)
        srv.start()
        t0 = time.perf_counter()
        tickets = []
        for k, s in enumerate(reqs):
            tickets.append(srv.submit(s, req_walkers, max_steps, target_sigma=target, burn_in=20, seed=900 + k,
                                      n_groups=16))
            time.sleep(gaps[k])
        while not all(srv.poll(t)["state"] in ("done", "failed", "cancelled") for t in tickets):
            time.sleep(0.02)
        wall = time.perf_counter() - t0
        srv.stop()
        st = [srv.poll(t) for t in tickets]
        steps = srv.info()["walker_steps"]
        srv.close()
        tt = np.array([x["total_seconds"] for x in st])
        reached = int(sum(x["result"]["e2_sigma"] <= target for x in st))
        return {"p50_s": float(np.percentile(tt, 50)), "p99_s": float(np.percentile(tt, 99)),
                "reached_target": reached, "requests": len(st), "throughput_req_per_s": len(st) / wall,
                "walker_steps_per_s": steps / wall, "failed": int(sum(x["state"] == "failed" for x in st))}

    served = one(max_active)
    plain = one(1)
    return {"metric": "time-to-target", "unit": "s", "target_sigma": target, "arrival_rate": rate,
            "served": served, "plain": plain,
            "p50_speedup": plain["p50_s"] / served["p50_s"], "p99_speedup": plain["p99_s"] / served["p99_s"],
            "config": {"workload": "served", "requests": len(reqs), "scan_points": n_scan,
                       "orbitals": sorted({int(s.n_orb) for s in reqs}),
                       "request_walkers": req_walkers, "max_steps": max_steps, "max_active": max_active,
                       "steps_per_round": steps_per_round}}


def run_served(args):
    r = measure_served(args.n_requests, args.rate, args.target_sigma, args.req_walkers, args.req_max_steps,
                       args.max_active, args.budget_gb)
    print(json.dumps({"mode": "served", "n_gpus": 1, "dtype": "f64", "data": "synthetic", **r}), flush=True)


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
