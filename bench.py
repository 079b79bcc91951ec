#!/usr/bin/env python
"""Benchmark of the recursive module-coupling eigensolver on B300.

Workload (one step): the XXZ Heisenberg chain N = 32, Delta = 1, bond couplings
J_i ~ U[0.5, 1.5] (seeded), leaves of 4 spins, k = 64 retained states per
level (effective dimension 4096, three boundary operators per bond), depth 3,
the 8 lowest states -- solved for a batch of independent instances, each
through the whole hot path (leaf build, every merge: diagonal and start block,
Chebyshev-filtered subspace iteration on the Kronecker-form product, FP64
finalisation, cut, gauge, operator rotation).

Metric: solves/s at 1e-8 relative energy error (a solve counts only if every
energy is within 1e-8 * max(1, |E|) of the oracle's stored value), with p50 /
p99 per-solve latency and the Kronecker-matvec throughput beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|fp64] [--batch B]

A step submits the batch to a solve server with ``--slots`` concurrent slots
(worker threads with their own CUDA streams) and waits for every result.
Under torchrun every rank solves its own batch of independent instances
(replicas: the solves shard with no exchange), timing is the max over ranks.
``--impl reference`` times the CPU oracle (the reference arm: there is no reference implementation).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The solve server runs one CUDA stream per slot; the driver maps streams onto
# CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 unless set), and kernels of
# streams that share a queue run in order, so with 16 slots a long one-CTA
# kernel of one solve holds back another's.  It must be set before the CUDA
# context exists (measured on one B300: 40.1 -> 73.5 solves/s with 32).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

import instances as I  # noqa: E402

GOLD = os.path.join(ROOT, "tests", "golden", "bench_xxz_n32_k64.json")
METRIC = "solves/s at 1e-8 energy error (XXZ N=32, k=64, 8 lowest states)"
UNIT = "solves/s"
RTOL = 1e-8
WORKLOAD = "xxz_n32_k64"
L2_FLUSH_BYTES = 512 << 20  # > 126 MB of L2

# Peak FP32 FMA throughput of the SIMT pipe: 148 SMs x 128 lanes x 2 FLOP x
# 2.032 GHz (unit counts and maximum clock of the part).
FP32_SIMT_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "mixed_tf32"])
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="skip the tile-tuning solve before warm-up")
    ap.add_argument("--profile-all-kinds", action="store_true",
                    help="time every kernel kind during the timed region (more host-side event records)")
    ap.add_argument("--workload", default="xxz", choices=["xxz", "serving"],
                    help="xxz: the batched XXZ N=32 k=64 benchmark (default); serving: Poisson request "
                         "stream of mixed chains through the continuous-batching server")
    ap.add_argument("--rates", default="10,100,1000", help="serving: arrival rates in requests/s")
    ap.add_argument("--requests", type=int, default=48, help="serving: requests per rate")
    ap.add_argument("--check", type=int, default=6, help="serving: requests re-solved alone in FP64 to check")
    return ap.parse_args()


def load_gold():
    with open(GOLD) as f:
        return {d["seed"]: np.array(d["energies"]) for d in json.load(f)["instances"]}


def batch_seeds(rank: int, batch: int, gold_seeds):
    """Rank r solves instances r*batch .. r*batch+batch-1 of the seed sequence
    (the first ones are those with stored oracle energies)."""
    base = sorted(gold_seeds)
    out = []
    for i in range(rank * batch, (rank + 1) * batch):
        out.append(base[i] if i < len(base) else I.seed_for(2) + 7919 * i)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("RMC_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def reduce_max(pg, value: float, device) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, value: float, device) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def chain_bytes(chain) -> int:
    """Host bytes the solve call copies in: term sites, Pauli letters, coefficients."""
    return len(chain.onsite) * (4 + 1 + 8) + len(chain.bonds) * (4 + 4 + 1 + 1 + 8)


# ---------------------------------------------------------------------------
# CPU legs: the oracle (allowed here only)
# ---------------------------------------------------------------------------

def _oracle_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        return max([d.get("num_threads", 1) for d in threadpool_info() if d.get("user_api") == "blas"] or [1])
    except Exception:
        return len(os.sched_getaffinity(0))


def oracle_merge_sample(chain, position: int):
    """Time the oracle on one merge (by post-order position) of the chain's
    recursion, leaves included for that merge: a bounded sample of one solve."""
    from oracle import rmc_oracle as O
    tree = O.split_tree(0, chain.n_sites, chain.leaf_sites)
    merges = []

    def collect(node, top):
        if isinstance(node[0], int):
            return
        collect(node[0], False)
        collect(node[1], False)
        merges.append((node, top))
    collect(tree, True)
    node, top = merges[position % len(merges)]
    # inputs of this merge: the two child blocks (built untimed)

    def build(nd, is_top):
        if isinstance(nd[0], int):
            return O.leaf_block(chain, nd[0], nd[1], chain.k, is_top)
        A = build(nd[0], False)
        B = build(nd[1], False)
        return O.merge_blocks(chain, A, B, chain.k, is_top)[0]
    A = build(node[0], False)
    B = build(node[1], False)
    t0 = time.perf_counter()
    O.merge_blocks(chain, A, B, chain.k, top)
    return time.perf_counter() - t0, len(merges)


def oracle_solve_time_estimate(chain, budget_s: float):
    """Estimate the oracle's time per solve from per-merge samples (each merge
    timed once, leaves timed once), stopping early when the budget runs out."""
    from oracle import rmc_oracle as O
    t0 = time.perf_counter()
    tree = O.split_tree(0, chain.n_sites, chain.leaf_sites)
    leaves = []

    def lv(nd):
        if isinstance(nd[0], int):
            leaves.append(nd)
        else:
            lv(nd[0]); lv(nd[1])
    lv(tree)
    for nd in leaves:
        O.leaf_block(chain, nd[0], nd[1], chain.k)
    leaf_t = time.perf_counter() - t0
    total = leaf_t
    _, n_m = oracle_merge_sample(chain, 0)
    sampled = 0
    for pos in range(n_m):
        dt, _ = oracle_merge_sample(chain, pos)
        total += dt
        sampled += 1
        if time.perf_counter() - t0 > budget_s:
            break
    if sampled < n_m:
        total = leaf_t + (total - leaf_t) * n_m / sampled
    return total, sampled, n_m


def run_reference(args):
    """The reference arm: the oracle as it stands (NumPy + LAPACK, dense eigh of
    every H_eff, Algorithm 1 as written) on the host cores.  A step is one whole
    oracle solve of one of the same seeded instances the GPU arm solves (about
    7 s on 16 host cores), so value is measured, not extrapolated."""
    from oracle import rmc_oracle as O
    # rank 0 alone runs it; the others exit without work (no process group:
    # the oracle needs no collective and no GPU)
    if int(os.environ.get("RANK", "0")) != 0:
        return
    gold = load_gold()
    seeds = batch_seeds(0, args.batch, gold.keys())
    chains = [I.xxz_n32(sd) for sd in seeds]
    for s in range(args.warmup):
        O.solve(chains[s % len(chains)])
    times, valid = [], 0
    for s in range(args.steps):
        sd = seeds[s % len(seeds)]
        t0 = time.perf_counter()
        E = O.solve(chains[s % len(chains)]).energies
        times.append(time.perf_counter() - t0)
        ref = gold.get(sd)
        valid += int(ref is not None and np.all(np.abs(E - ref) <= RTOL * np.maximum(1.0, np.abs(ref))))
    value = valid / sum(times)
    cores = _oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded XXZ chains, J_i ~ U[0.5,1.5])",
        "config": {"workload": WORKLOAD, "N": 32, "k": 64, "q": 8, "L0": 4, "delta": 1.0,
                   "precision": "fp64 dense eigh (oracle)", "l2": "n/a (CPU)"},
        "valid_solves": valid, "solves": args.steps,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} whole oracle solves (seeds {seeds[0]}...), one a step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def kernel_alone(P, torch, dev, reps: int = 20):
    """The fused Chebyshev filter alone (after the timed region) on the
    workload's dominant merge shape: 96 vectors of 64 x 64, three coupling
    operators, degree 10; CUDA events on the context's stream around `reps`
    launches.  FP32 on the FP32 pipe (the subspace iteration's filter) and FP64
    data in double-FP32 arithmetic (the refinement's filter).  Algorithmic
    FLOPs: 2 n_ops kA kB (kA + kB) + 3 kA kB per vector and product."""
    kA = kB = 64
    n_ops, nv, deg = 3, 96, 10
    rng = np.random.default_rng(7)
    EA, EB, oA, oB, coef = I.random_block_inputs(rng, kA, kB, n_ops)
    X = rng.standard_normal((nv, kA, kB))
    flops = nv * deg * (2.0 * n_ops * kA * kB * (kA + kB) + 3.0 * kA * kB)
    out = {}
    with P.Context(precision="mixed", device=dev.index) as ctx:
        stream = torch.cuda.ExternalStream(ctx.stream)
        for name, dtype, tdt in (("fused_filter_fp32", 1, torch.float32), ("fused_filter_df64", 3, torch.float64)):
            d = [torch.tensor(a, dtype=tdt, device=dev) for a in (EA, EB, oA, oB, X)]
            Y = torch.empty_like(d[4])
            torch.cuda.synchronize()

            def launch():
                ctx.cheb_filter(dtype, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                                d[3].data_ptr(), coef, d[4].data_ptr(), deg, -20.0, -10.0, 10.0, True, Y.data_ptr())
            for _ in range(3):
                launch()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                launch()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            tf = flops / (ms / 1e3) / 1e12
            if dtype == 1:
                out[name] = {"ms": ms, "achieved_tflops": tf, "peak_tflops": FP32_SIMT_PEAK_TFLOPS,
                             "frac": tf / FP32_SIMT_PEAK_TFLOPS, "bound": "alu", "ctas": nv,
                             "peak_source": "FP32 FMA pipe: 148 SMs x 128 lanes x 2 x 2.032 GHz"}
            else:
                out[name] = {"ms": ms, "achieved_fp64_equiv_tflops": tf, "fp64_pipe_peak_tflops": 1.13,
                             "ratio_to_fp64_pipe": tf / 1.13, "ctas": nv,
                             "note": "FP64-accurate products on the FP32 pipe (12 FP32 instructions each)"}
    return out


def run_ours(args):
    import torch

    import paper_2609_02394_b300 as P

    world, rank, local, pg = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gold = load_gold()
    seeds = batch_seeds(rank, args.batch, gold.keys())
    chains = [I.xxz_n32(s) for s in seeds]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # tile autotuning: one untimed solve of the first instance fills the
    # process-wide table the server's slots then read
    tiles = "untuned (first candidate of every product)"
    if not args.no_autotune:
        t0 = time.perf_counter()
        with P.Context(device=local, precision=args.precision) as tctx:
            tctx.autotune(chains[0])
        tiles = (f"autotuned: {len(P.tune_dump().splitlines())} shape bins, one tuning solve "
                 f"({time.perf_counter() - t0:.1f} s) before warm-up")
    srv = P.Server(slots=args.slots, device=local, precision=args.precision)

    def step():
        tids = [srv.submit(ch) for ch in chains]
        return [srv.poll(t, wait=True) for t in tids]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # live timing of the matvec kernel only (two event records per launch
    # group; timing every kind would add ~0.3 M event records a second to the
    # host's launch path); the per-kind breakdown comes from one profiled step
    # after the timed region
    kron_key = {"fp64": "kron_fp64", "mixed_tf32": "kron_working"}.get(args.precision, "fused_working")
    clocks = ClockSampler(local)
    clocks.start()
    l0 = srv.stats()["launches"]
    srv.profile(True, kinds=None if args.profile_all_kinds else [kron_key])
    srv.profile_read()
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms, lat_ms, queue_ms, valid, total = [], [], [], 0, 0
    e2e_s = 0.0
    for s in range(args.steps):
        flush.zero_()                       # evict the previous step's data from L2
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        t0 = time.perf_counter()
        outs = step()
        torch.cuda.synchronize()            # every slot's stream is idle here
        s1.record()
        s1.synchronize()
        e2e_s += time.perf_counter() - t0
        step_ms.append(s0.elapsed_time(s1))
        for (E, st, lat, qd), sd in zip(outs, seeds):
            lat_ms.append(lat)
            queue_ms.append(qd)
            total += 1
            ref = gold.get(sd)
            if st == 0 and ref is not None and np.all(np.abs(E - ref) <= RTOL * np.maximum(1.0, np.abs(ref))):
                valid += 1
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    wall = time.perf_counter() - wall0
    prof = srv.profile_read()
    l1 = srv.stats()["launches"]
    clk = clocks.stop()
    srv.profile(True)                       # every kind, one untimed step
    srv.profile_read()
    step()
    torch.cuda.synchronize()
    prof_all = srv.profile_read()
    srv.profile(False)
    srv.close()
    alone = kernel_alone(P, torch, dev) if rank == 0 else None

    dev_s = sum(step_ms) / 1e3
    max_dev_s = reduce_max(pg, dev_s, dev)
    max_e2e_s = reduce_max(pg, e2e_s, dev)
    valid_all = reduce_sum(pg, valid, dev)
    total_all = reduce_sum(pg, total, dev)

    # dominant kernel group and the Kronecker product's roofline
    # (algorithmic FLOPs / summed per-stream event time)
    # The Kronecker-form product is the path's matvec; in the mixed path it runs
    # as the single-launch Chebyshev filter (the two-stage form serves blocks
    # too wide for it).  Its per-launch times are the library's CUDA events on
    # each slot's stream over the timed region, so under concurrent slots they
    # include waits for SMs that other slots hold; kernel_alone gives the
    # same kernel timed by itself.
    dom = max(prof_all.items(), key=lambda kv: kv[1][2])
    kname = {"fp64": "Kronecker-form product, FP64 (fused and two-stage)",
             "mixed_tf32": "two-stage Kronecker-form product on tcgen05 (3xTF32)"}.get(
        args.precision, "cheb_fused_v4_kernel (single-launch FP32 Chebyshev filter)")
    kg, kl, kms, kfl = prof[kron_key]
    if args.precision == "fp64":
        peak, bound, peak_src = 1.13, "alu", "FP64 DFMA pipe, 1.13 TFLOP/s measured by a DFMA loop on this part"
    elif args.precision == "mixed_tf32":
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1800.0}
        peak = peaks["bf16_tflops"] * (1.1 / 2.25)
        bound = "tensor"
        peak_src = ("TF32 tensor peak = measured BF16 burst x nominal TF32/BF16 (1.1/2.25); the 3xTF32 "
                    "product executes 3 tensor products per useful one, so frac <= 1/3 by construction")
    else:
        peak, bound, peak_src = FP32_SIMT_PEAK_TFLOPS, "alu", "FP32 FMA pipe: 148 SMs x 128 lanes x 2 x 2.032 GHz"
    achieved = (kfl / (kms / 1e3)) / 1e12 if kms > 0 else 0.0
    whole_gpu = (kfl / dev_s) / 1e12 if dev_s > 0 else 0.0
    stream_ms = sum(v[2] for v in prof_all.values())
    breakdown = {k: {"launch_groups": v[0], "launches": v[1], "stream_ms": round(v[2], 3),
                     "share": round(v[2] / (stream_ms or 1), 4)} for k, v in prof_all.items()}
    breakdown["note"] = "one profiled step after the timed region, every kind timed (nested groups overlap)"

    if rank == 0:
        vals = sorted(lat_ms)
        p50 = vals[len(vals) // 2]
        p99 = vals[min(len(vals) - 1, int(round(0.99 * (len(vals) - 1))))]
        line = {
            "metric": METRIC, "value": valid_all / max_dev_s, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * max_dev_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "mixed_tf32": "tf32x3+f32+f64", "fp64": "f64"}[args.precision],
            "data": "synthetic (seeded XXZ chains, J_i ~ U[0.5,1.5])",
            "config": {"workload": WORKLOAD, "N": 32, "k": 64, "q": 8, "L0": 4, "delta": 1.0,
                       "batch_per_gpu": args.batch, "slots": args.slots, "precision": args.precision,
                       "parallelism": f"replicas x{world}", "l2": "flushed between steps (512 MB write)",
                       "tiles": tiles,
                       "timing": "CUDA events after device-wide synchronisation (work spans the slots' streams)"},
            "latency_ms": {"p50": p50, "p99": p99, "mean": statistics.mean(lat_ms),
                           "queue_p50": sorted(queue_ms)[len(queue_ms) // 2]},
            "valid_solves": int(valid_all), "solves": int(total_all),
            "matvec": {"tflops_per_stream": achieved, "tflops_whole_gpu": whole_gpu, "peak_tflops": peak,
                       "launch_groups": kg, "stream_ms": kms},
            "roofline": {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": None,
                         "peak_source": peak_src, "launches": kl,
                         "timing": "per-launch CUDA events on the slots' streams over the timed region "
                                   "(16 concurrent slots: intervals include waits for SMs)",
                         "dominant_group": dom[0], "dominant_share": round(dom[1][2] / (stream_ms or 1), 4)},
            "breakdown": breakdown,
            "kernel_alone": alone,
            "e2e": {"value": valid_all / max_e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(chain_bytes(c) for c in chains)),
                    "d2h_bytes_per_step": int(8 * sum(c.q for c in chains))},
            "gpu_launches": int(l1 - l0),
            "clocks": clk,
            "wall_s": wall,
        }
        if world == 1 and not args.no_cpu_baseline:
            est, sampled, n_m = oracle_solve_time_estimate(chains[0], budget_s=25.0)
            line["cpu_baseline"] = {"value": 1.0 / est, "unit": UNIT, "cores": _oracle_threads(), "kind": "oracle",
                                    "sample": f"one solve of seed {seeds[0]}: leaves + {sampled} of {n_m} merges "
                                              f"timed once each" + (", rest extrapolated" if sampled < n_m else "")}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_serving(args):
    """Serving: requests arrive as a Poisson stream (seeded) and are submitted on
    schedule to the continuous-batching server (slots run concurrently, each
    admitted under the 40 GB device-memory budget); latency is arrival to
    result.  A sample of requests is re-solved alone on the plain FP64 GPU path
    and compared within 1e-8 relative."""
    import torch

    import paper_2609_02394_b300 as P

    torch.cuda.init()
    budget = 40 << 30
    out = {"metric": "serving: solves/s and p50/p99 latency (arrival to result) at 1e-8 energy error",
           "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "dtype": "f32+f64" if args.precision == "mixed"
           else args.precision, "data": "synthetic (seeded mixed TFIM / XXZ / random-field request stream)",
           "config": {"workload": "serving", "N": "U{8..128}", "k": "{16,32,64,128,256}", "q": "U{1..16}",
                      "slots": args.slots, "mem_budget_gb": 40, "requests_per_rate": args.requests,
                      "precision": args.precision}, "rates": []}
    for ri, rate in enumerate(float(r) for r in args.rates.split(",")):
        reqs = I.serving_requests(args.requests, seed=I.seed_for(5) + ri)
        gaps = np.random.default_rng(I.seed_for(5) * 10 + ri).exponential(1.0 / rate, size=len(reqs))
        arrive = np.cumsum(gaps)
        srv = P.Server(slots=args.slots, precision=args.precision, mem_budget=budget)
        srv.profile(False)
        peak_reserved = 0
        t0 = time.perf_counter()
        tids, sub_t = [], []
        for i, r in enumerate(reqs):
            while time.perf_counter() - t0 < arrive[i]:
                time.sleep(min(0.001, max(0.0, arrive[i] - (time.perf_counter() - t0))))
            tids.append(srv.submit(r))
            sub_t.append(time.perf_counter() - t0)
            peak_reserved = max(peak_reserved, srv.stats()["reserved_bytes"])
        results = []
        for t in tids:
            while True:
                res = srv.poll(t, wait=False)
                if res is not None:
                    break
                peak_reserved = max(peak_reserved, srv.stats()["reserved_bytes"])
                time.sleep(0.002)
            results.append(res)
        torch.cuda.synchronize()
        srv.close()
        done_t = [s + res[2] / 1e3 for s, res in zip(sub_t, results)]
        ok = [res[1] == 0 for res in results]
        # accuracy sample: the cheapest requests, re-solved alone on the FP64 path
        order = sorted(range(len(reqs)), key=lambda i: (reqs[i].k, reqs[i].n_sites))[:args.check]
        checked, agree = 0, 0
        with P.Context(precision="fp64") as ctx:
            for i in order:
                if not ok[i]:
                    continue
                ref = ctx.solve_chain(reqs[i])
                checked += 1
                E = results[i][0]
                agree += int(np.all(np.abs(E - ref) <= RTOL * np.maximum(1.0, np.abs(ref))))
        lat = sorted(res[2] for res in results)
        span = max(done_t) - min(sub_t)
        out["rates"].append({
            "rate_req_s": rate, "requests": len(reqs), "completed_ok": int(sum(ok)),
            "solves_per_s": sum(ok) / span, "span_s": span,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))],
                           "max": lat[-1]},
            "queue_ms_p50": sorted(res[3] for res in results)[len(results) // 2],
            "peak_reserved_gb": peak_reserved / 2**30,
            "checked_vs_fp64": checked, "agree_within_1e-8": agree,
        })
        print(json.dumps(out["rates"][-1]), file=sys.stderr, flush=True)
    best = max(out["rates"], key=lambda r: r["solves_per_s"])
    out["value"] = best["solves_per_s"]
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
