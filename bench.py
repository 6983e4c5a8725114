#!/usr/bin/env python3
"""Benchmark of the hash- vs stride-seeded LCG path on GB300.

One step = the whole RNG microbenchmark workload on each GPU: 2^26 streams
(history ids rank*2^26 .. (rank+1)*2^26-1), each seeded by hash (s = 42) and,
separately, by stride (X0 = 1, Q = 152917), each drawing 64 uniforms through
libmc's fused seed+draw kernel, which writes every stream's final state and
the digest of its draws.  value = draws per second over all ranks.

Also reported: the dominant kernel's roofline (integer-issue bound), the
oracle on the host cores (cpu_baseline), an end-to-end number through the
public API including the device-to-host copy of every result, SM clocks
sampled during the timed region, and a `detail` object with seeding-only
rates and slab-transport histories/s (fp64 and fp32-guarded, single and
batched problems).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("particle histories/sec and RNG draws/sec on 1 GB300 "
          "(hash vs stride, % int-pipe roofline)")
N_STREAMS = 2**26
DRAWS = 64
# Integer operations per draw, two counts.  OPS_PER_DRAW is the count the
# hot-path table gives for one uniform of Eq. 1: the 64-bit multiply-add as
# IMAD.WIDE + 2 IMAD with the increment folded in (3), and at least 8 integer
# ALU operations to form the fp64 uniform (extract the 53 bits, count leading
# zeros, normalising shift, exponent insert).  The headline fraction uses it.
# OPS_PER_DRAW_KERNEL_FORM counts the summed form that csrc/rng.cu
# (draw_digest_m63_kernel, on the doubled state z = 2x) runs: the multiply-add
# (3); normalising shift, one bfind (1); the 53 uniform bits shifted into place
# as two words (4); the shift summed for the exponent field (1, fp32 pipe);
# digest add, one three-operand 64-bit add per two draws (1).  The exponent
# field and the range check fold into those sums, so the form never builds the
# fp64 value; both fractions are printed.
OPS_PER_DRAW = 11
OPS_PER_DRAW_KERNEL_FORM = 10
# DRAM bytes (read + write) per launch of the draw kernel at 2^26 streams, from
# an ncu capture of the kernel as built (mean of the hash and stride launches;
# profiles/draw_digest_m63_kernel_rng_microbench.md).
DRAW_KERNEL_TRAFFIC_BYTES = 1.013e9
# Streams of the materialised-uniform leg (fp64 uniforms stored, draw-major).
N_STREAMS_MATERIALISED = 2**22
# Executed thread instructions per flight of each transport kernel as built
# (ncu smsp__thread_inst_executed over every launch of a run, divided by its
# flights; profiles/transport_kernels_instructions_per_flight.md).  Times the
# measured flights/s, they place a transport workload against the issue peak.
INST_PER_FLIGHT = {
    "slab_small_fp64": 883, "slab_small_fp32": 741, "slab_long_fp64": 689, "slab_long_fp32": 523,
    "batched_fp64": 764, "batched_fp32": 604, "box_fp64": 2292, "box_fp32": 881,
    "box_fp64_event": 2697, "box_fp32_event": 1269,
    "pulse_hash": 366, "pulse_stride": 351, "pulse_census": 252,
}
# Bytes each flight of an event schedule moves through its particle bank: the
# particle's fields read and written once per iteration (slab: x, mu, w, the
# stream, draw and flight counts, history index, tally row, problem; box: the
# position, direction, inverse direction, weight and the same bookkeeping).
EVENT_BANK_BYTES_PER_FLIGHT = {"slab_fp64": 2 * 68, "slab_fp32": 2 * 60, "box_fp64": 2 * 128, "box_fp32": 2 * 88}
RECIPE_SM_MAX_MHZ = 2070.0
LANES_PER_SM_PER_CLK = 128  # 4 sub-partitions x 1 warp instruction x 32 lanes


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: MC_CLOCKS_DIR if set, else the system temporary directory
        out_dir = os.environ.get("MC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def int_issue_peak(num_sms):
    """Integer-issue roofline: every SM issues one warp instruction per clock
    on each of its 4 sub-partitions (128 lane-ops), at the recipe's maximum
    SM clock.  Returns lane-ops per second."""
    return num_sms * LANES_PER_SM_PER_CLK * RECIPE_SM_MAX_MHZ * 1e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# --------------------------------------------------------------------------- CPU

def oracle_draw_rate(target_cpu_s=12.0, threads=None):
    """The oracle (as it stands) on the host cores: hash- and stride-seeded
    streams, 64 draws each, on a bounded sample of the microbenchmark's ids.
    Returns (draws/s, threads, sample description)."""
    import oracle as O
    from paper_2403_06362_gb300 import workloads as W
    O.build()
    threads = threads or os.cpu_count() or 1

    def work(n, id0, out):
        a = O.seed_hash(W.LCG_M, W.HASH_SEED, id0, n)
        O.lcg_draw(W.LCG_M, W.LCG_G, W.LCG_C, a, DRAWS, want_u=False)
        b = O.seed_stride(W.LCG_M, W.LCG_G, W.LCG_C, W.STRIDE_X0, W.STRIDE_Q, id0, n)
        O.lcg_draw(W.LCG_M, W.LCG_G, W.LCG_C, b, DRAWS, want_u=False)
        out.append(n)

    t = time.perf_counter()
    work(4096, 0, [])
    per_stream = (time.perf_counter() - t) / 4096
    n_total = int(max(threads * 4096, min(N_STREAMS, target_cpu_s / per_stream)))
    per = n_total // threads
    ths, outs = [], []
    t = time.perf_counter()
    for i in range(threads):
        th = threading.Thread(target=work, args=(per, i * per, outs))
        th.start()
        ths.append(th)
    for th in ths:
        th.join()
    dt = time.perf_counter() - t
    draws = 2 * per * threads * DRAWS
    return draws / dt, threads, f"{per * threads} of the 2^26 ids (hash and stride), 64 draws each, {dt:.1f} s"


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle as O
    from paper_2403_06362_gb300 import workloads as W
    O.build()
    threads = os.cpu_count() or 1
    per = 2**15  # streams per thread per step and mode
    times = []

    def work(id0, n):
        a = O.seed_hash(W.LCG_M, W.HASH_SEED, id0, n)
        O.lcg_draw(W.LCG_M, W.LCG_G, W.LCG_C, a, DRAWS, want_u=False)
        b = O.seed_stride(W.LCG_M, W.LCG_G, W.LCG_C, W.STRIDE_X0, W.STRIDE_Q, id0, n)
        O.lcg_draw(W.LCG_M, W.LCG_G, W.LCG_C, b, DRAWS, want_u=False)

    def step(k):
        ths = [threading.Thread(target=work, args=(((k * threads + i) * per) % N_STREAMS, per))
               for i in range(threads)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()

    for k in range(args.warmup):
        step(k)
    for k in range(args.steps):
        t = time.perf_counter()
        step(args.warmup + k)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    draws = 2 * per * threads * DRAWS
    value = draws / (ms / 1e3)
    sample = f"{per * threads} streams per mode per step (of 2^26), 64 draws each"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "draws/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_block(),
        "cpu_baseline": {"value": value, "unit": "draws/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "draws/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def config_block():
    return {"workload": "rng microbenchmark: 2^26 streams per GPU (history ids), 64 uniforms each, "
                        "hash seeds (s=42) and stride seeds (X0=1, Q=152917), m=63 LCG "
                        "g=2806196910506780709 c=1; fused seed+draw, final state + digest per stream",
            "streams_per_gpu": N_STREAMS, "draws_per_stream": DRAWS, "modes": ["hash", "stride"],
            "l2": "L2 flushed before every step (256 MiB write); the step writes 1 GiB per mode"}


# --------------------------------------------------------------------------- GPU

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-detail", action="store_true")
    ap.add_argument("--profile-workload", default=None,
                    choices=["slab_long_fp64", "slab_long_fp32", "slab_small_fp64", "slab_small_fp32", "box_fp32", "box_fp64",
                             "batched_fp32", "batched_fp64", "pulse_hash", "pulse_stride", "pulse_census"],
                    help="run one transport workload (a warm-up run, then one run) and exit; for profilers")
    ap.add_argument("--histories", type=int, default=0, help="history count for --profile-workload")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1],
                    help="mc_run_config.schedule for --profile-workload (0 history, 1 event, as a captured graph)")
    ap.add_argument("--tally-atomics", type=int, default=0, choices=[0, 1, 2],
                    help="mc_run_config.tally_atomics for --profile-workload (0 library default, 1 per lane, "
                         "2 warp-aggregated)")
    ap.add_argument("--id-range", default=None,
                    help="B:E -- run only global histories [B, E) of --profile-workload (mc_run_config.range_*)")
    ap.add_argument("--block", type=int, default=0, help="mc_run_config.block for --profile-workload (0 default)")
    args = ap.parse_args()
    if args.profile_workload:
        return profile_workload(args)
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2403_06362_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import shard
    from paper_2403_06362_gb300 import workloads as W

    ctx = mc.Context(local)
    lcg = mc.make_lcg()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = N_STREAMS
    id0, _ = shard.weak_range(rank, n)  # this rank's block of stream ids
    specs = [mc.mc_seed_spec(mode=mc.MC_SEED_HASH, seed=W.HASH_SEED),
             mc.mc_seed_spec(mode=mc.MC_SEED_STRIDE, seed=W.STRIDE_X0, stride_q=W.STRIDE_Q)]
    st = [torch.empty(n, dtype=torch.int64, device=dev) for _ in specs]
    dg = [torch.empty(n, dtype=torch.int64, device=dev) for _ in specs]
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.int32, device=dev)

    def launch(i):
        mc.mc_lcg_draw(ctx, lcg, specs[i], id0, st[i], n, DRAWS, None, dg[i], stream)

    for _ in range(args.warmup):
        launch(0)
        launch(1)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        launch(0)
        ev[k][1].record(stream)
        launch(1)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    t_hash = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_str = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    ms_step = (sum(t_hash) + sum(t_str)) / args.steps
    if world > 1:
        t = torch.tensor([ms_step], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step = float(t.item())
    draws_per_step = 2 * n * DRAWS * world
    value = draws_per_step / (ms_step / 1e3)

    # Roofline of the dominant kernel (the fused seed+draw kernel): integer
    # issue.  achieved = hand-counted ops per draw x draws per launch / mean
    # launch time.
    props = torch.cuda.get_device_properties(dev)
    launch_ms = statistics.mean(t_hash + t_str)
    achieved = OPS_PER_DRAW * n * DRAWS / (launch_ms / 1e3)
    peak = int_issue_peak(props.multi_processor_count)
    roofline = {"bound": "alu", "kernel": "draw_digest_m63_kernel (fused seed + 64 draws, digest)",
                "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": DRAW_KERNEL_TRAFFIC_BYTES,
                "traffic_unit": "bytes per launch (ncu dram read+write)",
                "peak_note": f"derived: {props.multi_processor_count} SMs x 128 lane-ops/clk x "
                             f"{RECIPE_SM_MAX_MHZ:.0f} MHz (no measured integer peak exists)",
                "ops_per_draw": OPS_PER_DRAW,
                "ops_per_draw_kernel_form": OPS_PER_DRAW_KERNEL_FORM,
                "frac_kernel_form": OPS_PER_DRAW_KERNEL_FORM * n * DRAWS / (launch_ms / 1e3) / peak}

    # End to end through the public call on host buffers: mc_lcg_draw_host
    # returns every final state and digest into page-locked host memory
    # (2 GiB per step), slicing the range internally so that each slice's
    # device-to-host copy overlaps the next slice's kernel; the call returns
    # once the results are in host memory.  The device-to-host link (about
    # 190 GB/s measured on this machine) bounds the result.
    h_st = [torch.empty(n, dtype=torch.int64, pin_memory=True) for _ in specs]
    h_dg = [torch.empty(n, dtype=torch.int64, pin_memory=True) for _ in specs]
    e2e_steps = max(3, min(20, args.steps))
    for i in range(2):  # warm-up: the context's device slots and copy stream
        mc.mc_lcg_draw_host(ctx, lcg, specs[i], id0, h_st[i], n, DRAWS, h_dg[i], stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        for i in range(2):
            mc.mc_lcg_draw_host(ctx, lcg, specs[i], id0, h_st[i], n, DRAWS, h_dg[i], stream)
    torch.cuda.synchronize()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": draws_per_step / (e2e_ms / 1e3), "unit": "draws/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": 2 * 2 * n * 8,
           "note": "one mc_lcg_draw_host call per mode on page-locked host buffers, host clock around the calls; "
                   "inputs are scalars (seed, id range); every final state and digest reaches host memory"}

    detail = {"draws_per_s_hash": n * DRAWS * world / (statistics.mean(t_hash) / 1e3),
              "draws_per_s_stride": n * DRAWS * world / (statistics.mean(t_str) / 1e3),
              "ms_hash": statistics.mean(t_hash), "ms_stride": statistics.mean(t_str)}
    if not args.no_detail and rank == 0:
        detail.update(seeding_detail(mc, ctx, lcg, torch, dev, stream))
        detail.update(materialised_detail(mc, ctx, lcg, torch, dev, stream, specs))
        detail.update(transport_detail(mc, ctx, lcg, torch, dev, stream, W))

    del st, dg, flush
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_draw_rate()
        cpu = {"value": rate, "unit": "draws/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "draws/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": config_block(),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": 2 * args.steps, "detail": detail,
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def profile_workload(args):
    """One transport workload, run twice (warm-up + measured), for ncu."""
    import torch
    torch.cuda.set_device(0)
    from paper_2403_06362_gb300 import _build
    _build.build()
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import workloads as W
    ctx = mc.Context(0)
    lcg = mc.make_lcg()
    name = args.profile_workload
    keep = None
    if name.startswith("pulse"):
        # --histories N: N // 10^6 repetitions of 1000 x 1000 (default 30)
        reps = max(1, args.histories // 10**6) if args.histories else 30
        if name == "pulse_census":
            a = W.azurv1(seeding=W.SEED_HASH_HIER, n_census=20, n_reps=reps)
        else:
            a = W.azurv1(seeding=W.SEED_HASH_HIER if name.endswith("hash") else W.SEED_STRIDE, n_reps=reps)
        prob, keep = W.to_mc_pulse(a, mc)
        cp = mc.problem_array([prob])
        tally = mc.Tally(W.azurv1_tally_slots(a), 1)
        n = W.azurv1_histories(a)
    elif name.startswith("box"):
        b = W.box_large(W.SEED_HASH, n_histories=args.histories or 10**6)
        prob, keep = W.to_mc_box(b, mc)
        cp = mc.problem_array([prob])
        tally = mc.Tally(W.box_tally_slots(b), 1)
        n = b["n_histories"]
    else:
        if name.startswith("slab_long"):
            probs = W.slab_long(W.SEED_HASH, n_histories=args.histories or 10**5)
        elif name.startswith("slab_small"):
            probs = W.slab_small(W.SEED_HASH, n_histories=args.histories or 10**4)
        else:
            probs = W.slab_batched(W.SEED_HASH_HIER)
        cp = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
        tally = mc.Tally(W.tally_slots(probs), len(probs))
        n = sum(p["n_histories"] for p in probs)
    rb, re_ = (int(v) for v in args.id_range.split(":")) if args.id_range else (0, 0)
    cfg = mc.mc_run_config(precision=1 if "fp32" in name else 0, tally_atomics=args.tally_atomics,
                           schedule=args.schedule, use_graph=args.schedule, range_begin=rb, range_end=re_,
                           block=args.block)
    times = []
    for _ in range(2):
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mc.mc_transport_run(ctx, lcg, cp, cfg, tally.c)
        b2.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b2))
    flights = int(tally.counts.view(-1, 17)[:, 1].sum().item())  # over every problem
    print(json.dumps({"workload": name, "histories": n, "ms": times[-1], "flights": flights}))
    del keep
    ctx.close()


def seeding_detail(mc, ctx, lcg, torch, dev, stream):
    """Seeding only (mc_seed_hash / mc_seed_stride), HBM-store bound:
    8 bytes written per stream."""
    peaks, src = measured_peaks()
    n = N_STREAMS
    out = torch.empty(n, dtype=torch.int64, device=dev)
    res = {}
    for name, fn in (("hash", lambda: mc.mc_seed_hash(ctx, lcg, 42, 0, n, out, stream)),
                     ("stride", lambda: mc.mc_seed_stride(ctx, lcg, 1, 152917, 0, n, out, stream))):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(20):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ts)
        gbs = n * 8 / (ms / 1e3) / 1e9
        res[f"seeds_per_s_{name}"] = n / (ms / 1e3)
        res[f"seed_{name}_hbm"] = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": gbs / peaks["hbm_gbs"], "peak_source": src}
    return res


def materialised_detail(mc, ctx, lcg, torch, dev, stream, specs):
    """Mode (iii) of the microbenchmark: seeding plus 64 draws with every fp64
    uniform stored (draw-major, u[j][i]) and the final states, for the first
    2^22 of the 2^26 ids, hash- and stride-seeded.  HBM-store bound:
    8 bytes per draw plus 8 per stream written."""
    peaks, src = measured_peaks()
    n = N_STREAMS_MATERIALISED
    u = torch.empty(n * DRAWS, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int64, device=dev)
    res = {}
    for name, spec in zip(("hash", "stride"), specs):
        for _ in range(3):
            mc.mc_lcg_draw(ctx, lcg, spec, 0, st, n, DRAWS, u, None, stream)
        ts = []
        for _ in range(20):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mc.mc_lcg_draw(ctx, lcg, spec, 0, st, n, DRAWS, u, None, stream)
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ts)
        nbytes = n * DRAWS * 8 + n * 8
        gbs = nbytes / (ms / 1e3) / 1e9
        res[f"materialised_uniforms_{name}"] = {
            "streams": n, "draws_per_stream": DRAWS, "ms": ms, "draws_per_s": n * DRAWS / (ms / 1e3),
            "roofline": {"bound": "hbm", "kernel": "draw_kernel (uniforms stored)", "achieved": gbs,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                         "peak_source": src, "bytes_per_launch": nbytes}}
    del u, st
    return res


def transport_detail(mc, ctx, lcg, torch, dev, stream, W):
    """Transport throughput on the slab and box workloads (histories/s), the
    batched slab problems (one fp32 launch vs the plain fp64 single-problem
    loop), history vs event schedules with a bit-identity check, and the
    Section 5 normality procedure on the batch means, hash vs stride."""
    res = {}

    def timed(probs, reps=2, box=None, keep=False, hist=False, **cfgkw):
        if box is not None:
            prob, spec = W.to_mc_box(box, mc)
            cp = mc.problem_array([prob])
            tally = mc.Tally(W.box_tally_slots(box), 1)
            tally._keep = spec
        else:
            cp = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
            tally = mc.Tally(W.tally_slots(probs), len(probs),
                             n_histories=sum(q["n_histories"] for q in probs) if hist else 0)
        cfg = mc.mc_run_config(**cfgkw)
        mc.mc_transport_run(ctx, lcg, cp, cfg, tally.c, stream)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mc.mc_transport_run(ctx, lcg, cp, cfg, tally.c, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        return best, tally, cp

    peaks, peak_src = measured_peaks()
    issue_peak = int_issue_peak(torch.cuda.get_device_properties(dev).multi_processor_count)

    def issue_roofline(flights_per_s, key):
        ops = INST_PER_FLIGHT[key]
        ach = flights_per_s * ops
        return {"bound": "issue", "achieved": ach / 1e12, "peak": issue_peak / 1e12, "unit": "Tops/s",
                "frac": ach / issue_peak, "ops_per_flight": ops,
                "ops_note": "executed thread instructions per flight (ncu); derived issue peak"}

    def bank_roofline(flights_per_s, key):
        b = EVENT_BANK_BYTES_PER_FLIGHT[key]
        gbs = flights_per_s * b / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "bytes_per_flight": b, "peak_source": peak_src,
                "note": "particle bank read and written once per flight; not the bound (see DESIGN)"}

    def entry(ms, tally, cp, n, idx=0, key=None):
        r = mc.mc_tally_read(ctx, cp, idx, tally.c, stream, check=False)
        flights = int(tally.counts.view(-1, 17)[:, 1].sum().item())  # over every problem
        e = {"ms": ms, "histories_per_s": n / (ms / 1e3), "flights_per_s": flights / (ms / 1e3),
             "exceed_hist": r.counts["exceed_hist"], "max_draws": r.counts["max_draws"]}
        if key is not None:
            e["roofline"] = issue_roofline(flights / (ms / 1e3), key)
        return e

    for name, fn in (("slab_small", W.slab_small), ("slab_long", W.slab_long)):
        for sname, sd in (("hash", W.SEED_HASH), ("stride", W.SEED_STRIDE)):
            p = fn(sd)
            n = p[0]["n_histories"]
            for prec in (0, 1):
                ms, tally, cp = timed(p, reps=3 if name == "slab_small" else 1, hist=True, precision=prec)
                e = entry(ms, tally, cp, n, key=f"{name}_{'fp32' if prec else 'fp64'}")
                if prec == 0:
                    hist_bins = tally.bins.clone()
                    hist_state64 = tally.hist_state.clone()
                    r64 = mc.mc_tally_read(ctx, cp, 0, tally.c, stream, check=False)
                else:
                    # fp32-guarded flux against the fp64 flux, per bin: relative
                    # difference and the difference in fp64 standard errors
                    r32 = mc.mc_tally_read(ctx, cp, 0, tally.c, stream, check=False)
                    d = np.abs(r32.flux - r64.flux)
                    f64 = np.abs(r64.flux)
                    se = r64.rel_err * f64
                    e["fp32_vs_fp64_rel_diff_max"] = float(np.max(np.where(f64 > 0, d / np.where(f64 > 0, f64, 1), 0)))
                    e["fp32_vs_fp64_diff_in_se_max"] = float(np.max(np.where(se > 0, d / np.where(se > 0, se, 1), 0)))
                    # histories whose fp32 run ended in another state: a
                    # decision went the other way somewhere in them
                    e["fp32_histories_diverged"] = int((tally.hist_state != hist_state64).sum().item())
                res[f"{name}_{sname}_{'fp32' if prec else 'fp64'}"] = e
            ms, tally, cp = timed(p, reps=1, precision=0, schedule=1, use_graph=1)
            e = entry(ms, tally, cp, n)
            e["roofline"] = bank_roofline(e["flights_per_s"], "slab_fp64")
            e["bits_identical_to_history"] = bool(torch.equal(tally.bins, hist_bins))
            res[f"{name}_{sname}_fp64_event"] = e

    # Section 5: normality of the batch means, per bin, hash vs stride; and
    # the per-bin difference of the two tallies in standard errors (both
    # estimate the same flux with independent streams, so z ~ N(0, 1))
    norm = {}
    for name, fn in (("slab_small", W.slab_small), ("slab_long", W.slab_long)):
        reads = {}
        for sname, sd in (("hash", W.SEED_HASH), ("stride", W.SEED_STRIDE)):
            p = fn(sd)
            _, tally, cp = timed(p, reps=0, precision=0)
            r = mc.mc_tally_read(ctx, cp, 0, tally.c, stream)
            reads[sname] = r
            _, wv, pv = mc.mc_normality(r.batch)
            norm[f"{name}_{sname}"] = {"batches": int(r.batch.shape[0]), "points": int(r.batch.shape[1]),
                                       "fails_p_lt_0.05": int(np.sum(pv < 0.05)),
                                       "min_p": float(np.min(pv)), "median_p": float(np.median(pv))}
        h, st = reads["hash"], reads["stride"]
        se = np.sqrt((h.rel_err * h.flux) ** 2 + (st.rel_err * st.flux) ** 2)
        z = (h.flux - st.flux) / np.where(se > 0, se, 1.0)
        norm[f"{name}_hash_minus_stride"] = {"bins": int(z.size), "max_abs_z": float(np.max(np.abs(z))),
                                             "mean_z": float(np.mean(z)), "bins_abs_z_gt_3": int(np.sum(np.abs(z) > 3))}
    res["normality"] = norm

    # 256 batched slab problems
    probs = W.slab_batched(W.SEED_HASH_HIER)
    nh = sum(p["n_histories"] for p in probs)
    # the fp32 variants (eager, graph replay, autotuned) in three interleaved
    # rounds, the best of each: a 20 ms launch moves with the GPU's power
    # state over a long run, and interleaving keeps that out of the comparison
    ms32 = ms32g = ms32a = ms64 = float("inf")
    for _ in range(3):
        m, t32, _ = timed(probs, reps=1, precision=1)
        ms32 = min(ms32, m)
        ms32g = min(ms32g, timed(probs, reps=1, precision=1, use_graph=1)[0])
        ms32a = min(ms32a, timed(probs, reps=1, precision=1, schedule=2)[0])
        m, t64, _ = timed(probs, reps=1, precision=0)
        ms64 = min(ms64, m)
    # fp32-guarded against fp64: per-bin relative difference of the tallies
    # and the histories whose final stream state differs (a decision that went
    # the other way), from one untimed run of each with per-history outputs
    g32 = t32.bins.cpu().numpy().astype(np.float64)
    g64 = t64.bins.cpu().numpy().astype(np.float64)
    nzb = g64 != 0
    rel = np.abs(g32[nzb] - g64[nzb]) / np.abs(g64[nzb])
    cp_h = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    hs = {}
    for prec in (0, 1):
        th = mc.Tally(W.tally_slots(probs), len(probs), n_histories=nh)
        mc.mc_transport_run(ctx, lcg, cp_h, mc.mc_run_config(precision=prec), th.c, stream)
        torch.cuda.synchronize()
        hs[prec] = th.hist_state.cpu().numpy()
        del th
    diverged = int(np.count_nonzero(hs[0] != hs[1]))
    del hs
    singles = []
    for p in probs:
        q = dict(p)
        q["tally_offset"] = 0
        singles.append((mc.Tally(W.tally_slots([q]), 1), mc.problem_array([W.to_mc_problem(q, mc)])))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for tl, cp in singles:
        mc.mc_transport_run(ctx, lcg, cp, mc.mc_run_config(), tl.c, stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms_single = a.elapsed_time(b)
    best32 = min(ms32, ms32g, ms32a)
    res["slab_batched"] = {"histories": nh, "ms_batched_fp32": ms32, "ms_batched_fp32_graph": ms32g,
                           "ms_batched_fp32_autotuned": ms32a, "ms_batched_fp64": ms64,
                           "ms_single_fp64_loop": ms_single,
                           "histories_per_s_batched_fp32": nh / (best32 / 1e3),
                           "speedup_batched_fp32_over_single_fp64": ms_single / best32,
                           "fp32_vs_fp64_bin_rel_diff": {"max": float(rel.max()), "median": float(np.median(rel)),
                                                         "bins": int(rel.size)},
                           "fp32_histories_diverged": diverged}
    fl32 = int(t32.counts.view(-1, 17)[:, 1].sum().item())
    fl64 = int(t64.counts.view(-1, 17)[:, 1].sum().item())
    res["slab_batched"]["roofline_fp32"] = issue_roofline(fl32 / (ms32 / 1e3), "batched_fp32")
    res["slab_batched"]["roofline_fp64"] = issue_roofline(fl64 / (ms64 / 1e3), "batched_fp64")

    # Section 5 experiment: 30 repetitions x 1000 batches x 1000 sources, hash
    # (hierarchical seeds) vs stride; Shapiro-Wilk on each of the 20 points
    # over the 1000 batch means, per repetition (600 tests per mode)
    # ("census_hash": the same with 20 census phases and population control
    # by one-off hashed values back to 1000 per batch at every census)
    for sname, sd, nc in (("hash", W.SEED_HASH_HIER, 0), ("stride", W.SEED_STRIDE, 0),
                          ("census_hash", W.SEED_HASH_HIER, 20)):
        a = W.azurv1(seeding=sd, n_census=nc)
        prob, spec = W.to_mc_pulse(a, mc)
        cp = mc.problem_array([prob])
        tally = mc.Tally(W.azurv1_tally_slots(a), 1)
        cfg = mc.mc_run_config()
        mc.mc_transport_run(ctx, lcg, cp, cfg, tally.c, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mc.mc_transport_run(ctx, lcg, cp, cfg, tally.c, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r = mc.mc_tally_read(ctx, cp, 0, tally.c, stream)
        flux = r.batch.reshape(a["n_reps"], a["n_batches"], a["n_time_bins"])
        pvals = np.array([mc.mc_normality(flux[k])[2] for k in range(a["n_reps"])])  # [rep][point]
        n = W.azurv1_histories(a)
        res[f"pulse_paper_{sname}"] = {
            "ms": ms, "source_histories_per_s": n / (ms / 1e3), "collisions_per_s": r.counts["collisions"] / (ms / 1e3),
            "census_per_source": r.counts["leak_hi"] / n, "secondaries": r.counts["children"],
            "sw_fails_p_lt_0.05": int(np.sum(pvals < 0.05)), "sw_tests": int(pvals.size),
            "sw_median_p_per_point": [float(v) for v in np.median(pvals, axis=0)],
            "roofline": issue_roofline(r.counts["flights"] / (ms / 1e3),
                                       {"hash": "pulse_hash", "stride": "pulse_stride",
                                        "census_hash": "pulse_census"}[sname])}
        if nc:
            res[f"pulse_paper_{sname}"].update(
                n_census=nc, flights=r.counts["flights"], banked=r.counts["banked"],
                copies_beyond_first=r.counts["splits"], no_copy=r.counts["roulette_kills"])
        else:
            res[f"pulse_paper_{sname}"].update(
                paper_fails_context={"hash": "339/600", "stride": "369/600"}[sname],
                paper_runtime_context={"hash": "111.46 s (serial Python)", "stride": "113.26 s (serial Python)"}[sname])
        del spec

    # 3D two-region box, 10^8 source histories
    box = W.box_large(W.SEED_HASH)
    n = box["n_histories"]
    bits = {}
    for label, kw in (("fp32_history", dict(precision=1)), ("fp32_event", dict(precision=1, schedule=1, use_graph=1)),
                      ("fp64_history", dict(precision=0)), ("fp64_event", dict(precision=0, schedule=1, use_graph=1))):
        ms, tally, cp = timed(None, reps=1, box=box, **kw)
        prec = "fp32" if label.startswith("fp32") else "fp64"
        e = entry(ms, tally, cp, n, key=f"box_{prec}" + ("_event" if "event" in label else ""))
        if "event" in label:
            e["roofline_bank"] = bank_roofline(e["flights_per_s"], f"box_{prec}")
        r = mc.mc_tally_read(ctx, cp, 0, tally.c, stream, check=False)
        e.update(children=r.counts["children"], splits=r.counts["splits"], roulette_kills=r.counts["roulette_kills"])
        bits[label] = tally.bins.clone()
        res[f"box_large_hash_{label}"] = e
    res["box_large_hash_fp32_event"]["bits_identical_to_history"] = bool(torch.equal(bits["fp32_event"],
                                                                                      bits["fp32_history"]))
    res["box_large_hash_fp64_event"]["bits_identical_to_history"] = bool(torch.equal(bits["fp64_event"],
                                                                                      bits["fp64_history"]))
    # fp32-guarded mesh against fp64, voxel by voxel (the box's fp32 path keeps
    # plain fp32 positions)
    m32 = bits["fp32_history"].cpu().numpy().astype(np.float64)
    m64 = bits["fp64_history"].cpu().numpy().astype(np.float64)
    nz = m64 != 0
    vrel = np.abs(m32[nz] - m64[nz]) / np.abs(m64[nz])
    res["box_large_hash_fp32_history"]["fp32_vs_fp64_voxel_rel_diff"] = {
        "max": float(vrel.max()), "median": float(np.median(vrel)), "voxels": int(vrel.size),
        "total_rel_diff": float(abs(m32.sum() - m64.sum()) / m64.sum())}
    del bits
    return res


if __name__ == "__main__":
    main()
