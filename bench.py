#!/usr/bin/env python3
"""Benchmark of the data-parallel GKR prover: gates proved per second.

One step = the whole hot path over one batch of synthetic input: forward
evaluation of every layer from device-resident inputs, statement digests,
transcript, and the GKR layer sumcheck of every layer (copy phase, Libra's
x and y phases), ending with the proof bytes on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload slot|medium|tiny|batched|served|assoc]

The default workload is the slot-shaped circuit (32768 copies x 1024 gates
x 24 mixing layers, the largest configuration one GPU holds).  The same
JSON line carries the batched workload (64 independent instances of uneven
size, proofs/s against one instance at a time) and a served run (Poisson
arrivals into the continuous-batching server, p50/p99 latency and proofs/s
against the plain path measured on the same arrival trace); ``--workload
batched`` and ``--workload served`` run those alone at full size.

``--workload assoc`` times the second data-parallel workload of the paper:
the associative hash (Sec. 3.4.1) of every slot's validator indexes and the
pairwise-distinct check (Sec. 3.4.2) of every epoch, in validator indexes
per second.

With N > 1 (launched by torchrun, one rank per GPU) every rank proves its
own instance of the workload: independent proofs, no data-path collective
("replicas", weak scaling).  ``--impl reference`` times the CPU oracle (the
plain C implementation the tests check against) on a bounded sample of the
same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gates proved/sec (field mults/s vs roofline); batched proofs/sec and p99 latency vs plain"
UNIT = "gates/s"
# The binding unit of this path is the integer pipe: exact 256-bit modular
# products on 32-bit multiply-adds, no tensor cores.  Its peak is measured
# in the run (independent mad.lo chains on every SM, best of a second of
# launches), beside the derived 148 SMs x 64 multiply-adds per SM per clock
# x 2032 MHz.  One Montgomery product of 8-limb operands (CIOS) counts as
# 2*64 multiply halves for a*b plus 8 + 2*64 for the reduction = 264
# multiply-adds.  The copy round's algorithmic work is 2 + 4 f products per
# (pair, gate) item, f the share of mul gates: a mul gate's three products
# and three weight products at t = 0, 1, 2, an add gate's two weighted
# sums (t = 3 follows from the quadratic).
SMS, IMAD_PER_SM_CLK, SM_MAX_MHZ = 148, 64, 2032.0
IMAD_PER_FR_MUL = 264
ALU_PEAK_TIMAD = SMS * IMAD_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
# DRAM traffic (read + write bytes) of the dominant kernel per (pair, gate)
# item, from an ncu capture of the copy rounds of a slot-shaped layer (the
# first layers of the slot workload: every layer has the same shape, so the
# per-item traffic of a full-size launch is the same), with the launch
# shapes the tuner picks for those rounds; None when not captured for the
# current build of the kernel.
DOMINANT_TRAFFIC_BYTES_PER_ITEM = 3721676544 / 33553408


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload(name: str, depth: int | None = None):
    import synth
    circ = {"tiny": synth.tiny, "medium": synth.medium, "slot": synth.slot}[name]()
    if depth:  # the workload's first `depth` layers (for profiler captures)
        circ = synth.Circuit(circ.widths[:depth + 1], circ.types[:depth], circ.in1[:depth], circ.in2[:depth],
                             circ.n_copies, name=f"{circ.name}_first{depth}", seed=circ.seed, meta=circ.meta)
    return circ


def describe(circ) -> str:
    return (f"{circ.name}: {circ.n_copies} copies x {circ.widths[0]} gates x {circ.depth} layers, "
            f"{circ.meta.get('pct_mul')}% mul, {circ.meta.get('wiring')} wiring, seed {circ.seed}")


def gates_of(circ) -> int:
    return circ.n_copies * circ.gates_per_copy()


def gpu_uuid(dev):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


def host_cpu() -> dict:
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


# ---------------------------------------------------------------------------
# clocks during the timed region

FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
          "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
          "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class Clocks:
    def __init__(self, gpu: str | None):
        self.f = tempfile.TemporaryFile(mode="w+")
        cmd = ["nvidia-smi", f"--query-gpu={FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu:
            cmd += ["-i", gpu]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.t0 = self.t1 = None

    def mark(self, start: bool):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 - 1 <= r[0] <= self.t1 + 1] or rows
        sm = sorted(r[1] for r in inside)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k in range(4) if r[3][k].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[2] for r in inside), "reasons": reasons,
                "samples": len(inside)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)

def oracle_sample(name: str, layers: int, copies: int):
    """The workload's shape cut to ``copies`` copies and its first ``layers``
    layers (same widths, gate mix and wiring generator)."""
    import synth
    if name == "slot":
        return synth.mixing_circuit(3, copies, 1024, layers,
                                    name=f"slot-shaped sample: {copies} copies x 1024 gates x {layers} layers")
    w = {"tiny": 1024, "medium": 4096}[name]
    seed = {"tiny": 1, "medium": 2}[name]
    return synth.uniform_circuit(seed, copies, [w] * (layers + 1), 50,
                                 name=f"{name}-shaped sample: {copies} copies x {w} gates x {layers} layers")


def time_oracle(circ, threads: int = 1):
    import synth
    from oracle import Oracle
    o = Oracle()
    used = o.set_threads(threads)
    xb = synth.fr_bytes(synth.inputs_for(circ))
    o.proof_len(circ)
    t0 = time.perf_counter()
    o.prove(circ, xb)
    secs = time.perf_counter() - t0
    o.set_threads(1)
    return secs, used


def cpu_baseline(name: str):
    """The oracle on the host cores: all of them (OpenMP over copy pairs,
    rows and copies), and one thread on a smaller sample."""
    cores = os.cpu_count() or 1
    big = oracle_sample(name, 2, 4096 if name == "slot" else 1024)
    secs, used = time_oracle(big, cores)
    small = oracle_sample(name, 1, 1024 if name == "slot" else 256)
    secs1, _ = time_oracle(small, 1)
    return {"value": gates_of(big) / secs, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{big.name} (one proof incl. evaluation, {gates_of(big)} gates, {secs:.1f} s on {used} "
                      f"threads of the host's {cores})",
            "single_thread": {"value": gates_of(small) / secs1, "unit": UNIT, "cores": 1,
                              "sample": f"{small.name} ({gates_of(small)} gates, {secs1:.1f} s)"},
            "host": host_cpu()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    circ_full = workload(args.workload)
    cores = os.cpu_count() or 1
    circ = oracle_sample(args.workload, 1, 1024 if args.workload == "slot" else 256)
    for _ in range(args.warmup):
        time_oracle(circ, cores)
    total, used = 0.0, 1
    for _ in range(args.steps):
        secs, used = time_oracle(circ, cores)
        total += secs
    value = args.steps * gates_of(circ) / total
    sample = f"{circ.name} per step ({gates_of(circ)} gates, one proof incl. evaluation, {used} threads)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": describe(circ_full), "sample": circ.name},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# replicas over ranks (torchrun, one process per GPU)

def max_over_ranks(x: float, world: int, dev) -> float:
    """The largest value over the ranks of the default process group (a
    time: the job ends with its slowest rank); x itself with one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, steps: int, units_per_step: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each processed `steps`
    steps of `units_per_step` units within `seconds` (the slowest rank's)."""
    return world * steps * units_per_step / seconds


# ---------------------------------------------------------------------------
# the CUDA path

def measure_imad_peak(S, stream, uuid):
    """The integer pipe's multiply-add rate on this GPU: independent mad.lo
    chains on every SM, the best launch of about a second of them, with the
    SM clocks sampled meanwhile."""
    clocks = Clocks(uuid)
    time.sleep(0.3)
    clocks.mark(True)
    best, t_end, n = 0.0, time.time() + 1.2, 0
    while time.time() < t_end or n < 3:
        ms, ops = S.microbench(0, SMS * 8, 256, 16384, stream.cuda_stream)
        best = max(best, ops / (ms / 1e3) / 1e12)
        n += 1
    clocks.mark(False)
    clk = clocks.stop()
    ms_fr, ops_fr = S.microbench(2, SMS * 8, 256, 256, stream.cuda_stream)
    return {"tops": best, "launches": n, "clocks": clk, "fr_mul_gops": ops_fr / (ms_fr / 1e3) / 1e9,
            "how": "k_mb_madlo: 1184 CTAs x 256 threads, 8 independent mad.lo.u32 chains a thread, "
                   "best of the launches in about a second (CUDA events)"}


def copy_phase_equivalent(circ, breakdown: dict, peak: float) -> dict:
    """The copy phase as a whole (row sums, rounds, folds) against the
    item-by-item count of its work: 2 + 4 f products a (pair, gate) item for
    the round sums (a mul gate's three products and three weight products at
    t = 0, 1, 2; an add gate's two weighted sums) and one product a folded
    row element.  The recurrence form reaches the same sums with fewer
    products, so this is the rate at which the phase delivers that work, in
    Montgomery-product units of 264 multiply-adds, not the rate at which its
    kernels issue products (the dominant kernel's `frac` is that)."""
    import numpy as np
    rounds = (circ.n_copies - 1).bit_length()
    pairs = sum(circ.n_copies >> (k + 1) for k in range(rounds))
    sums = sum(pairs * (2 * circ.widths[i] + 4 * int(np.count_nonzero(np.asarray(circ.types[i]) == 1)))
               for i in range(circ.depth))
    folds = sum(pairs * circ.widths[i + 1] for i in range(circ.depth))
    ms = sum(breakdown[k]["ms"] for k in ("row_sums", "copy_round", "copy_fold"))
    if not ms:
        return None
    achieved = (sums + folds) * IMAD_PER_FR_MUL / (ms / 1e3) / 1e12
    return {"kernels": "k_rowdot + k_copy_c + k_copy_fold", "ms_per_step": ms,
            "item_by_item_products": sums + folds, "achieved": achieved, "unit": "TIMAD/s",
            "frac_equivalent": achieved / peak, "peak": peak}


def step_equivalent(circ, ms_per_step: float, peak: float) -> dict:
    """The whole step (evaluation and proof) against the per-gate count of
    the method's work: 3 + 5 f products a (copy, gate) for a layer with a
    share f of mul gates (2 + 4 f for the copy rounds' sums, one for the
    fold, f for the evaluation), in Montgomery-product units of 264
    multiply-adds.  Libra's phases, the digests and the transcript are
    extra time at no extra count."""
    import numpy as np
    products = sum(circ.n_copies * (3 * circ.widths[i] + 5 * int(np.count_nonzero(np.asarray(circ.types[i]) == 1)))
                   for i in range(circ.depth))
    if not ms_per_step:
        return None
    achieved = products * IMAD_PER_FR_MUL / (ms_per_step / 1e3) / 1e12
    return {"per_step_products": products, "ms_per_step": ms_per_step, "achieved": achieved, "unit": "TIMAD/s",
            "frac_equivalent": achieved / peak, "peak": peak}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2404_10404_b300 as S
    import synth
    from paper_2404_10404_b300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    build()
    dev = torch.device("cuda", torch.cuda.current_device())
    circ = workload(args.workload, args.depth)
    gates = gates_of(circ)
    t0 = time.time()
    xb = synth.fr_bytes(synth.inputs_for(circ))
    log(f"[bench] {circ.name}: inputs drawn in {time.time() - t0:.1f} s")
    host = torch.frombuffer(bytearray(xb), dtype=torch.uint8).pin_memory()
    del xb
    inputs = host.to(dev)
    stream = torch.cuda.Stream(device=dev)
    # the copy round's launch shape per (layer width, pairs) class of this
    # circuit, tuned (cached on disk per GPU) before the eval handle exists
    autotune = None
    if not args.no_tune:
        from paper_2404_10404_b300 import tune
        t_tune = time.time()
        classes = tune.classes_of([circ])
        cached = tune.load() or {}
        table = tune.tune(classes, log=log)
        autotune = {"classes": len(classes), "from_cache": sum(c in cached for c in classes),
                    "seconds": round(time.time() - t_tune, 1),
                    "non_default": sum(table[c] != tune.DEFAULT_SHAPE for c in classes),
                    "first_round_us_default_vs_tuned": tune.gains(classes)}
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, inputs, stream)
    buf = ctypes.create_string_buffer(gc.proof_len)

    def step(src):
        ev.update(src, stream)
        return S.prove(gc, ev, None, stream, out=buf)

    proof = step(inputs)
    parity = None
    gold_path = os.path.join(ROOT, "tests", "golden", "oracle_full_size.json")
    if os.path.exists(gold_path):
        g = json.load(open(gold_path)).get(args.workload)
        if g and not args.depth:
            parity = hashlib.sha256(proof).hexdigest() == g["proof_sha256"]
    for _ in range(max(0, args.warmup - 1)):
        step(inputs)

    uuid = gpu_uuid(dev)
    imad = measure_imad_peak(S, stream, uuid)
    clocks = Clocks(uuid)
    time.sleep(0.5)
    # timed region: no per-kernel events, so the proofs replay their CUDA graphs;
    # the layer values (GiBs) are far larger than L2 and every step re-reads them
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = S.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark(True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(inputs)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark(False)
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = S.kernel_launches() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    value = aggregate_rate(world, args.steps, gates, ms / 1e3)
    # roofline of the dominant kernel: its launches timed with CUDA events on
    # the launching stream over further steps right after the timed region
    # (per-launch events need launch-by-launch issue instead of graph replay)
    S.profile_enable(1 << S.PROF_COPY_ROUND)
    for _ in range(min(args.steps, 10)):
        step(inputs)
    torch.cuda.synchronize(dev)
    prof_ms, prof_n, prof_work = S.profile_read(S.PROF_COPY_ROUND)
    S.profile_enable(0)

    # end to end through the public API: host inputs (pinned) in, proof out
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    for _ in range(args.steps):
        step(host)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - w0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e = {"value": aggregate_rate(world, args.steps, gates, e2e_s), "unit": UNIT, "h2d_bytes_per_step": host.numel(),
           "d2h_bytes_per_step": gc.proof_len}

    # per-kernel breakdown of one step (untimed pass)
    S.profile_enable(sum(1 << k for k in S.PROF_KINDS))
    step(inputs)
    torch.cuda.synchronize(dev)
    rounds = S.profile_launches(S.PROF_COPY_ROUND)
    per_round = [{"ms": round(m, 4), "fr_mults": w, "gmul_s": round(w / m / 1e6, 2) if m else None}
                 for m, w in rounds[:max(1, len(rounds) // max(1, circ.depth))]]
    breakdown = {}
    for k, name in S.PROF_KINDS.items():
        kms, kn, kw = S.profile_read(k)
        breakdown[name] = {"ms": round(kms, 4), "launches": kn, "fr_mults": kw}
    S.profile_enable(0)

    # (pair, gate) items of the timed copy rounds (the unit of the traffic figure)
    items = sum(circ.n_copies // 2 ** (k + 1) * circ.widths[i] for i in range(circ.depth)
                for k in range((circ.n_copies - 1).bit_length()))
    achieved = prof_work * IMAD_PER_FR_MUL / (prof_ms / 1e3) / 1e12 if prof_ms else None
    peak = imad["tops"]
    per_launch_items = items / max(1, len(rounds)) if rounds else None
    # the per-item traffic was captured on slot-shaped rounds: the other
    # workloads' rounds have other shapes, so they report none
    traffic = (DOMINANT_TRAFFIC_BYTES_PER_ITEM * per_launch_items
               if DOMINANT_TRAFFIC_BYTES_PER_ITEM and per_launch_items and args.workload == "slot" and not args.depth
               else None)
    roofline = {"bound": "alu", "kernel": "k_copy_c (copy-phase round: the mul entries' t^2 terms, the pairs' "
                                          "message terms and row-sum update)", "achieved": achieved,
                "peak": peak, "unit": "TIMAD/s", "frac": achieved / peak if achieved else None,
                "traffic": traffic,
                "peak_source": "measured in this run (mad.lo stream, integer pipe) of measured",
                "peak_measurement": imad,
                "frac_of_derived_peak": achieved / ALU_PEAK_TIMAD if achieved else None,
                "derived_peak": {"tops": ALU_PEAK_TIMAD, "how": "148 SMs x 64 IMAD/clk x 2032 MHz"},
                "work_counted": "per round, one Montgomery product (264 multiply-adds) and one full 512-bit "
                                "product (128) per mul entry and pair, and 4 (first round) or 8 Montgomery "
                                "products per pair",
                "per_launch_ms": prof_ms / prof_n if prof_n else None, "launches_timed": prof_n,
                "fr_mults_per_launch": prof_work / prof_n if prof_n else None,
                "items_per_launch": per_launch_items,
                "copy_phase": copy_phase_equivalent(circ, breakdown, peak),
                "step": step_equivalent(circ, ms / args.steps, peak)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": describe(circ), "n_copies": circ.n_copies, "width": circ.widths[0],
                       "depth": circ.depth, "gates_per_step": gates, "proof_bytes": gc.proof_len,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: the resident layer values are "
                             f"{gc.eval_bytes / 2**30:.1f} GiB, every step re-evaluates and re-reads them"},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "parity": {"proof_matches_oracle_sha256": parity},
            "breakdown_ms_per_step": breakdown, "copy_rounds_first_layer": per_round,
            "copy_round_autotune": autotune}
    del ev, gc, inputs
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    if world == 1 and not args.no_extra:
        # the rest of the metric: batched proofs/s and served p50/p99 against
        # the plain one-at-a-time path, on the batched workload's instances
        try:
            specs, pins = batched_setup(args.instances)
            bres, singles = batched_core(S, dev, stream, specs, pins, args.budget_gb)
            line["batched"] = bres
            line["served"] = served_core(S, dev, specs, pins, singles, args.extra_jobs, args.loads,
                                         args.budget_gb, args.slots)
            del pins
        except Exception as e:  # the headline stands without them
            line["batched_or_served_error"] = repr(e)
    if rank != 0:
        return
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# associative hash (Sec. 3.4.1, Algorithm 1) and pairwise-distinct check
# (Sec. 3.4.2, Algorithm 2) over validator indexes

ASSOC_METRIC = "validator indexes/s (associative hash of every slot + pairwise-distinct check of every epoch)"
ASSOC_UNIT = "indexes/s"
# multiply-adds per evaluation of F on a validator index (below 2^32), as the
# kernel forms it: the first cube and the second base exact in 64-bit
# integers (about 30 multiply-adds with the second base's square), the
# second base times R^2 by four fixed-multiplier rows (4 x 16 + 34), one
# Montgomery product for its cube, a R by two rows (2 x 16 + 34), and the
# last cube as a Montgomery square (72 + 136) and product
IMAD_PER_F = 30 + (4 * 16 + 34) + IMAD_PER_FR_MUL + (2 * 16 + 34) + (72 + 136) + IMAD_PER_FR_MUL
ASSOC_EPOCHS, ASSOC_EPOCH, ASSOC_SLOT, ASSOC_LOG_UNIVERSE = 64, 1 << 20, 1 << 15, 21
# DRAM read + write bytes per index of k_assoc_chunks (ncu capture of one
# launch over 2^23 indexes): the 32-byte value read once plus the chunk
# tables and partial sums
ASSOC_TRAFFIC_PER_INDEX = (268.816896e6 + 3.927552e6) / 2**23


def assoc_inputs(epochs: int):
    """Per epoch 2^20 distinct indexes below 2^21 in seeded order, and the
    same indexes sorted (the prover's claimed permutation A*)."""
    import numpy as np
    import synth
    a = np.empty((epochs * ASSOC_EPOCH, 4), dtype=np.uint64)
    s = np.empty_like(a)
    for e in range(epochs):
        idx = synth.validator_indexes(6 * 2**32 + e, ASSOC_EPOCH, ASSOC_LOG_UNIVERSE)
        a[e * ASSOC_EPOCH:(e + 1) * ASSOC_EPOCH] = idx
        s[e * ASSOC_EPOCH:(e + 1) * ASSOC_EPOCH] = idx[np.argsort(idx[:, 0], kind="stable")]
    return a, s


def assoc_describe(epochs: int) -> str:
    return (f"assoc: {epochs} epochs x 2^20 validator indexes (distinct, below 2^21, seeded order), "
            f"hash of every slot list of 2^15 (Algorithm 1), Algorithm 2 on every epoch against its sorted list "
            f"(the epoch's hash of the list as the sum of its slots' hashes)")


def time_assoc_oracle(a_bytes: bytes, s_bytes: bytes):
    from oracle import Oracle
    o = Oracle()
    t0 = time.perf_counter()
    for k in range(0, len(a_bytes), 32 * ASSOC_SLOT):
        o.assoc_hash(a_bytes[k:k + 32 * ASSOC_SLOT])
    o.pairwise_distinct_check(a_bytes, s_bytes)
    return time.perf_counter() - t0


def run_assoc_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    a, s = assoc_inputs(1)
    ab, sb = a.tobytes(), s.tobytes()
    for _ in range(args.warmup):
        time_assoc_oracle(ab[:32 * ASSOC_SLOT], sb[:32 * ASSOC_SLOT])
    total = 0.0
    for _ in range(args.steps):
        total += time_assoc_oracle(ab, sb)
    value = args.steps * ASSOC_EPOCH / total
    sample = "one epoch (2^20 indexes) per step: its 32 slot hashes and Algorithm 2 on it"
    line = {"impl": "reference", "metric": ASSOC_METRIC, "value": value, "unit": ASSOC_UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": assoc_describe(ASSOC_EPOCHS), "sample": sample},
            "cpu_baseline": {"value": value, "unit": ASSOC_UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": ASSOC_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_assoc(args):
    import numpy as np
    import torch

    import paper_2404_10404_b300 as S
    from oracle import Oracle
    from paper_2404_10404_b300.build import build

    torch.cuda.set_device(0)
    build()
    dev = torch.device("cuda", 0)
    epochs = args.epochs
    n = epochs * ASSOC_EPOCH
    t0 = time.time()
    a, s = assoc_inputs(epochs)
    log(f"[bench] assoc: {n} indexes drawn in {time.time() - t0:.1f} s")
    host_a = torch.from_numpy(a.view(np.uint8).reshape(-1)).pin_memory()
    host_s = torch.from_numpy(s.view(np.uint8).reshape(-1)).pin_memory()
    da, ds = host_a.to(dev), host_s.to(dev)
    slot_offs = np.arange(0, n + 1, ASSOC_SLOT, dtype=np.uint64)
    stream = torch.cuda.Stream(device=dev)
    st = stream.cuda_stream

    per = ASSOC_EPOCH // ASSOC_SLOT

    def step(xa, xs):
        # every slot's hash (Algorithm 1) and Algorithm 2 on every epoch, the
        # epoch's hash of A being the sum of its slots' hashes (AH is a sum)
        return S.assoc_epochs(xa, xs, slot_offs, per, stream=st)

    h, res, ha, hs = step(da, ds)
    # parity: every epoch's indexes are distinct (Algorithm 2 must accept
    # each); two slot hashes and the first epoch's hashes of A and of A*
    # against the oracle; each epoch's hash of A* equals its hash of A
    o = Oracle()
    ab = a.tobytes()
    ok = all(r == 1 for r in res)
    for g in (0, len(slot_offs) - 2):
        ok &= h[g] == o.assoc_hash(ab[32 * g * ASSOC_SLOT:32 * (g + 1) * ASSOC_SLOT])
    ok &= ha[0] == o.assoc_hash(ab[:32 * ASSOC_EPOCH])
    ok &= hs[0] == o.assoc_hash(s.tobytes()[:32 * ASSOC_EPOCH])
    ok &= all(ha[e] == hs[e] for e in range(epochs))
    for _ in range(max(0, args.warmup - 1)):
        step(da, ds)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)
    time.sleep(0.5)
    torch.cuda.synchronize(dev)
    launches0 = S.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark(True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(da, ds)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark(False)
    ms = ev0.elapsed_time(ev1)
    launches = S.kernel_launches() - launches0
    clk = clocks.stop()
    # the two summing kernels timed with events on their stream
    S.profile_enable((1 << S.PROF_ASSOC_HASH) | (1 << S.PROF_ASSOC_PAIR))
    for _ in range(min(args.steps, 5)):
        step(da, ds)
    torch.cuda.synchronize(dev)
    kern = {}
    for kind, name in ((S.PROF_ASSOC_HASH, "k_assoc_chunks (slot hashes)"),
                       (S.PROF_ASSOC_PAIR, "pairwise-distinct check (k_assoc_chunks on A*, k_order_chunks)")):
        kms, kn, kf = S.profile_read(kind)
        kern[name] = (kms, kn, kf)
    S.profile_enable(0)
    # the dominant kernel is k_assoc_chunks (two of the step's three
    # launches); the slot-hash scope times exactly one launch of it
    dom = "k_assoc_chunks (slot hashes)"
    kms, kn, kf = kern[dom]
    achieved = kf * IMAD_PER_F / (kms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": ALU_PEAK_TIMAD, "unit": "TIMAD/s",
                "frac": achieved / ALU_PEAK_TIMAD, "traffic": ASSOC_TRAFFIC_PER_INDEX * kf / kn,
                "traffic_source": "ncu dram bytes of one launch over 2^23 indexes, scaled to the launch's indexes",
                "per_launch_ms": kms / kn, "launches_timed": kn,
                "f_evaluations_per_launch": kf / kn, "imad_per_f": IMAD_PER_F,
                "peak_source": "derived: 148 SMs x 64 IMAD/clk x 2032 MHz",
                "kernels_ms_per_step": {k: round(v[0] / v[1], 4) for k, v in kern.items()}}
    # the prover's side (not in the step): sorting one epoch's list on the
    # device into A*, the input Algorithm 2 checks
    # (the unsorted copies are made before the timed region, on the sort's
    # stream)
    reps = 20
    with torch.cuda.stream(stream):
        ep = da[:32 * ASSOC_EPOCH].clone()
        for _ in range(3):
            S.sort_elements(ep.clone(), ep, ASSOC_EPOCH, stream=st)
        works = [da[:32 * ASSOC_EPOCH].clone() for _ in range(reps)]
    torch.cuda.synchronize(dev)
    srt0, srt1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    srt0.record(stream)
    passes = 0
    for work in works:
        _, passes = S.sort_elements(work, work, ASSOC_EPOCH, stream=st)
    srt1.record(stream)
    torch.cuda.synchronize(dev)
    sort_ms = srt0.elapsed_time(srt1) / reps
    sort_ok = bool(torch.equal(work, ds[:32 * ASSOC_EPOCH]))
    # bytes per element: the differing-bytes scan reads it once; every pass
    # reads it twice (histogram, scatter) and writes it once
    sort_bytes = ASSOC_EPOCH * 32 * (1 + 3 * passes)
    prover_sort = {"elements": ASSOC_EPOCH, "ms": sort_ms, "passes": passes,
                   "GB_s": sort_bytes / (sort_ms / 1e3) / 1e9, "equals_numpy_sort": sort_ok,
                   "note": "one epoch per call incl. the call's copies in and out of its buffers"}
    # end to end from pinned host memory: the calls copy the lists in
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    for _ in range(args.steps):
        step(host_a, host_s)
    e2e_s = time.perf_counter() - w0
    e2e = {"value": args.steps * n / e2e_s, "unit": ASSOC_UNIT, "h2d_bytes_per_step": 2 * 32 * n,
           "d2h_bytes_per_step": 32 * (len(slot_offs) - 1) + 68 * epochs}
    line = {"metric": ASSOC_METRIC, "value": args.steps * n / (ms / 1e3), "unit": ASSOC_UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": assoc_describe(epochs), "indexes_per_step": n,
                       "slots_per_step": len(slot_offs) - 1, "epochs_per_step": epochs,
                       "l2": f"inputs larger than L2: {n * 32 / 2**30:.2f} GiB of indexes and as much sorted"},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "parity": {"oracle_and_definition": bool(ok)}, "prover_sort": prover_sort}
    if not args.no_cpu_baseline:
        secs = time_assoc_oracle(ab[:32 * ASSOC_EPOCH], s.tobytes()[:32 * ASSOC_EPOCH])
        line["cpu_baseline"] = {"value": ASSOC_EPOCH / secs, "unit": ASSOC_UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one epoch (2^20 indexes): 32 slot hashes and Algorithm 2, {secs:.1f} s, "
                                          "single-threaded C oracle on the host"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched: many independent instances of uneven size

def batched_setup(n: int):
    """The first n instances of the batched workload and their inputs in
    pinned host memory."""
    import torch
    import synth
    t0 = time.time()
    specs = [synth.batched_instance(j) for j in range(n)]
    pins = [torch.frombuffer(bytearray(synth.fr_bytes(synth.inputs_for(c))), dtype=torch.uint8).pin_memory()
            for c in specs]
    log(f"[bench] batched: {n} instances drawn in {time.time() - t0:.1f} s")
    return specs, pins


def batched_core(S, dev, stream, specs, pins, budget_gb: float):
    """Proofs/s of the instances proved by sisu_gkr_prove_batch against one
    at a time, admitted in waves that fit the budget; the concurrency is
    tuned on the first wave.  Returns (result, the single-instance proofs)."""
    import torch

    from paper_2404_10404_b300 import tune
    budget = int(budget_gb * 2**30)
    # the copy round's launch shape per (layer width, pairs) class of these
    # instances, tuned once (cached on disk per GPU) before any handle exists
    t_tune = time.time()
    classes = tune.classes_of(specs)
    cached = tune.load() or {}
    table = tune.tune(classes, log=log, min_items=0)  # concurrent proofs: every class
    t_tune = time.time() - t_tune
    gains = tune.gains(classes)
    gcs_all = [S.Circuit.from_spec(c) for c in specs]
    foot = [S.server_footprint(g, True) for g in gcs_all]
    waves, cur, used = [], [], 0
    for k in range(len(specs)):
        if cur and used + foot[k] > budget:
            waves.append(cur)
            cur, used = [], 0
        cur.append(k)
        used += foot[k]
    if cur:
        waves.append(cur)
    gates = sum(gates_of(c) for c in specs)
    t_plain = t_batch = 0.0
    tuned, tune_log, singles = None, {}, [None] * len(specs)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for wave in waves:
        gcs = [gcs_all[k] for k in wave]
        evs = [S.Eval(gcs_all[k], pins[k], stream) for k in wave]
        # warm-up: workspace allocation, first proof, graph capture
        single = [S.prove(g, e, None, stream) for g, e in zip(gcs, evs)]
        for g, e in zip(gcs, evs):
            S.prove(g, e, None, stream)
        for k, p in zip(wave, single):
            singles[k] = p
        if tuned is None:  # the concurrency, on the first wave
            best = None
            for kc in (1, 2, 4, 8, 16, 32):
                S.prove_batch(gcs, evs, None, stream, kc)
                torch.cuda.synchronize(dev)
                ev0.record(stream)
                out = S.prove_batch(gcs, evs, None, stream, kc)
                ev1.record(stream)
                torch.cuda.synchronize(dev)
                ms = ev0.elapsed_time(ev1)
                tune_log[kc] = round(ms, 3)
                assert out == single, "batched proofs differ from single-instance proofs"
                if best is None or ms < best[1]:
                    best = (kc, ms)
            tuned = best[0]
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for g, e in zip(gcs, evs):
            S.prove(g, e, None, stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t_plain += ev0.elapsed_time(ev1) / 1e3
        ev0.record(stream)
        out = S.prove_batch(gcs, evs, None, stream, tuned)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t_batch += ev0.elapsed_time(ev1) / 1e3
        assert out == single, "batched proofs differ from single-instance proofs"
        del evs
        torch.cuda.synchronize(dev)
    n = len(specs)
    res = {"value": n / t_batch, "unit": "proofs/s", "ms": 1e3 * t_batch,
           "workload": f"batched: {n} instances, C = 2^U{{6..14}}, W = 2^U{{8..12}}, d = U{{8..24}}, "
                       f"60% mul, uniform wiring, seeds 4*2^32+j",
           "waves": [len(w) for w in waves], "budget_gb": budget_gb, "gates": gates,
           "timed": "proving only (statement digests, transcript, every layer's sumcheck, proof bytes to the "
                    "host); each instance evaluated once before",
           "plain_one_at_a_time": {"value": n / t_plain, "unit": "proofs/s", "seconds": t_plain},
           "speedup_vs_plain": t_plain / t_batch, "gates_per_s_batched": gates / t_batch,
           "autotune": {"concurrency": tuned, "ms_first_wave": tune_log,
                        "copy_round": {"classes": len(classes), "from_cache": sum(c in cached for c in classes),
                                       "seconds": round(t_tune, 1),
                                       "non_default": sum(table[c] != tune.DEFAULT_SHAPE for c in classes),
                                       "first_round_us_default_vs_tuned": gains,
                                       "how": "per (log2 W, log2 pairs) class: 27 launch shapes (128/256/384 "
                                              "threads x 3 splits (whole pairs a CTA or shares of a pair) x 3 "
                                              "share sizes) timed on the first copy round of a one-layer "
                                              "circuit of that shape, best of 3"}},
           "parity": "every batched proof equals the single-instance proof"}
    return res, singles


def run_batched(args):
    import torch

    import paper_2404_10404_b300 as S
    from paper_2404_10404_b300.build import build

    torch.cuda.set_device(0)
    build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    specs, pins = batched_setup(args.instances)
    res, _ = batched_core(S, dev, stream, specs, pins, args.budget_gb)
    line = {"metric": "batched proofs/sec", "value": res["value"], "unit": "proofs/s", "n_gpus": 1, "steps": 1,
            "warmup": 2, "ms_per_step": res["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": res["workload"], "waves": res["waves"], "budget_gb": args.budget_gb,
                       "gates": res["gates"], "timed": res["timed"]},
            **{k: res[k] for k in ("plain_one_at_a_time", "speedup_vs_plain", "gates_per_s_batched", "autotune",
                                   "parity")}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# served: Poisson arrivals into the continuous-batching server, against the
# plain path (evaluation + proof, one job at a time) on the same arrivals

def served_core(S, dev, specs, pins, singles, njobs: int, loads, budget_gb: float, slots: int, seed: int = 5):
    """Jobs pick one of the instances uniformly (sizes drawn as in the
    batched workload) with that instance's inputs; every proof is compared
    with the instance's single-instance proof."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    gcs = [S.Circuit.from_spec(c) for c in specs]
    alone = [hashlib.sha256(p).hexdigest() for p in singles]
    jobs = rng.integers(0, len(specs), size=njobs)
    budget = int(budget_gb * 2**30)
    stream = torch.cuda.Stream(device=dev)

    def summary(lat, done_at, arrivals, bad):
        ls = np.array(lat)
        span = max(done_at) - float(arrivals[0])
        return {"p50_ms": float(np.percentile(ls, 50)), "p99_ms": float(np.percentile(ls, 99)),
                "proofs_per_s": len(lat) / span, "mismatches": bad}

    def serve(arrivals):
        srv = S.Server(budget, slots)
        t0 = time.perf_counter()
        pending, lat, done_at, bad, k = {}, [0.0] * njobs, [0.0] * njobs, 0, 0
        finished = 0
        while finished < njobs:
            now = time.perf_counter() - t0
            while k < njobs and arrivals[k] <= now:
                pending[srv.submit(gcs[jobs[k]], pins[jobs[k]])] = k
                k += 1
            for t in list(pending):
                st, proof, ms = srv.poll(t)
                if st in (srv.QUEUED, srv.RUNNING):
                    continue
                jk = pending.pop(t)
                if st != srv.DONE or hashlib.sha256(proof).hexdigest() != alone[jobs[jk]]:
                    bad += 1
                lat[jk] = ms
                done_at[jk] = time.perf_counter() - t0
                finished += 1
            time.sleep(0.0002)
        srv.close()
        return summary(lat, done_at, arrivals, bad)

    def plain(arrivals):
        # the plain path one job at a time in arrival order: evaluation from
        # the pinned host inputs and the proof, a fresh eval handle per job
        t0 = time.perf_counter()
        lat, done_at, bad = [], [], 0
        for k in range(njobs):
            now = time.perf_counter() - t0
            if arrivals[k] > now:
                time.sleep(arrivals[k] - now)
            j = jobs[k]
            ev = S.Eval(gcs[j], pins[j], stream)
            p = S.prove(gcs[j], ev, None, stream)
            del ev
            t = time.perf_counter() - t0
            bad += hashlib.sha256(p).hexdigest() != alone[j]
            lat.append(1e3 * (t - arrivals[k]))
            done_at.append(t)
        return summary(lat, done_at, arrivals, bad)

    zeros = np.zeros(njobs)
    peak = serve(zeros)
    peak_plain = plain(zeros)
    rate = peak["proofs_per_s"]
    by_load = {}
    for load in loads:
        gaps = rng.exponential(1.0 / (load * rate), size=njobs)
        arrivals = np.cumsum(gaps) - gaps[0]
        by_load[str(load)] = {"offered_proofs_per_s": load * rate, "served": serve(arrivals),
                              "plain_one_at_a_time": plain(arrivals)}
    return {"value": rate, "unit": "proofs/s",
            "workload": f"served: {njobs} jobs, each one of the {len(specs)} batched instances drawn uniformly "
                        f"with its inputs (pinned host memory), Poisson arrivals at the offered loads, "
                        f"{budget_gb:g} GB budget, {slots} slots",
            "peak": peak, "plain_peak": peak_plain, "by_load": by_load,
            "plain": "evaluation + proof per job through the public API, one at a time in arrival order, "
                     "measured on the same arrival times",
            "parity": "every proof (served and plain) equals the instance's single-instance proof"}


def run_served(args):
    import torch

    import paper_2404_10404_b300 as S
    from paper_2404_10404_b300.build import build

    torch.cuda.set_device(0)
    build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    specs, pins = batched_setup(args.instances)
    singles = []
    for c, x in zip(specs, pins):
        g = S.Circuit.from_spec(c)
        singles.append(S.prove(g, S.Eval(g, x, stream), None, stream))
        torch.cuda.synchronize(dev)
    res = served_core(S, dev, specs, pins, singles, args.jobs, args.loads, args.budget_gb, args.slots)
    line = {"metric": "served p50/p99 proof latency and proofs/sec", "value": res["value"], "unit": "proofs/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * args.jobs / res["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": res["workload"], "loads": args.loads},
            **{k: res[k] for k in ("peak", "plain_peak", "by_load", "plain", "parity")}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["slot", "medium", "tiny", "batched", "served", "assoc"], default="slot")
    ap.add_argument("--jobs", type=int, default=2000, help="served: number of jobs")
    ap.add_argument("--extra-jobs", type=int, default=200,
                    help="served jobs in the default run's line (the full configuration: --workload served)")
    ap.add_argument("--slots", type=int, default=16, help="served: concurrent jobs")
    ap.add_argument("--loads", type=float, nargs="+", default=[0.25, 0.5, 0.9], help="served: offered loads")
    ap.add_argument("--instances", type=int, default=64, help="batched: number of instances")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="batched and served: device memory")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="leave the batched and served keys out of the line")
    ap.add_argument("--no-tune", action="store_true", help="keep the copy round's default launch shapes")
    ap.add_argument("--epochs", type=int, default=ASSOC_EPOCHS, help="assoc: epochs of 2^20 indexes per step")
    ap.add_argument("--depth", type=int, default=None,
                    help="keep only the workload's first layers (profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference" and args.workload == "assoc":
        run_assoc_reference(args)
    elif args.impl == "reference":
        if args.workload in ("batched", "served"):
            args.workload = "slot"
        run_reference(args)
    elif args.workload == "assoc":
        run_assoc(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
