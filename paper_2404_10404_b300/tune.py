"""Autotuner of the copy round's launch shape.

A copy round of a layer whose next layer has 2^sn positions and 2^lh
pairs can launch with 128, 256 or 384-thread CTAs, with whole pairs a CTA
or shares of a pair's mul entries, and with a share's size set by the
entries it takes at least.  Which is fastest depends on (sn, lh): wide
rounds want every SM busy on whole pairs, small ones short chains.  For
each (sn, lh) class asked for, the tuner proves a one-layer circuit of
that shape (2^(lh+1) copies, 2^sn gates, 60% mul) under every candidate,
times its first copy round with CUDA events on the launching stream (best
of three), and keeps the fastest; the table is cached on disk per GPU
name and loaded into the library with ``sisu_tune_copy_round``, and
applies to the copy rounds of layered circuits.  Proof bytes do not depend
on the launch shape (every candidate's proof is compared with the
default's).
"""
from __future__ import annotations

import json
import os
import time

CTA_THREADS = (128, 256, 384)
DEFAULT_SHAPE = (256, 0, 0)  # the kernel's shape with no table entry
FORMS = (0, 1, 2)            # 0 whole pairs while pairs are at least the CTAs, 1 shares, 2 whole pairs
MIN_ITEMS = (0, 2, 4)        # 0: half a CTA's threads of entries a share; k: k entries a thread at least
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "copy_round.json")


def candidates():
    for bd in CTA_THREADS:
        for form in FORMS:
            for mi in MIN_ITEMS:
                yield bd, form, mi * bd


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def load(path: str = DEFAULT_CACHE) -> dict | None:
    """The cached table for this GPU ({(sn, lh): (bd, form, min_items)}),
    or None."""
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    entry = data.get(_gpu_name())
    if not entry:
        return None
    return {tuple(map(int, k.split(","))): tuple(v) for k, v in entry["table"].items()}


def apply(table: dict):
    import paper_2404_10404_b300 as S
    for (sn, lh), (bd, form, mi) in table.items():
        S.tune_copy_round(sn, lh, bd, form, mi)


def reset(classes):
    import paper_2404_10404_b300 as S
    for sn, lh in classes:
        S.tune_copy_round(sn, lh, 0)


def _time_first_round(S, gc, ev, stream, reps: int = 3) -> tuple[float, bytes]:
    import torch
    best, proof = None, None
    for _ in range(reps):
        S.profile_enable(1 << S.PROF_COPY_ROUND)
        proof = S.prove(gc, ev, None, stream)
        torch.cuda.synchronize()
        rounds = S.profile_launches(S.PROF_COPY_ROUND)
        S.profile_read(S.PROF_COPY_ROUND)
        S.profile_enable(0)
        ms = rounds[0][0]
        best = ms if best is None else min(best, ms)
    return best, proof


# For one proof at a time, classes with fewer (pair, gate) items a round
# keep the default shape: their rounds are latency-bound inside a proof,
# and shapes timed on a lone round there made the medium proof slower
# (18.5 -> 18.7 ms with every class tuned, 18.4-18.6 with this floor),
# while the throughput-bound classes gain inside the proof as in isolation
# (slot 92.8 -> 91.4-91.7 ms).  Concurrent proofs (the batched workload)
# tune every class: 118.4 proofs/s against 115.2 with the floor.
MIN_TUNED_ITEMS = 1 << 20


def tune(classes, path: str = DEFAULT_CACHE, log=None, min_items: int = MIN_TUNED_ITEMS) -> dict:
    """Tune every (sn, lh) class in ``classes`` with at least min_items
    (pair, gate) items a round (cached entries of this GPU are kept; the
    smaller classes keep the default shape and are not cached), apply the
    table and write the cache.  Returns the shapes of every class."""
    import torch

    import paper_2404_10404_b300 as S
    import synth
    cached = load(path) or {}
    table = dict(cached)
    small = {c: DEFAULT_SHAPE for c in classes if c not in cached and (1 << (c[0] + c[1])) < min_items}
    todo = sorted({c for c in classes if c not in table and c not in small})
    timings = {}
    stream = torch.cuda.current_stream()
    t0 = time.time()
    for sn, lh in todo:
        spec = synth.uniform_circuit(7 * (1 << 32) + 64 * sn + lh, 2 << lh, [1 << sn, 1 << sn], 60,
                                     name=f"tune_W{1 << sn}_C{2 << lh}")
        gc = S.Circuit.from_spec(spec)
        # random canonical inputs drawn on the device (below 2^253 < r): the
        # timing does not depend on the values
        x = torch.randint(0, 256, ((2 << lh) << sn, 32), dtype=torch.uint8, device="cuda")
        x[:, 31] &= 0x1F
        ev = S.Eval(gc, x.reshape(-1), stream)
        del x
        S.tune_copy_round(sn, lh, 0)
        ref_ms, ref = _time_first_round(S, gc, ev, stream)
        best = (DEFAULT_SHAPE, ref_ms)
        per = {"default": round(ref_ms * 1e3, 2)}
        for bd, form, mi in candidates():
            S.tune_copy_round(sn, lh, bd, form, mi)
            ms, proof = _time_first_round(S, gc, ev, stream)
            if proof != ref:
                raise RuntimeError(f"launch shape {(bd, form, mi)} changed the proof of {spec.name}")
            per[f"{bd},{form},{mi}"] = round(ms * 1e3, 2)
            if ms < best[1]:
                best = ((bd, form, mi), ms)
        table[(sn, lh)] = best[0]
        S.tune_copy_round(sn, lh, *best[0])
        timings[f"{sn},{lh}"] = per
        del ev, gc
        if log:
            log(f"[tune] W 2^{sn}, pairs 2^{lh}: {best[0]} {best[1] * 1e3:.1f} us (default {ref_ms * 1e3:.1f} us)")
    apply(table)
    reset(small)
    if todo:
        try:
            data = json.load(open(path))
        except (OSError, ValueError):
            data = {}
        prev = data.get(_gpu_name(), {}).get("timings_us", {})
        prev.update(timings)
        data[_gpu_name()] = {"table": {f"{k[0]},{k[1]}": list(v) for k, v in table.items()},
                             "timings_us": prev, "seconds": round(time.time() - t0, 1)}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass  # a read-only location: the table applies to this process only
    return {**table, **small}


def gains(classes, path: str = DEFAULT_CACHE):
    """Summed first-round microseconds over the classes: the default launch
    shape against the tuned one (from the cached timings)."""
    try:
        timings = json.load(open(path))[_gpu_name()]["timings_us"]
    except (OSError, ValueError, KeyError):
        return None
    d = t = 0.0
    for sn, lh in classes:
        per = timings.get(f"{sn},{lh}")
        if not per:
            continue
        d += per["default"]
        t += min(per.values())
    return [round(d, 1), round(t, 1)]


def classes_of(specs):
    """The (sn, lh) classes of every copy round of the circuits."""
    out = set()
    for c in specs:
        C = 1 << max(0, (c.n_copies - 1).bit_length())
        for w in c.widths[1:]:
            sn = max(0, (int(w) - 1).bit_length())
            h = C // 2
            while h >= 1:
                out.add((sn, h.bit_length() - 1))
                h //= 2
    return out
