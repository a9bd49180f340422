"""Copy-sharded proving over ranks (the distributed GKR of Sec. 3.2.1).

Rank q of ``world`` (a power of two) holds copies b = j * world + q and runs
its share of every layer's copy rounds on its own GPU; the ranks exchange
four round sums per copy round (all-gather), one row per layer (to rank 0)
and, after rank 0 has finished the layer, the transcript state (broadcast).
Every step of the arithmetic runs in the library's kernels (``Shard``); this
module only sequences the calls and the exchanges, which it delegates to an
exchange object:

- ``VirtualExchange``: every rank in this process, on one GPU, each with its
  own evaluation, workspace and buffers; an exchange is a device copy on the
  calling stream.  Used to check, on one GPU, that the sharded proof is the
  one-GPU proof.
- ``DistExchange``: one rank per process over ``torch.distributed`` (NCCL for
  device buffers; gloo for host buffers), rank order = process-group rank.

The same driver (``prove_sharded``) runs any object with the ``Shard`` calls
and named buffers, so the exchange logic is exercised apart from the GPU.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


class VirtualExchange:
    """All ranks in one process: ``sends[q]`` and ``recvs[q]`` are rank q's
    tensors (same device); copies run on the current stream."""

    def all_gather(self, sends, recvs):
        import torch
        cat = torch.cat([s.reshape(-1) for s in sends])
        for r in recvs:
            r.reshape(-1)[:cat.numel()].copy_(cat)

    def broadcast0(self, bufs):
        for b in bufs[1:]:
            b.copy_(bufs[0])


class DistExchange:
    """One rank per process over the default process group."""

    def all_gather(self, sends, recvs):
        import torch.distributed as dist
        assert len(sends) == len(recvs) == 1, "one rank per process"
        dist.all_gather_into_tensor(recvs[0].reshape(-1), sends[0].reshape(-1))

    def broadcast0(self, bufs):
        import torch.distributed as dist
        assert len(bufs) == 1, "one rank per process"
        dist.broadcast(bufs[0], src=0)


def prove_sharded(ranks: Sequence, exchange, stream=None):
    """One proof by the ranks in ``ranks`` (this process's, in rank order),
    all in step.  Each rank offers the ``Shard`` calls (``roots``, ``begin``,
    ``layer_begin``, ``copy_round``, ``absorb``, ``row``, ``finish``,
    ``proof``), the attributes ``rank``, ``depth`` and ``local_rounds``, and
    ``buf(name)`` for its exchange buffers.  Rows are all-gathered (only
    rank 0 reads them).  Returns rank 0's proof bytes, or None when rank 0
    is not in this process."""
    def gather(name):
        exchange.all_gather([r.buf(name + "_send") for r in ranks], [r.buf(name + "_recv") for r in ranks])

    for r in ranks:
        r.roots(stream)
    gather("roots")
    for r in ranks:
        r.begin(stream)
    depth, kl = ranks[0].depth, ranks[0].local_rounds
    for i in range(depth):
        for r in ranks:
            r.layer_begin(i, stream)
        for k in range(kl):
            for r in ranks:
                r.copy_round(i, k, stream)
            gather("sums")
            for r in ranks:
                r.absorb(i, k, stream)
        for r in ranks:
            r.row(i, stream)
        gather("row")
        for r in ranks:
            if r.rank == 0:
                r.finish(i, stream)
        exchange.broadcast0([r.buf("state") for r in ranks])
    for r in ranks:
        if r.rank == 0:
            return r.proof(stream)
    return None


def rank_inputs(inputs: bytes, n_copies: int, width: int, rank: int, world: int) -> bytes:
    """The rows of copies b = j * world + rank, j = 0, 1, ... (canonical
    32-byte elements, ``width`` a row, copy-major)."""
    a = np.frombuffer(inputs, dtype=np.uint8).reshape(n_copies, width * 32)
    return a[rank::world].tobytes()


class GpuRank:
    """A rank on the current GPU: its evaluation, ``Shard`` and exchange
    buffers (device tensors)."""

    def __init__(self, spec, inputs, rank: int, world: int, transcript=None, stream=None):
        import torch

        import paper_2404_10404_b300 as S
        if spec.n_copies % world:
            raise S.SisuError(-1, "the copy count must be a multiple of the world size")
        local = spec.n_copies // world
        self.circ = S.Circuit.from_spec(spec, n_copies=local)
        self.ev = S.Eval(self.circ, rank_inputs(bytes(inputs), spec.n_copies, spec.widths[-1], rank, world), stream)
        sizes = S.shard_buffer_sizes(self.ev, world)
        self.bufs = {n: torch.zeros(max(16, b), dtype=torch.uint8, device="cuda") for n, b in sizes.items()}
        self.shard = S.Shard(self.ev, rank, world, self.bufs, transcript)
        self.rank, self.depth, self.local_rounds = rank, self.shard.depth, self.shard.local_rounds

    def buf(self, name):
        return self.bufs[name]

    def roots(self, stream=None):
        self.shard.roots(stream)

    def begin(self, stream=None):
        self.shard.begin(stream)

    def layer_begin(self, i, stream=None):
        self.shard.layer_begin(i, stream)

    def copy_round(self, i, k, stream=None):
        self.shard.copy_round(i, k, stream)

    def absorb(self, i, k, stream=None):
        self.shard.absorb(i, k, stream)

    def row(self, i, stream=None):
        self.shard.row(i, stream)

    def finish(self, i, stream=None):
        self.shard.finish(i, stream)

    def proof(self, stream=None):
        return self.shard.proof(stream)


def prove_virtual(spec, inputs, world: int, transcript=None, stream=None) -> bytes:
    """The proof of ``spec`` on ``inputs`` (host bytes, all copies) by
    ``world`` ranks sharing the current GPU."""
    import torch
    stream = stream or torch.cuda.current_stream()
    ranks = [GpuRank(spec, inputs, q, world, transcript, stream) for q in range(world)]
    with torch.cuda.stream(stream):
        return prove_sharded(ranks, VirtualExchange(), stream)
