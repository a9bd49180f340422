"""Copy-sharded proving (the distributed GKR of Sec. 3.2.1) on CPU: the
library's sharding driver (paper_2404_10404_b300.shard.prove_sharded) runs
the oracle's restatement of one rank's steps (oracle/shard_ref.py), first
with every rank in one process (VirtualExchange on host tensors), then as
2 and 4 gloo processes (DistExchange).  Rank 0's proof must equal the
one-rank proofs of the C oracle and of the brute-force prover: copy bits
bound most significant first make the rank bits the last ones, so sharding
leaves the bytes unchanged."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import brute  # noqa: E402
from oracle.shard_ref import OracleRank  # noqa: E402
from paper_2404_10404_b300.shard import DistExchange, VirtualExchange, prove_sharded, rank_inputs  # noqa: E402


def _spec(kind: str):
    if kind == "uniform":
        return synth.uniform_circuit(11, 16, [32, 16, 32], 50, name="shard-uniform")
    if kind == "deep":
        return synth.uniform_circuit(12, 8, [32, 64, 8, 32], 70, name="shard-deep")
    return synth.mixing_circuit(13, 16, 32, 2, name="shard-mixing")


def _ranks(spec, x, world, domain=None):
    return [OracleRank(spec, synth.fr_ints(x[q::world]), q, world, domain) for q in range(world)]


@pytest.mark.parametrize("kind", ["uniform", "deep", "mixing"])
def test_virtual_ranks_equal_one_rank_proof(oracle, kind):
    spec = _spec(kind)
    x = synth.inputs_for(spec)
    want = oracle.prove(spec, synth.fr_bytes(x))
    for world in (1, 2, 4, spec.n_copies):  # world = n_copies: one copy a rank, no local round
        assert prove_sharded(_ranks(spec, x, world), VirtualExchange()) == want, world


def test_one_rank_restatement_equals_brute_force():
    spec = synth.uniform_circuit(14, 4, [32, 32], 60, name="shard-brute")
    x = synth.inputs_for(spec)
    assert prove_sharded(_ranks(spec, x, 1), VirtualExchange()) == brute.prove(spec, synth.fr_ints(x))
    assert prove_sharded(_ranks(spec, x, 4), VirtualExchange()) == brute.prove(spec, synth.fr_ints(x))


def test_domain_reaches_every_rank(oracle):
    spec = _spec("uniform")
    x = synth.inputs_for(spec)
    want = oracle.prove(spec, synth.fr_bytes(x), b"shard-domain")
    assert prove_sharded(_ranks(spec, x, 4, b"shard-domain"), VirtualExchange()) == want


def test_rank_inputs_take_every_world_th_copy():
    spec = _spec("uniform")
    xb = synth.fr_bytes(synth.inputs_for(spec))
    row = 32 * spec.widths[-1]
    for world in (2, 4):
        for q in range(world):
            part = rank_inputs(xb, spec.n_copies, spec.widths[-1], q, world)
            assert part == b"".join(xb[b * row:(b + 1) * row] for b in range(q, spec.n_copies, world))


def test_virtual_exchange_orders_by_rank():
    import torch
    sends = [torch.full((3,), q, dtype=torch.uint8) for q in range(4)]
    recvs = [torch.zeros(12, dtype=torch.uint8) for _ in range(4)]
    VirtualExchange().all_gather(sends, recvs)
    for r in recvs:
        assert r.tolist() == [0] * 3 + [1] * 3 + [2] * 3 + [3] * 3
    bufs = [torch.full((2,), q + 5, dtype=torch.uint8) for q in range(3)]
    VirtualExchange().broadcast0(bufs)
    assert all(b.tolist() == [5, 5] for b in bufs)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank: int, world: int, port: int, kind: str, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the exchange's own order: rank q's buffer lands at q * size
        ex = DistExchange()
        recv = torch.zeros(2 * world, dtype=torch.uint8)
        ex.all_gather([torch.full((2,), 10 + rank, dtype=torch.uint8)], [recv])
        st = torch.full((3,), 40 + rank, dtype=torch.uint8)
        ex.broadcast0([st])
        order_ok = recv.tolist() == [10 + q for q in range(world) for _ in range(2)] and st.tolist() == [40] * 3
        spec = _spec(kind)
        x = synth.inputs_for(spec)
        me = OracleRank(spec, synth.fr_ints(x[rank::world]), rank, world)
        proof = prove_sharded([me], ex)
        out.put((rank, order_ok, proof))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,kind", [(2, "uniform"), (4, "mixing")])
def test_gloo_ranks_prove_the_one_rank_proof(oracle, world, kind):
    spec = _spec(kind)
    want = oracle.prove(spec, synth.fr_bytes(synth.inputs_for(spec)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, world, port, kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(r[1] for r in res), "exchange order"
    assert res[0][2] == want
    assert all(r[2] is None for r in res[1:])
