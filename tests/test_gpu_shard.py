"""Copy-sharded proofs on the GPU (the distributed GKR of Sec. 3.2.1): N
virtual ranks share one GPU, each with its own evaluation of its copies
(b = j N + q), workspace and exchange buffers, the exchanges being device
copies (VirtualExchange).  Every sharded proof must equal the one-GPU proof
and the oracle's, byte for byte."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


CASES = {
    # several tiles in the local rounds, ragged layer widths inside
    "uniform": lambda: synth.uniform_circuit(21, 256, [64, 32, 200, 64], 60, name="gs-uniform"),
    "mixing": lambda: synth.mixing_circuit(22, 128, 64, 3, name="gs-mixing"),
    "wide": lambda: synth.uniform_circuit(23, 64, [512, 1024, 512], 50, name="gs-wide"),
    "accumulation": lambda: synth.accumulation_circuit(24, 64, [32, 64, 32], name="gs-acc"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_virtual_ranks_equal_one_gpu_and_oracle(S, oracle, name):
    from paper_2404_10404_b300.shard import prove_virtual
    spec = CASES[name]()
    xb = synth.fr_bytes(synth.inputs_for(spec))
    want = oracle.prove(spec, xb)
    gc = S.Circuit.from_spec(spec)
    assert S.prove(gc, S.Eval(gc, xb)) == want
    for world in (1, 2, 4, 8):
        assert prove_virtual(spec, xb, world) == want, world


def test_one_copy_a_rank(S, oracle):
    """world = n_copies: no local copy round, rank 0 runs them all."""
    from paper_2404_10404_b300.shard import prove_virtual
    spec = synth.uniform_circuit(25, 16, [32, 48, 32], 50, name="gs-one")
    xb = synth.fr_bytes(synth.inputs_for(spec))
    assert prove_virtual(spec, xb, 16) == oracle.prove(spec, xb)


def test_domain_and_repeated_proofs(S, oracle):
    from paper_2404_10404_b300.shard import GpuRank, VirtualExchange, prove_sharded
    import torch
    spec = synth.uniform_circuit(26, 64, [32, 32, 32], 60, name="gs-dom")
    xb = synth.fr_bytes(synth.inputs_for(spec))
    tr = S.Transcript(b"shard-domain")
    want = oracle.prove(spec, xb, b"shard-domain")
    stream = torch.cuda.current_stream()
    ranks = [GpuRank(spec, xb, q, 4, tr, stream) for q in range(4)]
    for _ in range(2):  # the shards are reusable: every proof starts from the roots
        assert prove_sharded(ranks, VirtualExchange(), stream) == want


def test_slot_shaped_layers(S):
    """Two layers of the slot workload's shape (1024-wide mixing layers,
    4096 copies) on 8 ranks, against the one-GPU proof."""
    from paper_2404_10404_b300.shard import prove_virtual
    spec = synth.mixing_circuit(3, 4096, 1024, 2, name="gs-slot2")
    xb = synth.fr_bytes(synth.inputs_for(spec))
    gc = S.Circuit.from_spec(spec)
    assert prove_virtual(spec, xb, 8) == S.prove(gc, S.Eval(gc, xb))


def test_refused_shapes(S):
    import torch
    narrow = synth.uniform_circuit(27, 8, [16, 16], 50, name="gs-narrow")
    gc = S.Circuit.from_spec(narrow, n_copies=4)
    ev = S.Eval(gc, synth.fr_bytes(synth.inputs_for(narrow))[:4 * 16 * 32])
    bufs = {n: torch.zeros(max(16, b), dtype=torch.uint8, device="cuda")
            for n, b in S.shard_buffer_sizes(ev, 2).items()}
    with pytest.raises(S.SisuError) as e:  # rows under 1 KiB
        S.Shard(ev, 0, 2, bufs)
    assert e.value.code == -1
    ok = synth.uniform_circuit(28, 6, [32, 32], 50, name="gs-pad")
    gp = S.Circuit.from_spec(ok)  # 6 copies: padded to 8
    ep = S.Eval(gp, synth.fr_bytes(synth.inputs_for(ok)))
    bufs = {n: torch.zeros(max(16, b), dtype=torch.uint8, device="cuda")
            for n, b in S.shard_buffer_sizes(ep, 2).items()}
    with pytest.raises(S.SisuError):  # padded copies
        S.Shard(ep, 0, 2, bufs)
    with pytest.raises(S.SisuError):  # world not a power of two
        S.shard_buffer_sizes(ep, 3)
    with pytest.raises(S.SisuError):  # rank beyond world
        S.Shard(ep, 2, 2, bufs)


def test_nccl_exchange_one_rank(S, oracle):
    """The torch.distributed exchange over NCCL on device buffers, in a
    one-rank process group (the only multi-process form one GPU allows):
    the sharded driver's all-gathers and broadcast run through NCCL and the
    proof equals the oracle's."""
    import socket

    import torch
    import torch.distributed as dist
    from paper_2404_10404_b300.shard import DistExchange, GpuRank, prove_sharded
    import os
    if dist.is_initialized():
        pytest.skip("a process group already exists")
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        spec = synth.uniform_circuit(29, 64, [64, 32, 64], 60, name="gs-nccl")
        xb = synth.fr_bytes(synth.inputs_for(spec))
        stream = torch.cuda.current_stream()
        rank = GpuRank(spec, xb, 0, 1, None, stream)
        with torch.cuda.stream(stream):
            proof = prove_sharded([rank], DistExchange(), stream)
        assert proof == oracle.prove(spec, xb)
    finally:
        dist.destroy_process_group()
