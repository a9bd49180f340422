"""Helpers shared by the GPU tests: device buffers through torch, circuits
and inputs through the seeded generator."""
import hashlib
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def to_device(data: bytes):
    """A CUDA uint8 tensor holding ``data`` (16-byte aligned)."""
    torch = torch_cuda()
    t = torch.empty(max(16, len(data)), dtype=torch.uint8, device="cuda")
    if data:
        t[:len(data)].copy_(torch.frombuffer(bytearray(data), dtype=torch.uint8))
    return t


def from_device(t, n: int) -> bytes:
    return t[:n].cpu().numpy().tobytes()


def golden(name: str):
    path = os.path.join(GOLDEN, "oracle_full_size.json")
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get(name)


def sha(b: bytes) -> str:
    return hashlib.sha256(b).hexdigest()


def ints_of(b: bytes):
    return [int.from_bytes(b[i:i + 32], "little") for i in range(0, len(b), 32)]


def bytes_of(vals) -> bytes:
    return b"".join(int(v).to_bytes(32, "little") for v in vals)


def rand_fr(rng: np.random.Generator, n: int, P: int):
    return [int.from_bytes(rng.bytes(32), "little") % P for _ in range(n)]
