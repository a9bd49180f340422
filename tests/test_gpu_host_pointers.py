"""Every entry point that hands a caller's buffer to its kernels refuses a
host address where it expects device memory, before anything is launched:
a kernel that read or wrote host memory through that address would fault
the GPU.  Each case passes a host array (ordinary or page-locked) as the
device buffer and checks the INVALID_ARG code, the message and that the
library launched no kernel."""
import ctypes
import time

import numpy as np
import pytest

import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu

INVALID_ARG = -1


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


@pytest.fixture(scope="module")
def hosts():
    """Host arrays at 256-byte aligned addresses (so that no alignment
    check answers first)."""
    import torch
    plain = np.zeros((1 << 16) + 256, dtype=np.uint8)
    addr = plain.ctypes.data
    addr += (-addr) % 256
    pinned = torch.zeros((1 << 16) + 256, dtype=torch.uint8).pin_memory()
    paddr = pinned.data_ptr()
    paddr += (-paddr) % 256
    return [("pageable", addr, plain), ("pinned", paddr, pinned)]


@pytest.fixture(scope="module")
def small(S):
    spec = synth.uniform_circuit(41, 4, [32, 32, 32], 50, name="host-pointer checks")
    xb = synth.fr_bytes(synth.inputs_for(spec))
    gc = S.Circuit.from_spec(spec)
    return spec, xb, gc, S.Eval(gc, xb)


def _refused(S, call):
    before = S.kernel_launches()
    with pytest.raises(S.SisuError) as e:
        call()
    assert S.kernel_launches() == before
    return e.value


def _rc_refused(S, rc):
    assert rc == INVALID_ARG
    assert b"device memory" in S._lib.sisu_last_error()


def test_eval_and_outputs(S, small, hosts):
    spec, xb, gc, ev = small
    for _, addr, _ in hosts:
        assert _refused(S, lambda: S.Eval(gc, addr)).code == INVALID_ARG
        assert _refused(S, lambda: ev.update(addr)).code == INVALID_ARG
        assert _refused(S, lambda: ev.outputs_to(addr)).code == INVALID_ARG
    # the handle still works, and device inputs are still taken
    ev.update(to_device(xb))
    assert S.prove(gc, ev) == S.prove(gc, S.Eval(gc, xb))


def test_field_batch_and_digest(S, hosts):
    dev = to_device(bytes(32 * 64))
    for _, addr, _ in hosts:
        for a, b, out in ((addr, dev.data_ptr(), dev.data_ptr()), (dev.data_ptr(), addr, dev.data_ptr()),
                          (dev.data_ptr(), dev.data_ptr(), addr)):
            assert _refused(S, lambda: S.fr_batch(0, a, b, out, 64)).code == INVALID_ARG
        assert _refused(S, lambda: S.statement_digest(addr, 1000)).code == INVALID_ARG
    # the binding refuses host arrays itself
    with pytest.raises(S.SisuError):
        S.statement_digest(np.zeros(64, dtype=np.uint8), 64)


def test_associative_hash_and_sort(S, hosts):
    dev = to_device(bytes(32 * 256))
    lib = S._lib
    for _, addr, _ in hosts:
        before = S.kernel_launches()
        out = ctypes.create_string_buffer(32)
        _rc_refused(S, lib.sisu_assoc_hash(addr, 256, None, 1, None, ctypes.cast(out, ctypes.c_void_p)))
        res = ctypes.c_int()
        _rc_refused(S, lib.sisu_pairwise_distinct_check(dev.data_ptr(), addr, 256, 1, None, ctypes.byref(res),
                                                        None, None))
        passes = ctypes.c_uint32()
        _rc_refused(S, lib.sisu_sort_elements(addr, 256, 1, None, dev.data_ptr(), ctypes.byref(passes)))
        _rc_refused(S, lib.sisu_sort_elements(dev.data_ptr(), 256, 1, None, addr, ctypes.byref(passes)))
        assert S.kernel_launches() == before


def test_server_submit(S, small, hosts):
    spec, xb, gc, _ = small
    srv = S.Server(budget_bytes=64 << 20, max_active=1)
    try:
        for _, addr, _ in hosts:
            assert _refused(S, lambda: srv.submit(gc, addr)).code == INVALID_ARG
        # a job with device inputs still runs
        dev_inputs = to_device(xb)
        t = srv.submit(gc, dev_inputs)
        deadline = time.time() + 60
        while True:
            st, proof, _ = srv.poll(t)
            if st not in (S.Server.QUEUED, S.Server.RUNNING) or time.time() > deadline:
                break
            time.sleep(0.01)
        assert st == S.Server.DONE
        assert proof == S.prove(gc, S.Eval(gc, xb))
    finally:
        srv.close()


def test_shard_exchange_buffers(S, small, hosts):
    spec, xb, gc, ev = small
    sizes = (ctypes.c_size_t * len(S.SHARD_BUFFERS))()
    assert S._lib.sisu_shard_buffer_sizes(ev.h, 2, sizes) == 0
    devs = {n: to_device(bytes(max(16, sizes[k]))) for k, n in enumerate(S.SHARD_BUFFERS)}
    for _, addr, _ in hosts:
        for bad in S.SHARD_BUFFERS:
            bufs = S._ShardBuffers(**{n: (addr if n == bad else devs[n].data_ptr()) for n in S.SHARD_BUFFERS})
            h = ctypes.c_void_p()
            before = S.kernel_launches()
            _rc_refused(S, S._lib.sisu_shard_create(ev.h, 0, 2, None, ctypes.byref(bufs), ctypes.byref(h)))
            assert not h.value
            assert S.kernel_launches() == before
