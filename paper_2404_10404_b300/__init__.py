"""Python binding of libsisu.so, the B300-native data-parallel GKR prover.

Argument marshalling only: every step of evaluation and proving runs in the
library's CUDA kernels behind the C ABI declared in ``include/sisu.h``.
The library is loaded on first use.  Importing this package does not import
torch; device buffers are passed as
objects with ``data_ptr()`` (torch CUDA tensors) or as raw integer pointers.
If the library has not been built the import fails with an error that says
how to build it: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsisu.so")

OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "INDEX_OOB", -3: "NOT_CANONICAL", -4: "OOM", -5: "CUDA",
    -6: "TIMEOUT", -7: "REJECT", -8: "ZERO_INVERSE", -9: "TOO_LARGE", -10: "BUFFER",
}
FR_ADD, FR_SUB, FR_MUL, FR_INV, FR_EQ1 = 0, 1, 2, 3, 4
ENTRY_POINTS = [
    "sisu_circuit_create", "sisu_circuit_create_host", "sisu_circuit_create_acc", "sisu_circuit_create_acc_host",
    "sisu_circuit_create_general", "sisu_circuit_create_general_host",
    "sisu_circuit_destroy", "sisu_circuit_info", "sisu_circuit_eval",
    "sisu_eval_update", "sisu_eval_outputs", "sisu_eval_layer", "sisu_eval_destroy",
    "sisu_transcript_create", "sisu_transcript_destroy", "sisu_gkr_prove", "sisu_gkr_prove_into",
    "sisu_gkr_verify", "sisu_fr_batch", "sisu_statement_digest", "sisu_microbench",
    "sisu_kernel_launches", "sisu_free", "sisu_last_error", "sisu_version",
    "sisu_profile_enable", "sisu_profile_read", "sisu_profile_launches", "sisu_statement_digest_noalloc",
    "sisu_gkr_prove_batch", "sisu_server_create", "sisu_server_submit", "sisu_server_poll",
    "sisu_server_pending", "sisu_server_pause", "sisu_server_destroy", "sisu_job_footprint",
    "sisu_shard_buffer_sizes", "sisu_shard_create", "sisu_shard_destroy", "sisu_shard_info", "sisu_shard_roots",
    "sisu_shard_begin", "sisu_shard_layer_begin", "sisu_shard_copy_round", "sisu_shard_absorb", "sisu_shard_row",
    "sisu_shard_finish", "sisu_shard_proof", "sisu_tune_copy_round",
    "sisu_assoc_hash", "sisu_assoc_hash_segments", "sisu_pairwise_distinct_check",
    "sisu_pairwise_distinct_check_segments", "sisu_sort_elements", "sisu_assoc_epochs",
]
PROF_COPY_ROUND, PROF_COPY_FOLD, PROF_EVAL, PROF_GATE_ROUND, PROF_DIGEST = 0, 1, 2, 3, 4
PROF_LAYER_INIT, PROF_PHASE_INIT, PROF_TRANSCRIPT, PROF_INPUTS = 5, 6, 7, 8
PROF_ASSOC_HASH, PROF_ASSOC_PAIR, PROF_ROW_SUMS = 9, 10, 11
PROF_KINDS = {0: "copy_round", 1: "copy_fold", 2: "eval_layer", 3: "gate_round", 4: "digest",
              5: "layer_init", 6: "phase_init", 7: "transcript", 8: "inputs", 11: "row_sums"}


class SisuError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Layer(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("type", ctypes.POINTER(ctypes.c_uint8)),
                ("in1", ctypes.POINTER(ctypes.c_uint32)), ("in2", ctypes.POINTER(ctypes.c_uint32))]


class _GeneralLayer(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("type", ctypes.POINTER(ctypes.c_uint8)),
                ("in1", ctypes.POINTER(ctypes.c_uint32)), ("src", ctypes.POINTER(ctypes.c_uint32)),
                ("in2", ctypes.POINTER(ctypes.c_uint32))]


class _AccLayer(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("n_entries", ctypes.c_uint32),
                ("out", ctypes.POINTER(ctypes.c_uint32)), ("type", ctypes.POINTER(ctypes.c_uint8)),
                ("in1", ctypes.POINTER(ctypes.c_uint32)), ("in2", ctypes.POINTER(ctypes.c_uint32))]


SHARD_BUFFERS = ("roots_send", "roots_recv", "sums_send", "sums_recv", "row_send", "row_recv", "state")


class _ShardBuffers(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in SHARD_BUFFERS]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2404_10404_b300.build` (needs nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, u32, u8p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "sisu_circuit_create": ([ctypes.POINTER(_Layer), u32, u32, u32, pp], ctypes.c_int),
        "sisu_circuit_create_host": ([ctypes.POINTER(_Layer), u32, u32, u32, pp], ctypes.c_int),
        "sisu_circuit_create_acc": ([ctypes.POINTER(_AccLayer), u32, u32, u32, pp], ctypes.c_int),
        "sisu_circuit_create_acc_host": ([ctypes.POINTER(_AccLayer), u32, u32, u32, pp], ctypes.c_int),
        "sisu_circuit_create_general": ([ctypes.POINTER(_GeneralLayer), u32, u32, u32, pp], ctypes.c_int),
        "sisu_circuit_create_general_host": ([ctypes.POINTER(_GeneralLayer), u32, u32, u32, pp], ctypes.c_int),
        "sisu_circuit_destroy": ([vp], None),
        "sisu_circuit_info": ([vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32),
                               ctypes.POINTER(sz), ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_circuit_eval": ([vp, u8p, ctypes.c_int, vp, pp], ctypes.c_int),
        "sisu_eval_update": ([vp, u8p, ctypes.c_int, vp], ctypes.c_int),
        "sisu_eval_outputs": ([vp, u8p, sz, ctypes.c_int, vp], ctypes.c_int),
        "sisu_eval_layer": ([vp, u32, u8p, sz, vp], ctypes.c_int),
        "sisu_eval_destroy": ([vp], None),
        "sisu_transcript_create": ([u8p, sz, pp], ctypes.c_int),
        "sisu_transcript_destroy": ([vp], None),
        "sisu_gkr_prove": ([vp, vp, vp, vp, pp, ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_gkr_prove_into": ([vp, vp, vp, vp, u8p, sz, ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_gkr_verify": ([vp, u8p, u8p, u8p, sz, u8p, sz], ctypes.c_int),
        "sisu_server_create": ([sz, u32, vp, sz, pp], ctypes.c_int),
        "sisu_server_submit": ([vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "sisu_server_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), vp, sz, ctypes.POINTER(sz),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "sisu_server_pending": ([vp, ctypes.POINTER(u32), ctypes.POINTER(u32)], ctypes.c_int),
        "sisu_server_pause": ([vp, ctypes.c_int], ctypes.c_int),
        "sisu_job_footprint": ([vp, ctypes.c_int, ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_server_destroy": ([vp], None),
        "sisu_gkr_prove_batch": ([ctypes.POINTER(vp), ctypes.POINTER(vp), u32, vp, vp, u32, ctypes.POINTER(vp),
                                  ctypes.POINTER(sz), ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_shard_buffer_sizes": ([vp, u32, ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_shard_create": ([vp, u32, u32, vp, ctypes.POINTER(_ShardBuffers), pp], ctypes.c_int),
        "sisu_shard_destroy": ([vp], None),
        "sisu_shard_info": ([vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_shard_roots": ([vp, vp], ctypes.c_int),
        "sisu_shard_begin": ([vp, vp], ctypes.c_int),
        "sisu_shard_layer_begin": ([vp, u32, vp], ctypes.c_int),
        "sisu_shard_copy_round": ([vp, u32, u32, vp], ctypes.c_int),
        "sisu_shard_absorb": ([vp, u32, u32, vp], ctypes.c_int),
        "sisu_shard_row": ([vp, u32, vp], ctypes.c_int),
        "sisu_shard_finish": ([vp, u32, vp], ctypes.c_int),
        "sisu_shard_proof": ([vp, vp, vp, sz, ctypes.POINTER(sz)], ctypes.c_int),
        "sisu_tune_copy_round": ([u32, u32, u32, u32, u32], ctypes.c_int),
        "sisu_fr_batch": ([ctypes.c_int, vp, vp, vp, sz, vp], ctypes.c_int),
        "sisu_statement_digest": ([vp, sz, u8p, vp], ctypes.c_int),
        "sisu_statement_digest_noalloc": ([vp, sz, vp, vp], ctypes.c_int),
        "sisu_microbench": ([ctypes.c_int, u32, u32, u32, vp, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "sisu_assoc_hash": ([vp, ctypes.c_uint64, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "sisu_assoc_hash_segments": ([vp, ctypes.POINTER(ctypes.c_uint64), u32, vp, ctypes.c_int, vp, vp],
                                     ctypes.c_int),
        "sisu_pairwise_distinct_check": ([vp, vp, ctypes.c_uint64, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                                          vp, vp], ctypes.c_int),
        "sisu_pairwise_distinct_check_segments": ([vp, vp, ctypes.POINTER(ctypes.c_uint64), u32, ctypes.c_int, vp,
                                                   ctypes.POINTER(ctypes.c_int), vp, vp], ctypes.c_int),
        "sisu_sort_elements": ([vp, ctypes.c_uint64, ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_uint32)],
                               ctypes.c_int),
        "sisu_assoc_epochs": ([vp, vp, ctypes.POINTER(ctypes.c_uint64), u32, u32, ctypes.c_int, vp, vp,
                               ctypes.POINTER(ctypes.c_int), vp, vp], ctypes.c_int),
        "sisu_kernel_launches": ([], ctypes.c_uint64),
        "sisu_free": ([vp], None),
        "sisu_last_error": ([], ctypes.c_char_p),
        "sisu_version": ([], ctypes.c_char_p),
        "sisu_profile_enable": ([u32], ctypes.c_int),
        "sisu_profile_read": ([u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "sisu_profile_launches": ([u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), sz,
                                   ctypes.POINTER(sz)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib_handle = None


def _lib_get():
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = _load()
    return _lib_handle


class _LazyLib:
    def __getattr__(self, name):
        return getattr(_lib_get(), name)


_lib = _LazyLib()


def _check(rc: int):
    if rc != OK:
        raise SisuError(rc, _lib.sisu_last_error().decode(errors="replace"))


def _ptr(buf):
    """(pointer, on_device, keepalive) for bytes, numpy arrays, torch tensors or ints."""
    if buf is None:
        return None, 0, None
    if isinstance(buf, int):
        return buf, 1, None
    if hasattr(buf, "data_ptr") and hasattr(buf, "is_cuda"):
        return buf.data_ptr(), int(bool(buf.is_cuda)), buf
    if isinstance(buf, (bytes, bytearray)):
        arr = np.frombuffer(bytes(buf), dtype=np.uint8)
        return arr.ctypes.data, 0, arr
    arr = np.ascontiguousarray(buf)
    return arr.ctypes.data, 0, arr


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", stream)


def library_path() -> str:
    return LIB_PATH


def version() -> str:
    return _lib.sisu_version().decode()


def kernel_launches() -> int:
    return int(_lib.sisu_kernel_launches())


class Circuit:
    """A layered circuit on the device (``sisu_circuit_create``).

    ``widths[i]`` gates in layer i (0 = outputs, d = inputs); ``types``,
    ``in1``, ``in2`` per gate layer; ``n_copies`` identical copies.  With
    ``outs`` (accumulation gates, ``sisu_circuit_create_acc``) the three
    arrays of a layer list its entries and ``outs[i]`` the gate of each.
    """

    def __init__(self, widths, types, in1, in2, n_copies: int, host_only: bool = False, outs=None, src=None):
        d = len(widths) - 1
        self._keep = []
        u32p, u8p = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint8)
        if src is not None:  # general circuit (Sec. 2.7): second inputs from layer src
            layers = (_GeneralLayer * d)()
            for i in range(d):
                t = np.ascontiguousarray(types[i], dtype=np.uint8)
                a = np.ascontiguousarray(in1[i], dtype=np.uint32)
                r = np.ascontiguousarray(src[i] if src[i] is not None else np.full(len(a), i + 1), dtype=np.uint32)
                b = np.ascontiguousarray(in2[i], dtype=np.uint32)
                if not (len(t) == len(a) == len(r) == len(b) == int(widths[i])):
                    raise SisuError(-1, f"layer {i}: wiring arrays must have {widths[i]} entries")
                self._keep += [t, a, r, b]
                layers[i] = _GeneralLayer(int(widths[i]), t.ctypes.data_as(u8p), a.ctypes.data_as(u32p),
                                          r.ctypes.data_as(u32p), b.ctypes.data_as(u32p))
            h = ctypes.c_void_p()
            create = _lib.sisu_circuit_create_general_host if host_only else _lib.sisu_circuit_create_general
            _check(create(layers, d, int(widths[d]), int(n_copies), ctypes.byref(h)))
            self._finish(h, widths, n_copies)
            return
        layers = (_Layer * d)() if outs is None else (_AccLayer * d)()
        for i in range(d):
            t = np.ascontiguousarray(types[i], dtype=np.uint8)
            a = np.ascontiguousarray(in1[i], dtype=np.uint32)
            b = np.ascontiguousarray(in2[i], dtype=np.uint32)
            if outs is None:
                if not (len(t) == len(a) == len(b) == int(widths[i])):
                    raise SisuError(-1, f"layer {i}: wiring arrays must have {widths[i]} entries")
                self._keep += [t, a, b]
                layers[i] = _Layer(int(widths[i]), t.ctypes.data_as(u8p), a.ctypes.data_as(u32p),
                                   b.ctypes.data_as(u32p))
            else:
                o = (np.arange(int(widths[i]), dtype=np.uint32) if outs[i] is None
                     else np.ascontiguousarray(outs[i], dtype=np.uint32))
                if not (len(t) == len(a) == len(b) == len(o)):
                    raise SisuError(-1, f"layer {i}: entry arrays of different lengths")
                self._keep += [t, a, b, o]
                layers[i] = _AccLayer(int(widths[i]), len(o), o.ctypes.data_as(u32p), t.ctypes.data_as(u8p),
                                      a.ctypes.data_as(u32p), b.ctypes.data_as(u32p))
        h = ctypes.c_void_p()
        if outs is None:
            create = _lib.sisu_circuit_create_host if host_only else _lib.sisu_circuit_create
        else:
            create = _lib.sisu_circuit_create_acc_host if host_only else _lib.sisu_circuit_create_acc
        _check(create(layers, d, int(widths[d]), int(n_copies), ctypes.byref(h)))
        self._finish(h, widths, n_copies)

    def _finish(self, h, widths, n_copies):
        d = len(widths) - 1
        self._keep = None
        self.h = h
        self.widths = [int(w) for w in widths]
        self.n_copies = int(n_copies)
        dep, lc = ctypes.c_uint32(), ctypes.c_uint32()
        lw = (ctypes.c_uint32 * (d + 1))()
        pl, eb = ctypes.c_size_t(), ctypes.c_size_t()
        _check(_lib.sisu_circuit_info(h, ctypes.byref(dep), ctypes.byref(lc), lw, ctypes.byref(pl),
                                      ctypes.byref(eb)))
        self.depth = int(dep.value)
        self.log_copies = int(lc.value)
        self.log_widths = list(lw)
        self.proof_len = int(pl.value)
        self.eval_bytes = int(eb.value)

    @classmethod
    def from_spec(cls, spec, host_only: bool = False, n_copies: int | None = None):
        """From any object with widths, types, in1, in2 and n_copies (and
        outs, for accumulation gates); ``n_copies`` overrides the copy count
        (a rank's share of a copy-sharded proof)."""
        outs = getattr(spec, "outs", None)
        if outs is not None and all(o is None for o in outs):
            outs = None
        return cls(spec.widths, spec.types, spec.in1, spec.in2, spec.n_copies if n_copies is None else n_copies,
                   host_only=host_only, outs=outs, src=getattr(spec, "src", None))

    def __del__(self):
        if getattr(self, "h", None):
            _lib.sisu_circuit_destroy(self.h)
            self.h = None


class Eval:
    """Resident values of every layer (``sisu_circuit_eval``)."""

    def __init__(self, circ: Circuit, inputs, stream=None):
        p, on_dev, keep = _ptr(inputs)
        h = ctypes.c_void_p()
        _check(_lib.sisu_circuit_eval(circ.h, p, on_dev, _stream(stream), ctypes.byref(h)))
        del keep
        self.h = h
        self.circ = circ

    def update(self, inputs, stream=None):
        p, on_dev, keep = _ptr(inputs)
        _check(_lib.sisu_eval_update(self.h, p, on_dev, _stream(stream)))
        del keep

    def outputs(self, stream=None) -> bytes:
        n = 32 * self.circ.n_copies * self.circ.widths[0]
        buf = ctypes.create_string_buffer(n)
        _check(_lib.sisu_eval_outputs(self.h, ctypes.cast(buf, ctypes.c_void_p), n, 0, _stream(stream)))
        return buf.raw

    def outputs_to(self, dev_buf, stream=None):
        p, _, keep = _ptr(dev_buf)
        n = 32 * self.circ.n_copies * self.circ.widths[0]
        _check(_lib.sisu_eval_outputs(self.h, p, n, 1, _stream(stream)))

    def layer(self, l: int, stream=None) -> bytes:
        n = 32 << (self.circ.log_copies + self.circ.log_widths[l])
        buf = ctypes.create_string_buffer(n)
        _check(_lib.sisu_eval_layer(self.h, l, ctypes.cast(buf, ctypes.c_void_p), n, _stream(stream)))
        return buf.raw

    def __del__(self):
        if getattr(self, "h", None):
            _lib.sisu_eval_destroy(self.h)
            self.h = None


def shard_buffer_sizes(ev: Eval, world: int) -> dict:
    """Bytes of each exchange buffer of a rank (``sisu_shard_buffer_sizes``)."""
    sizes = (ctypes.c_size_t * len(SHARD_BUFFERS))()
    _check(_lib.sisu_shard_buffer_sizes(ev.h, int(world), sizes))
    return dict(zip(SHARD_BUFFERS, (int(x) for x in sizes)))


class Shard:
    """One rank's part of a copy-sharded proof (``sisu_shard_*``).

    ``buffers`` maps the names of SHARD_BUFFERS to 16-byte aligned device
    buffers (torch tensors or pointers) of the sizes shard_buffer_sizes
    gives; they must outlive the shard."""

    def __init__(self, ev: Eval, rank: int, world: int, buffers: dict, transcript=None):
        keep = []
        ptrs = {}
        for n in SHARD_BUFFERS:
            p, _, k = _ptr(buffers.get(n))
            ptrs[n] = p
            keep.append(k)
        b = _ShardBuffers(**ptrs)
        h = ctypes.c_void_p()
        _check(_lib.sisu_shard_create(ev.h, int(rank), int(world), transcript.h if transcript else None,
                                      ctypes.byref(b), ctypes.byref(h)))
        self.h = h
        self._keep = (ev, buffers, transcript)
        lr, cb, pl = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_size_t()
        _check(_lib.sisu_shard_info(h, ctypes.byref(lr), ctypes.byref(cb), ctypes.byref(pl)))
        self.rank, self.world = int(rank), int(world)
        self.local_rounds, self.copy_bits, self.proof_len = int(lr.value), int(cb.value), int(pl.value)
        self.depth = ev.circ.depth

    def roots(self, stream=None):
        _check(_lib.sisu_shard_roots(self.h, _stream(stream)))

    def begin(self, stream=None):
        _check(_lib.sisu_shard_begin(self.h, _stream(stream)))

    def layer_begin(self, layer: int, stream=None):
        _check(_lib.sisu_shard_layer_begin(self.h, layer, _stream(stream)))

    def copy_round(self, layer: int, k: int, stream=None):
        _check(_lib.sisu_shard_copy_round(self.h, layer, k, _stream(stream)))

    def absorb(self, layer: int, k: int, stream=None):
        _check(_lib.sisu_shard_absorb(self.h, layer, k, _stream(stream)))

    def row(self, layer: int, stream=None):
        _check(_lib.sisu_shard_row(self.h, layer, _stream(stream)))

    def finish(self, layer: int, stream=None):
        _check(_lib.sisu_shard_finish(self.h, layer, _stream(stream)))

    def proof(self, stream=None) -> bytes:
        buf = ctypes.create_string_buffer(self.proof_len)
        n = ctypes.c_size_t()
        _check(_lib.sisu_shard_proof(self.h, _stream(stream), ctypes.cast(buf, ctypes.c_void_p), self.proof_len,
                                     ctypes.byref(n)))
        return buf.raw[:n.value]

    def __del__(self):
        if getattr(self, "h", None):
            _lib.sisu_shard_destroy(self.h)
            self.h = None


class Transcript:
    """Fiat-Shamir domain (``sisu_transcript_create``); None = default."""

    def __init__(self, domain: bytes | None = None):
        h = ctypes.c_void_p()
        dom = bytes(domain) if domain else None
        buf = ctypes.create_string_buffer(dom) if dom else None
        _check(_lib.sisu_transcript_create(ctypes.cast(buf, ctypes.c_void_p) if buf else None,
                                           len(dom) if dom else 0, ctypes.byref(h)))
        self.h = h
        self.domain = dom

    def __del__(self):
        if getattr(self, "h", None):
            _lib.sisu_transcript_destroy(self.h)
            self.h = None


def prove(circ: Circuit, ev: Eval, transcript: Transcript | None = None, stream=None, out=None) -> bytes:
    """Proof bytes (``sisu_gkr_prove_into``); ``out`` may be a reusable
    ctypes buffer of at least ``circ.proof_len`` bytes."""
    n = circ.proof_len
    buf = out if out is not None else ctypes.create_string_buffer(n)
    ln = ctypes.c_size_t()
    _check(_lib.sisu_gkr_prove_into(circ.h, ev.h, transcript.h if transcript else None, _stream(stream),
                                    ctypes.cast(buf, ctypes.c_void_p), n, ctypes.byref(ln)))
    return buf.raw[:ln.value]


def prove_alloc(circ: Circuit, ev: Eval, transcript: Transcript | None = None, stream=None) -> bytes:
    """Proof bytes through ``sisu_gkr_prove`` (library-allocated buffer)."""
    p = ctypes.c_void_p()
    ln = ctypes.c_size_t()
    _check(_lib.sisu_gkr_prove(circ.h, ev.h, transcript.h if transcript else None, _stream(stream),
                               ctypes.byref(p), ctypes.byref(ln)))
    try:
        return ctypes.string_at(p, ln.value)
    finally:
        _lib.sisu_free(p)


def prove_batch(circs, evals, transcript: Transcript | None = None, stream=None, concurrency: int = 0):
    """Proofs of independent instances on concurrent streams (``sisu_gkr_prove_batch``)."""
    n = len(circs)
    if n != len(evals):
        raise SisuError(-1, "circuits and evals differ in number")
    bufs = [ctypes.create_string_buffer(c.proof_len) for c in circs]
    ch = (ctypes.c_void_p * n)(*[c.h.value for c in circs])
    eh = (ctypes.c_void_p * n)(*[e.h.value for e in evals])
    ph = (ctypes.c_void_p * n)(*[ctypes.cast(b, ctypes.c_void_p).value for b in bufs])
    caps = (ctypes.c_size_t * n)(*[c.proof_len for c in circs])
    lens = (ctypes.c_size_t * n)()
    _check(_lib.sisu_gkr_prove_batch(ch, eh, n, transcript.h if transcript else None, _stream(stream),
                                     concurrency, ph, caps, lens))
    return [bufs[i].raw[:lens[i]] for i in range(n)]


class Server:
    """Continuous-batching proof server (``sisu_server_*``)."""

    QUEUED, RUNNING, DONE = 0, 1, 2

    def __init__(self, budget_bytes: int, max_active: int = 8, domain: bytes | None = None):
        h = ctypes.c_void_p()
        dom = bytes(domain) if domain else None
        buf = ctypes.create_string_buffer(dom) if dom else None
        _check(_lib.sisu_server_create(budget_bytes, max_active, ctypes.cast(buf, ctypes.c_void_p) if buf else None,
                                       len(dom) if dom else 0, ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, circ: Circuit, inputs) -> int:
        """Queue a job; ``inputs`` must stay alive and unchanged until it is done."""
        p, on_dev, keep = _ptr(inputs)
        t = ctypes.c_uint64()
        _check(_lib.sisu_server_submit(self.h, circ.h, p, on_dev, ctypes.byref(t)))
        self._keep[t.value] = (keep, circ, circ.proof_len)
        return t.value

    def poll(self, ticket: int, with_order: bool = False):
        """(status, proof bytes or None, latency ms or None), plus the job's
        admission order (jobs admitted before it) when ``with_order``."""
        keep, circ, n = self._keep[ticket]
        st = ctypes.c_int()
        buf = ctypes.create_string_buffer(n)
        ln = ctypes.c_size_t()
        lat = ctypes.c_double()
        order = ctypes.c_uint64()
        _check(_lib.sisu_server_poll(self.h, ticket, ctypes.byref(st), ctypes.cast(buf, ctypes.c_void_p), n,
                                     ctypes.byref(ln), ctypes.byref(lat), ctypes.byref(order)))
        if st.value in (self.QUEUED, self.RUNNING):
            return (st.value, None, None, None) if with_order else (st.value, None, None)
        del self._keep[ticket]
        res = (st.value, (buf.raw[:ln.value] if st.value == self.DONE else None), lat.value)
        return res + (order.value,) if with_order else res

    def pause(self, paused: bool = True):
        """Stop (or resume) admissions; running jobs continue."""
        _check(_lib.sisu_server_pause(self.h, int(bool(paused))))

    def pending(self):
        q, r = ctypes.c_uint32(), ctypes.c_uint32()
        _check(_lib.sisu_server_pending(self.h, ctypes.byref(q), ctypes.byref(r)))
        return q.value, r.value

    def close(self):
        if getattr(self, "h", None):
            _lib.sisu_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def tune_copy_round(log_width: int, log_pairs: int, cta_threads: int, form: int = 0, min_items: int = 0):
    """Set the copy round's launch shape for one (layer width, pairs) class
    (``sisu_tune_copy_round``; cta_threads 0 restores the default)."""
    _check(_lib.sisu_tune_copy_round(int(log_width), int(log_pairs), int(cta_threads), int(form), int(min_items)))


def server_footprint(circ: Circuit, inputs_on_device: bool = False) -> int:
    """Device bytes a server job of ``circ`` takes from the budget."""
    n = ctypes.c_size_t()
    _check(_lib.sisu_job_footprint(circ.h, int(inputs_on_device), ctypes.byref(n)))
    return n.value


def verify(circ: Circuit, inputs: bytes, outputs: bytes, proof: bytes, domain: bytes | None = None) -> int:
    """SISU_OK (0) or a negative code, SISU_ERR_REJECT (-7) for a bad proof."""
    ib, ob, pb = (np.frombuffer(bytes(x), dtype=np.uint8) for x in (inputs, outputs, proof))
    db = np.frombuffer(bytes(domain), dtype=np.uint8) if domain else None
    return int(_lib.sisu_gkr_verify(circ.h, ib.ctypes.data, ob.ctypes.data, pb.ctypes.data, len(pb),
                                    db.ctypes.data if db is not None else None, len(db) if db is not None else 0))


def fr_batch(op: int, a, b, out, n: int, stream=None):
    """Elementwise field op on device arrays of n canonical elements."""
    pa, _, ka = _ptr(a)
    pb, _, kb = _ptr(b)
    po, _, ko = _ptr(out)
    _check(_lib.sisu_fr_batch(op, pa, pb, po, n, _stream(stream)))


def assoc_hash(elems, n: int | None = None, h_pre: bytes | None = None, stream=None) -> bytes:
    """Associative hash (Sec. 3.4.1, Algorithm 1) of n canonical elements
    (bytes/numpy on the host, or a CUDA tensor), continued from h_pre."""
    p, dev, keep = _ptr(elems)
    if n is None:
        n = (elems.numel() * elems.element_size() if hasattr(elems, "numel") else len(elems)) // 32
    out = ctypes.create_string_buffer(32)
    pre = None if h_pre is None else ctypes.create_string_buffer(bytes(h_pre), 32)
    _check(_lib.sisu_assoc_hash(p, n, ctypes.cast(pre, ctypes.c_void_p) if pre is not None else None, dev,
                                _stream(stream), ctypes.cast(out, ctypes.c_void_p)))
    return out.raw


def assoc_hash_segments(elems, offsets, h_pre: bytes | None = None, stream=None) -> list:
    """The hash of every segment [offsets[g], offsets[g+1]) of the elements,
    each continued from its 32-byte value in h_pre (concatenated) if given."""
    p, dev, keep = _ptr(elems)
    m = len(offsets) - 1
    offs, _keep_offs = _u64_offsets(offsets)
    out = ctypes.create_string_buffer(32 * max(1, m))
    pre = None if h_pre is None else ctypes.create_string_buffer(bytes(h_pre), 32 * m)
    _check(_lib.sisu_assoc_hash_segments(p, offs, m, ctypes.cast(pre, ctypes.c_void_p) if pre is not None else None,
                                         dev, _stream(stream), ctypes.cast(out, ctypes.c_void_p)))
    raw = out.raw
    return [raw[32 * g:32 * g + 32] for g in range(m)]


def pairwise_distinct_check(a, a_sorted, n: int | None = None, stream=None):
    """Algorithm 2 (Sec. 3.4.2): (result, hash of a, hash of a_sorted)."""
    pa, dev, ka = _ptr(a)
    ps, dev2, ks = _ptr(a_sorted)
    if dev != dev2:
        raise ValueError("a and a_sorted must both be host or both be device arrays")
    if n is None:
        n = (a.numel() * a.element_size() if hasattr(a, "numel") else len(a)) // 32
    res = ctypes.c_int(-1)
    ha, hs = ctypes.create_string_buffer(32), ctypes.create_string_buffer(32)
    _check(_lib.sisu_pairwise_distinct_check(pa, ps, n, dev, _stream(stream), ctypes.byref(res),
                                             ctypes.cast(ha, ctypes.c_void_p), ctypes.cast(hs, ctypes.c_void_p)))
    return res.value, ha.raw, hs.raw


def _u64_offsets(offsets):
    """Offsets as a C uint64 array: a contiguous numpy uint64 array is passed
    by pointer (the caller keeps the returned array alive), anything else
    converted first."""
    arr = np.ascontiguousarray(np.asarray(offsets), dtype=np.uint64)
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), arr


def assoc_epochs(a, a_sorted, slot_offsets, slots_per_epoch: int, stream=None):
    """Every slot's hash (Algorithm 1) and Algorithm 2 on every epoch of
    `slots_per_epoch` slots, the epoch's hash of `a` taken as the sum of its
    slots' hashes: (slot hashes, epoch results, epoch hashes of a, epoch
    hashes of a_sorted)."""
    pa, dev, ka = _ptr(a)
    ps, dev2, ks = _ptr(a_sorted)
    if dev != dev2:
        raise ValueError("a and a_sorted must both be host or both be device arrays")
    m = len(slot_offsets) - 1
    ne = m // slots_per_epoch if slots_per_epoch else 0
    offs, _keep_offs = _u64_offsets(slot_offsets)
    sh = ctypes.create_string_buffer(32 * max(1, m))
    res = (ctypes.c_int * max(1, ne))()
    ha, hs = ctypes.create_string_buffer(32 * max(1, ne)), ctypes.create_string_buffer(32 * max(1, ne))
    _check(_lib.sisu_assoc_epochs(pa, ps, offs, m, slots_per_epoch, dev, _stream(stream),
                                  ctypes.cast(sh, ctypes.c_void_p), res, ctypes.cast(ha, ctypes.c_void_p),
                                  ctypes.cast(hs, ctypes.c_void_p)))
    rsh, ra, rs = sh.raw, ha.raw, hs.raw
    return ([rsh[32 * g:32 * g + 32] for g in range(m)], list(res)[:ne],
            [ra[32 * e:32 * e + 32] for e in range(ne)], [rs[32 * e:32 * e + 32] for e in range(ne)])


def pairwise_distinct_check_segments(a, a_sorted, offsets, stream=None):
    """Algorithm 2 on every segment: (results, hashes of a, hashes of a_sorted)."""
    pa, dev, ka = _ptr(a)
    ps, dev2, ks = _ptr(a_sorted)
    if dev != dev2:
        raise ValueError("a and a_sorted must both be host or both be device arrays")
    m = len(offsets) - 1
    offs, _keep_offs = _u64_offsets(offsets)
    res = (ctypes.c_int * max(1, m))()
    ha, hs = ctypes.create_string_buffer(32 * max(1, m)), ctypes.create_string_buffer(32 * max(1, m))
    _check(_lib.sisu_pairwise_distinct_check_segments(pa, ps, offs, m, dev, _stream(stream), res,
                                                      ctypes.cast(ha, ctypes.c_void_p),
                                                      ctypes.cast(hs, ctypes.c_void_p)))
    ra, rs = ha.raw, hs.raw
    return list(res)[:m], [ra[32 * g:32 * g + 32] for g in range(m)], [rs[32 * g:32 * g + 32] for g in range(m)]


def sort_elements(elems, out=None, n: int | None = None, stream=None):
    """Ascending sort of canonical elements (the prover's A* for Algorithm 2).
    Host input (bytes/numpy) returns (sorted bytes, passes); for a CUDA
    tensor, `out` (a CUDA tensor of the same size, may be `elems`) receives
    the result and (out, passes) is returned."""
    p, dev, keep = _ptr(elems)
    if n is None:
        n = (elems.numel() * elems.element_size() if hasattr(elems, "numel") else len(elems)) // 32
    passes = ctypes.c_uint32(0)
    if dev:
        if out is None:
            raise ValueError("device input needs a device output buffer")
        po, dev_o, keep_o = _ptr(out)
        _check(_lib.sisu_sort_elements(p, n, 1, _stream(stream), po, ctypes.byref(passes)))
        return out, passes.value
    buf = ctypes.create_string_buffer(max(1, 32 * n))
    _check(_lib.sisu_sort_elements(p, n, 0, _stream(stream), ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(passes)))
    return buf.raw[:32 * n], passes.value


def statement_digest(data, length: int, stream=None) -> bytes:
    """The statement digest of ``length`` bytes of the CUDA device buffer
    ``data`` (host arrays are refused: the kernels read ``data`` in place)."""
    p, on_dev, keep = _ptr(data)
    if length and not on_dev:
        raise SisuError(-1, "data must be a CUDA device buffer")
    out = ctypes.create_string_buffer(32)
    _check(_lib.sisu_statement_digest(p, length, ctypes.cast(out, ctypes.c_void_p), _stream(stream)))
    return out.raw


def statement_digest_noalloc(data, length: int, out, stream=None):
    """The statement digest written to the 32-byte device buffer ``out``,
    using the library's fixed scratch instead of any allocation (inputs up
    to 64 MiB; see include/sisu.h for who needs this and its limits)."""
    p, on_dev, keep = _ptr(data)
    po, out_dev, keep_out = _ptr(out)
    if (length and not on_dev) or not out_dev:
        raise SisuError(-1, "data and out must be CUDA device buffers")
    _check(_lib.sisu_statement_digest_noalloc(p, length, po, _stream(stream)))


def microbench(kind: int, blocks: int, threads: int, iters: int, stream=None):
    """(milliseconds, operations) of an integer-pipe microbenchmark."""
    ms, ops = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sisu_microbench(kind, blocks, threads, iters, _stream(stream), ctypes.byref(ms), ctypes.byref(ops)))
    return ms.value, ops.value


def profile_enable(kind_mask: int):
    """Time the launches of the kernel kinds in the mask with CUDA events."""
    _check(_lib.sisu_profile_enable(kind_mask))


def profile_launches(kind: int, cap: int = 4096):
    """[(milliseconds, field products)] of the recorded launches of one kind."""
    ms = (ctypes.c_double * cap)()
    w = (ctypes.c_double * cap)()
    n = ctypes.c_size_t()
    _check(_lib.sisu_profile_launches(kind, ms, w, cap, ctypes.byref(n)))
    return [(ms[i], w[i]) for i in range(min(cap, n.value))]


def profile_read(kind: int):
    """(milliseconds, launches, algorithmic field products) since the last read."""
    ms, n, w = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double()
    _check(_lib.sisu_profile_read(kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
    return ms.value, int(n.value), w.value


def last_error() -> str:
    return _lib.sisu_last_error().decode(errors="replace")
