"""ctypes binding to the plain C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sisu_oracle.c")
LIB_PATH = os.path.join(HERE, "libsisu_oracle.so")

OK, ERR_ARG, ERR_CANON, ERR_REJECT, ERR_OOM = 0, -1, -2, -3, -4


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2; OpenMP loops that run on one
    thread unless Oracle.set_threads asks for more)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, SRC])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _u8(b):
    return ctypes.cast(ctypes.c_char_p(bytes(b)), ctypes.POINTER(ctypes.c_uint8))


class _CircuitHandle:
    def __init__(self, lib, circ):
        self.lib = lib
        err = ctypes.c_int(0)
        u32 = ctypes.POINTER(ctypes.c_uint32)
        if getattr(circ, "accumulates", False):  # accumulation gates: entry lists
            widths, cnt, outs, types, in1, in2 = circ.flat_entries()
            self._keep = (widths, cnt, outs, types, in1, in2)
            self.h = lib.so_circuit_new_entries(
                ctypes.c_uint32(circ.depth), widths.ctypes.data_as(u32), cnt.ctypes.data_as(u32),
                outs.ctypes.data_as(u32), types.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                in1.ctypes.data_as(u32), in2.ctypes.data_as(u32), ctypes.c_uint32(circ.n_copies),
                ctypes.byref(err))
        else:
            widths, types, in1, in2 = circ.flat()
            self._keep = (widths, types, in1, in2)
            self.h = lib.so_circuit_new(
                ctypes.c_uint32(circ.depth), widths.ctypes.data_as(u32),
                types.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                in1.ctypes.data_as(u32), in2.ctypes.data_as(u32),
                ctypes.c_uint32(circ.n_copies), ctypes.byref(err))
        if not self.h:
            raise ValueError(f"oracle rejected the circuit (code {err.value})")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.so_circuit_free(self.h)
            self.h = None


class _GeneralHandle:
    def __init__(self, lib, circ):
        self.lib = lib
        err = ctypes.c_int(0)
        u32 = ctypes.POINTER(ctypes.c_uint32)
        d = circ.depth
        widths = np.ascontiguousarray(circ.widths, dtype=np.uint32)
        types = np.ascontiguousarray(np.concatenate([circ.types[i] for i in range(d)]), dtype=np.uint8)
        in1 = np.ascontiguousarray(np.concatenate([circ.in1[i] for i in range(d)]), dtype=np.uint32)
        src = np.ascontiguousarray(np.concatenate([circ.layer_src(i) for i in range(d)]), dtype=np.uint32)
        in2 = np.ascontiguousarray(np.concatenate([circ.in2[i] for i in range(d)]), dtype=np.uint32)
        self._keep = (widths, types, in1, src, in2)
        self.h = lib.so_gcircuit_new(ctypes.c_uint32(d), widths.ctypes.data_as(u32),
                                     types.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), in1.ctypes.data_as(u32),
                                     src.ctypes.data_as(u32), in2.ctypes.data_as(u32), ctypes.c_uint32(circ.n_copies),
                                     ctypes.byref(err))
        if not self.h:
            raise ValueError(f"oracle rejected the general circuit (code {err.value})")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.so_gcircuit_free(self.h)
            self.h = None


class Oracle:
    """The oracle's entry points, on canonical little-endian byte strings."""

    def __init__(self, lib_path: str | None = None):
        lib = ctypes.CDLL(lib_path or build_oracle())
        vp, u8p, u32p, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint32), ctypes.c_size_t
        lib.so_circuit_new.restype = vp
        lib.so_circuit_new.argtypes = [ctypes.c_uint32, u32p, u8p, u32p, u32p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int)]
        lib.so_circuit_new_entries.restype = vp
        lib.so_circuit_new_entries.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u8p, u32p, u32p, ctypes.c_uint32,
                                               ctypes.POINTER(ctypes.c_int)]
        lib.so_circuit_free.argtypes = [vp]
        lib.so_proof_len.restype = sz
        lib.so_proof_len.argtypes = [vp]
        lib.so_prove.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p, sz, ctypes.c_char_p, sz, ctypes.POINTER(sz)]
        lib.so_verify.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, sz, ctypes.c_char_p, sz]
        lib.so_fr_op.argtypes = [ctypes.c_int, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, sz]
        lib.so_reduce512.argtypes = [ctypes.c_char_p, ctypes.c_char_p]
        lib.so_sha256.argtypes = [ctypes.c_char_p, sz, ctypes.c_char_p]
        lib.so_sha256_constants.argtypes = [u32p, u32p]
        lib.so_statement_digest.argtypes = [ctypes.c_char_p, sz, ctypes.c_char_p]
        lib.so_mle.argtypes = [ctypes.c_char_p, ctypes.c_uint32, ctypes.c_char_p, ctypes.c_char_p]
        lib.so_eval_layer.argtypes = [vp, ctypes.c_char_p, ctypes.c_uint32, ctypes.c_char_p]
        lib.so_outputs.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
        lib.so_wiring_digest.argtypes = [vp, ctypes.c_char_p]
        lib.so_assoc_F.argtypes = [ctypes.c_char_p, sz, ctypes.c_char_p]
        lib.so_assoc_hash.argtypes = [ctypes.c_char_p, sz, ctypes.c_char_p, ctypes.c_char_p]
        lib.so_pairwise_distinct_check.argtypes = [ctypes.c_char_p, ctypes.c_char_p, sz]
        lib.so_gcircuit_new.restype = vp
        lib.so_gcircuit_new.argtypes = [ctypes.c_uint32, u32p, u8p, u32p, u32p, u32p, ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_int)]
        lib.so_gcircuit_free.argtypes = [vp]
        lib.so_gproof_len.restype = sz
        lib.so_gproof_len.argtypes = [vp]
        lib.so_gprove.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p, sz, ctypes.c_char_p, sz, ctypes.POINTER(sz)]
        lib.so_gverify.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, sz, ctypes.c_char_p, sz]
        lib.so_goutputs.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
        lib.so_gcircuit_log_xwidth.restype = ctypes.c_uint32
        lib.so_gcircuit_log_xwidth.argtypes = [vp, ctypes.c_uint32]
        lib.so_gcircuit_blocks.restype = ctypes.c_uint32
        lib.so_gcircuit_blocks.argtypes = [vp, ctypes.c_uint32]
        lib.so_set_threads.restype = ctypes.c_int
        lib.so_set_threads.argtypes = [ctypes.c_int]
        lib.so_circuit_log_copies.restype = ctypes.c_uint32
        lib.so_circuit_log_copies.argtypes = [vp]
        lib.so_circuit_log_width.restype = ctypes.c_uint32
        lib.so_circuit_log_width.argtypes = [vp, ctypes.c_uint32]
        self.lib = lib
        self._handles = {}

    # -- general circuits (Sec. 2.7) ---------------------------------------
    def ghandle(self, circ):
        key = ("g", id(circ))
        h = self._handles.get(key)
        if h is None or h[0] is not circ:
            h = (circ, _GeneralHandle(self.lib, circ))
            self._handles[key] = h
        return h[1].h

    def general_proof_len(self, circ) -> int:
        return int(self.lib.so_gproof_len(self.ghandle(circ)))

    def general_shape(self, circ):
        """Per gate layer: (log2 width of its virtual layer, blocks)."""
        h = self.ghandle(circ)
        return [(int(self.lib.so_gcircuit_log_xwidth(h, i)), int(self.lib.so_gcircuit_blocks(h, i)))
                for i in range(circ.depth)]

    def prove_general(self, circ, inputs: bytes, domain: bytes | None = None) -> bytes:
        n = self.general_proof_len(circ)
        buf = ctypes.create_string_buffer(n)
        ln = ctypes.c_size_t(0)
        rc = self.lib.so_gprove(self.ghandle(circ), bytes(inputs), domain, len(domain or b""), buf, n,
                                ctypes.byref(ln))
        if rc != OK:
            raise ValueError(f"oracle prove failed (code {rc})")
        return buf.raw[:ln.value]

    def verify_general(self, circ, inputs: bytes, outputs: bytes, proof: bytes,
                       domain: bytes | None = None) -> int:
        return int(self.lib.so_gverify(self.ghandle(circ), bytes(inputs), bytes(outputs), bytes(proof),
                                       len(proof), domain, len(domain or b"")))

    def outputs_general(self, circ, inputs: bytes) -> bytes:
        out = ctypes.create_string_buffer(32 * circ.n_copies * circ.widths[0])
        rc = self.lib.so_goutputs(self.ghandle(circ), bytes(inputs), out)
        if rc != OK:
            raise ValueError(f"oracle eval failed (code {rc})")
        return out.raw

    def set_threads(self, n: int) -> int:
        """Threads of the prover's copy sums, folds and evaluation; returns
        the number in effect (the proof bytes do not depend on it)."""
        return int(self.lib.so_set_threads(int(n)))

    # -- circuits ---------------------------------------------------------
    def handle(self, circ):
        key = id(circ)
        h = self._handles.get(key)
        if h is None or h[0] is not circ:
            h = (circ, _CircuitHandle(self.lib, circ))
            self._handles[key] = h
        return h[1].h

    def proof_len(self, circ) -> int:
        return int(self.lib.so_proof_len(self.handle(circ)))

    def log_sizes(self, circ):
        h = self.handle(circ)
        return (int(self.lib.so_circuit_log_copies(h)),
                [int(self.lib.so_circuit_log_width(h, i)) for i in range(circ.depth + 1)])

    def wiring_digest(self, circ) -> bytes:
        out = ctypes.create_string_buffer(32)
        self.lib.so_wiring_digest(self.handle(circ), out)
        return out.raw

    def prove(self, circ, inputs: bytes, domain: bytes | None = None) -> bytes:
        n = self.proof_len(circ)
        buf = ctypes.create_string_buffer(n)
        ln = ctypes.c_size_t(0)
        rc = self.lib.so_prove(self.handle(circ), bytes(inputs), domain, len(domain or b""),
                               buf, n, ctypes.byref(ln))
        if rc != OK:
            raise ValueError(f"oracle prove failed (code {rc})")
        return buf.raw[:ln.value]

    def verify(self, circ, inputs: bytes, outputs: bytes, proof: bytes,
               domain: bytes | None = None) -> int:
        return int(self.lib.so_verify(self.handle(circ), bytes(inputs), bytes(outputs), bytes(proof),
                                      len(proof), domain, len(domain or b"")))

    def outputs(self, circ, inputs: bytes) -> bytes:
        out = ctypes.create_string_buffer(32 * circ.n_copies * circ.widths[0])
        rc = self.lib.so_outputs(self.handle(circ), bytes(inputs), out)
        if rc != OK:
            raise ValueError(f"oracle eval failed (code {rc})")
        return out.raw

    def eval_layer(self, circ, inputs: bytes, layer: int) -> bytes:
        c, s = self.log_sizes(circ)
        out = ctypes.create_string_buffer(32 << (c + s[layer]))
        rc = self.lib.so_eval_layer(self.handle(circ), bytes(inputs), layer, out)
        if rc != OK:
            raise ValueError(f"oracle eval failed (code {rc})")
        return out.raw

    # -- primitives ---------------------------------------------------------
    def fr_op(self, op: int, a: bytes, b: bytes | None = None) -> bytes:
        n = len(a) // 32
        out = ctypes.create_string_buffer(32 * n)
        rc = self.lib.so_fr_op(op, bytes(a), bytes(b if b is not None else a), out, n)
        if rc != OK:
            raise ValueError(f"oracle field op failed (code {rc})")
        return out.raw

    def reduce512(self, x: int) -> int:
        out = ctypes.create_string_buffer(32)
        self.lib.so_reduce512(x.to_bytes(64, "little"), out)
        return int.from_bytes(out.raw, "little")

    def sha256(self, msg: bytes) -> bytes:
        out = ctypes.create_string_buffer(32)
        self.lib.so_sha256(bytes(msg), len(msg), out)
        return out.raw

    def sha256_constants(self):
        k = (ctypes.c_uint32 * 64)()
        h = (ctypes.c_uint32 * 8)()
        self.lib.so_sha256_constants(k, h)
        return list(k), list(h)

    def statement_digest(self, data: bytes) -> bytes:
        out = ctypes.create_string_buffer(32)
        self.lib.so_statement_digest(bytes(data), len(data), out)
        return out.raw

    def mle(self, table: bytes, m: int, point: bytes) -> bytes:
        out = ctypes.create_string_buffer(32)
        rc = self.lib.so_mle(bytes(table), m, bytes(point), out)
        if rc != OK:
            raise ValueError(f"oracle mle failed (code {rc})")
        return out.raw


    # -- associative hash (Sec. 3.4.1) and pairwise-distinct check (Sec. 3.4.2)
    def assoc_F(self, elems: bytes) -> bytes:
        n = len(elems) // 32
        out = ctypes.create_string_buffer(max(1, 32 * n))
        rc = self.lib.so_assoc_F(bytes(elems), n, out)
        if rc != OK:
            raise ValueError(f"oracle F failed (code {rc})")
        return out.raw[:32 * n]

    def assoc_hash(self, elems: bytes, h_pre: bytes | None = None) -> bytes:
        out = ctypes.create_string_buffer(32)
        rc = self.lib.so_assoc_hash(bytes(elems), len(elems) // 32, None if h_pre is None else bytes(h_pre), out)
        if rc != OK:
            raise ValueError(f"oracle associative hash failed (code {rc})")
        return out.raw

    def pairwise_distinct_check(self, a: bytes, a_sorted: bytes) -> int:
        assert len(a) == len(a_sorted)
        rc = self.lib.so_pairwise_distinct_check(bytes(a), bytes(a_sorted), len(a) // 32)
        if rc < 0:
            raise ValueError(f"oracle pairwise-distinct check failed (code {rc})")
        return rc


def ints_to_bytes(vals) -> bytes:
    return b"".join(int(v).to_bytes(32, "little") for v in vals)


def bytes_to_ints(b: bytes) -> list:
    return [int.from_bytes(b[i:i + 32], "little") for i in range(0, len(b), 32)]


def as_u64(b: bytes) -> np.ndarray:
    return np.frombuffer(b, dtype="<u8").reshape(-1, 4)
