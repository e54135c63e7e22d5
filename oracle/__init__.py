"""CPU oracle for the Gompresso-style decompression path.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The product
library (``paper_1606_00519_gb300``) never imports, links or calls it, and the
two share no code: only the stream format (documented field by field in
``gmp_oracle.c``'s header) is common.

The arithmetic lives in ``gmp_oracle.c`` (plain serial C, each function citing
the paper's section it follows), compiled with gcc on first use into
``oracle/_build/liboracle.so``.  This module is argument marshalling only.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against values fixed by the paper or by mathematics (round trips, the Fig. 1
example, the MRR examples of Sec. 4.1 and Sec. 5.1, Kraft equality,
textbook-Huffman optimality, brute-force enumeration on tiny inputs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status values of the stream format
OK, BAD_HEADER, CORRUPT_SYMBOL, BITSTREAM, BAD_OFFSET, OUTPUT_OVERRUN, MRR_NO_PROGRESS = range(7)
STATUS_NAMES = {0: "OK", 1: "BAD_HEADER", 2: "CORRUPT_SYMBOL", 3: "BITSTREAM", 4: "BAD_OFFSET",
                5: "OUTPUT_OVERRUN", 6: "MRR_NO_PROGRESS", -1: "ERR_ARG", -2: "ERR_CAP", -3: "ERR_NOMEM"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}")


def build(force: bool = False) -> str:
    """Compile gmp_oracle.c (gcc, no GPU needed)."""
    src = os.path.join(_HERE, "gmp_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, src])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_uint32), ("n_sub", ctypes.c_uint32), ("window", ctypes.c_uint32),
                ("cwl", ctypes.c_uint32), ("min_match", ctypes.c_uint32), ("max_match", ctypes.c_uint32),
                ("chain_depth", ctypes.c_uint32), ("de", ctypes.c_uint32), ("byte_mode", ctypes.c_uint32)]


class Info(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("block_size", ctypes.c_uint32), ("n_sub", ctypes.c_uint32),
                ("cwl", ctypes.c_uint32), ("window", ctypes.c_uint32), ("min_match", ctypes.c_uint32),
                ("max_match", ctypes.c_uint32), ("orig_size", ctypes.c_uint64), ("n_blocks", ctypes.c_uint64),
                ("stream_bytes", ctypes.c_uint64)]


class Report(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_uint64), ("n_seq", ctypes.c_uint64), ("n_matches", ctypes.c_uint64),
                ("lit_bytes", ctypes.c_uint64), ("match_bytes", ctypes.c_uint64),
                ("kraft_ok", ctypes.c_int32), ("lengths_ok", ctypes.c_int32), ("offsets_ok", ctypes.c_int32),
                ("blocks_ok", ctypes.c_int32), ("subblocks_ok", ctypes.c_int32),
                ("de_weak_ok", ctypes.c_int32), ("mrr_ok", ctypes.c_int32),
                ("groups", ctypes.c_uint64), ("rounds", ctypes.c_uint64), ("max_rounds", ctypes.c_uint64),
                ("copies", ctypes.c_uint64), ("round_hist", ctypes.c_uint64 * 34),
                ("first_error", ctypes.c_int32), ("subblocks_even", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "round_hist"}
        d["round_hist"] = list(self.round_hist)
        return d


def _get():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            sz = ctypes.c_uint64
            L.orc_offset_encode.argtypes = [ctypes.c_uint32, u32p, u32p, u32p]
            L.orc_offset_nextra.argtypes = [ctypes.c_uint32]
            L.orc_offset_nextra.restype = ctypes.c_uint32
            L.orc_offset_decode.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_offset_decode.restype = ctypes.c_uint32
            L.orc_package_merge.argtypes = [u64p, ctypes.c_int, ctypes.c_int, u8p]
            L.orc_canonical_codes.argtypes = [u8p, ctypes.c_int, u32p]
            L.orc_kraft_scaled.argtypes = [u8p, ctypes.c_int, ctypes.c_int]
            L.orc_kraft_scaled.restype = ctypes.c_uint64
            L.orc_compress_bound.argtypes = [sz, ctypes.POINTER(Params)]
            L.orc_compress_bound.restype = ctypes.c_uint64
            L.orc_compress.argtypes = [u8p, sz, ctypes.POINTER(Params), u8p, sz]
            L.orc_compress.restype = ctypes.c_int64
            L.orc_encode_tokens.argtypes = [u32p, u32p, u32p, sz, u8p, ctypes.POINTER(Params), u8p, sz]
            L.orc_encode_tokens.restype = ctypes.c_int64
            L.orc_stream_info.argtypes = [u8p, sz, ctypes.POINTER(Info)]
            L.orc_decompress.argtypes = [u8p, sz, u8p, sz, u64p]
            L.orc_decompress_block.argtypes = [u8p, sz, sz, u8p, sz]
            L.orc_block_tokens.argtypes = [u8p, sz, sz, u32p, u32p, u32p, sz, u8p, sz, u64p, u64p]
            L.orc_lz77_decode.argtypes = [u32p, u32p, u32p, sz, u8p, ctypes.c_uint32, u8p, sz, u64p]
            L.orc_validate.argtypes = [u8p, sz, ctypes.POINTER(Report)]
            L.orc_mrr_rounds.argtypes = [u32p, u32p, u32p, sz, u8p, ctypes.c_int, u32p, u64p]
            _lib = L
    return _lib


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _u32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _bytes(x) -> np.ndarray:
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x, dtype=np.uint8)
    return np.frombuffer(bytes(x), dtype=np.uint8)


def params(block_size=64 * 1024, n_sub=16, window=8 * 1024, cwl=12, max_match=64, chain_depth=64,
           de=False, byte_mode=False) -> Params:
    """Compressor parameters; byte_mode selects Gompresso/Byte records
    (no Huffman trees, n_sub and cwl unused)."""
    return Params(block_size, n_sub, window, cwl, 3, max_match, chain_depth, 1 if de else 0,
                  1 if byte_mode else 0)


# ---------------------------------------------------------------- primitives

def offset_encode(d: int):
    s, n, e = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    rc = _get().orc_offset_encode(d, ctypes.byref(s), ctypes.byref(n), ctypes.byref(e))
    if rc:
        raise OracleError(rc, "offset_encode")
    return s.value, n.value, e.value


def offset_nextra(sym: int) -> int:
    return _get().orc_offset_nextra(sym)


def offset_decode(sym: int, extra: int) -> int:
    return _get().orc_offset_decode(sym, extra)


def package_merge(freq, limit: int) -> np.ndarray:
    f = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(f.size, np.uint8)
    rc = _get().orc_package_merge(_u64(f), f.size, limit, _u8(out))
    if rc:
        raise OracleError(rc, "package_merge")
    return out


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(ln.size, np.uint32)
    rc = _get().orc_canonical_codes(_u8(ln), ln.size, _u32(out))
    if rc:
        raise OracleError(rc, "canonical_codes")
    return out


def kraft_scaled(lengths, limit: int) -> int:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    return int(_get().orc_kraft_scaled(_u8(ln), ln.size, limit))


# ---------------------------------------------------------------- codec

def compress(data, p: Params) -> np.ndarray:
    src = _bytes(data)
    L = _get()
    cap = int(L.orc_compress_bound(src.size, ctypes.byref(p)))
    out = np.zeros(cap, np.uint8)
    n = L.orc_compress(_u8(src), src.size, ctypes.byref(p), _u8(out), cap)
    if n < 0:
        raise OracleError(n, "compress")
    return out[:n].copy()


def encode_tokens(ts, p: Params) -> np.ndarray:
    """One-block stream holding the given sequences (a datagen.TokenStream or
    any object with lit_len, mlen, off, lits arrays)."""
    ll = np.ascontiguousarray(ts.lit_len, np.uint32)
    ml = np.ascontiguousarray(ts.mlen, np.uint32)
    of = np.ascontiguousarray(ts.off, np.uint32)
    lits = np.ascontiguousarray(ts.lits, np.uint8)
    if lits.size == 0:
        lits = np.zeros(1, np.uint8)
    tot = int(ll.sum(dtype=np.int64) + ml.sum(dtype=np.int64))
    cap = 4096 + 64 * 12 + 2 * tot + ll.size * 8
    out = np.zeros(cap, np.uint8)
    n = _get().orc_encode_tokens(_u32(ll), _u32(ml), _u32(of), ll.size, _u8(lits), ctypes.byref(p), _u8(out), cap)
    if n < 0:
        raise OracleError(n, "encode_tokens")
    return out[:n].copy()


def stream_info(stream) -> Info:
    s = _bytes(stream)
    info = Info()
    rc = _get().orc_stream_info(_u8(s), s.size, ctypes.byref(info))
    if rc:
        raise OracleError(rc, "stream_info")
    return info


def decompress(stream) -> np.ndarray:
    s = _bytes(stream)
    info = stream_info(s)
    out = np.zeros(max(1, info.orig_size), np.uint8)
    n = ctypes.c_uint64()
    rc = _get().orc_decompress(_u8(s), s.size, _u8(out), out.size, ctypes.byref(n))
    if rc:
        raise OracleError(rc, "decompress")
    return out[:n.value]


def decompress_status(stream) -> int:
    """Status code of a full serial decode (0 when the stream is valid)."""
    s = _bytes(stream)
    info = Info()
    L = _get()
    rc = L.orc_stream_info(_u8(s), s.size, ctypes.byref(info))
    if rc:
        return rc
    out = np.zeros(max(1, min(info.orig_size, 1 << 34)), np.uint8)
    n = ctypes.c_uint64()
    return L.orc_decompress(_u8(s), s.size, _u8(out), out.size, ctypes.byref(n))


def decompress_block(stream, b: int) -> np.ndarray:
    s = _bytes(stream)
    info = stream_info(s)
    size = min(info.block_size, info.orig_size - b * info.block_size)
    out = np.zeros(max(1, size), np.uint8)
    rc = _get().orc_decompress_block(_u8(s), s.size, b, _u8(out), out.size)
    if rc:
        raise OracleError(rc, f"decompress_block {b}")
    return out[:size]


@dataclass
class Tokens:
    lit_len: np.ndarray
    mlen: np.ndarray
    off: np.ndarray
    lits: np.ndarray


def block_tokens(stream, b: int) -> Tokens:
    s = _bytes(stream)
    info = stream_info(s)
    size = min(info.block_size, info.orig_size - b * info.block_size)
    cap = size // 3 + 2
    ll = np.zeros(cap, np.uint32)
    ml = np.zeros(cap, np.uint32)
    of = np.zeros(cap, np.uint32)
    lits = np.zeros(max(1, size), np.uint8)
    ns, nl = ctypes.c_uint64(), ctypes.c_uint64()
    rc = _get().orc_block_tokens(_u8(s), s.size, b, _u32(ll), _u32(ml), _u32(of), cap, _u8(lits), lits.size,
                                 ctypes.byref(ns), ctypes.byref(nl))
    if rc:
        raise OracleError(rc, f"block_tokens {b}")
    k = ns.value
    return Tokens(ll[:k].copy(), ml[:k].copy(), of[:k].copy(), lits[:nl.value].copy())


def lz77_decode(lit_len, mlen, off, lits, window: int = 32768) -> np.ndarray:
    ll = np.ascontiguousarray(lit_len, np.uint32)
    ml = np.ascontiguousarray(mlen, np.uint32)
    of = np.ascontiguousarray(off, np.uint32)
    lt = _bytes(lits)
    if lt.size == 0:
        lt = np.zeros(1, np.uint8)
    tot = int(ll.sum(dtype=np.int64) + ml.sum(dtype=np.int64))
    out = np.zeros(max(1, tot), np.uint8)
    n = ctypes.c_uint64()
    rc = _get().orc_lz77_decode(_u32(ll), _u32(ml), _u32(of), ll.size, _u8(lt), window, _u8(out), out.size,
                                ctypes.byref(n))
    if rc:
        raise OracleError(rc, "lz77_decode")
    return out[:n.value]


def validate(stream) -> dict:
    s = _bytes(stream)
    r = Report()
    rc = _get().orc_validate(_u8(s), s.size, ctypes.byref(r))
    d = r.as_dict()
    d["rc"] = rc
    return d


def mrr_rounds(lit_len, mlen, off, lits, de_single_pass: bool = False) -> np.ndarray:
    """Rounds of each 32-sequence group under MRR (or 1 per group for the DE
    one-pass schedule); raises if the schedule would read unavailable bytes."""
    ll = np.ascontiguousarray(lit_len, np.uint32)
    ml = np.ascontiguousarray(mlen, np.uint32)
    of = np.ascontiguousarray(off, np.uint32)
    lt = _bytes(lits)
    if lt.size == 0:
        lt = np.zeros(1, np.uint8)
    ng = (ll.size + 31) // 32
    out = np.zeros(max(1, ng), np.uint32)
    n = ctypes.c_uint64()
    rc = _get().orc_mrr_rounds(_u32(ll), _u32(ml), _u32(of), ll.size, _u8(lt), 1 if de_single_pass else 0,
                               _u32(out), ctypes.byref(n))
    if rc:
        raise OracleError(rc, "mrr_rounds")
    return out[:ng]
