"""Seeded synthetic inputs, shared by the CPU oracle's tests, the GPU tests and
the benchmark.

This module makes inputs only: byte strings, LZ77 token streams built by
construction, file-size mixes and arrival times.  It holds none of the codec's
arithmetic (no parsing, no Huffman coding, no decoding).  The generators are
plain C (``gen.c``, counter-based splitmix64 draws) behind ctypes, compiled on
first use with gcc; the mixes and arrivals use numpy's seeded PCG64.

The paper's data sets (an English Wikipedia XML dump and the Hollywood-2009
Matrix-Market CSV file, Section 5) are not available; ``markov_text`` and
``csv_records`` stand in for them.  The workload table ``WORKLOADS`` names
every configuration the tests and the benchmark use.
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
_LIB_PATH = os.path.join(_BUILD, "libgmpgen.so")
_lock = threading.Lock()
_lib = None

# Concentration of the Markov successor distribution.  Calibrated once so that
# the text compresses about 2.5-3x with this project's compressors (LZ77 with a
# 8-32 KiB window, 12-bit length-limited Huffman): rho = 0.25 (order 2) and
# 0.15 (order 3) with lambda = 0.9 give 2.6-2.7x.
TEXT_LAMBDA = {2: 0.9, 3: 0.9}
TEXT_RHO = {2: 0.25, 3: 0.15}


def build(force: bool = False) -> str:
    """Compile gen.c into _build/libgmpgen.so (gcc, no GPU needed)."""
    src = os.path.join(_HERE, "gen.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                               "-o", tmp, src, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.gen_markov_text.argtypes = [u8p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int]
            lib.gen_csv_records.argtypes = [u8p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int]
            lib.gen_nesting_tokens.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t, u32p, u32p,
                                               u32p, ctypes.c_size_t, u8p, ctypes.c_size_t,
                                               ctypes.POINTER(ctypes.c_size_t),
                                               ctypes.POINTER(ctypes.c_size_t)]
            _lib = lib
    return _lib


def _ptr(a, t=ctypes.c_uint8):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def markov_text(n: int, seed: int, order: int = 2, lam: float | None = None,
                rho: float | None = None) -> np.ndarray:
    """n bytes of order-`order` byte Markov text (English-like letters, ~18 %
    spaces, a 1.5 % noise floor that the 4096-entry sampling table turns into
    about 1-2 % of bytes outside letters and punctuation)."""
    if lam is None:
        lam = TEXT_LAMBDA[order]
    if rho is None:
        rho = TEXT_RHO[order]
    out = np.empty(n, dtype=np.uint8)
    rc = _get().gen_markov_text(_ptr(out), n, seed & (2**64 - 1), order, lam, rho, _threads())
    if rc != 0:
        raise ValueError("bad markov_text parameters")
    return out


def csv_records(n: int, seed: int, zipf_s: float = 1.1, p_repeat: float = 0.1) -> np.ndarray:
    """n bytes of CSV-like rows of 8 fields (Zipf ids, 2-decimal prices, ISO
    dates over 5 years, 20 categorical tokens); a row repeats one of the last
    64 rows with one field changed with probability p_repeat."""
    out = np.empty(n, dtype=np.uint8)
    rc = _get().gen_csv_records(_ptr(out), n, seed & (2**64 - 1), zipf_s, p_repeat, _threads())
    if rc != 0:
        raise ValueError("bad csv_records parameters")
    return out


@dataclass
class TokenStream:
    """A block's LZ77 sequences: sequence i is lit_len[i] literal bytes (taken
    in order from `lits`) followed by a copy of mlen[i] bytes from distance
    off[i] (mlen 0: no copy)."""
    lit_len: np.ndarray
    mlen: np.ndarray
    off: np.ndarray
    lits: np.ndarray

    @property
    def n_seq(self) -> int:
        return int(self.lit_len.size)

    @property
    def out_bytes(self) -> int:
        return int(self.lit_len.sum(dtype=np.int64) + self.mlen.sum(dtype=np.int64))


def nesting_tokens(seed: int, m: int, n_inst: int) -> TokenStream:
    """Token stream of the nesting-depth data set with m interleaved repeated
    16-byte strings (depth 32/m inside each 32-sequence group)."""
    cap = n_inst + 2
    ll = np.zeros(cap, np.uint32)
    ml = np.zeros(cap, np.uint32)
    of = np.zeros(cap, np.uint32)
    lits = np.zeros(17 * (m + n_inst) + 16, np.uint8)
    nseq = ctypes.c_size_t()
    nl = ctypes.c_size_t()
    rc = _get().gen_nesting_tokens(seed & (2**64 - 1), m, n_inst, _ptr(ll, ctypes.c_uint32),
                                   _ptr(ml, ctypes.c_uint32), _ptr(of, ctypes.c_uint32), cap,
                                   _ptr(lits), lits.size, ctypes.byref(nseq), ctypes.byref(nl))
    if rc != 0:
        raise ValueError(f"nesting_tokens failed ({rc})")
    k = nseq.value
    return TokenStream(ll[:k].copy(), ml[:k].copy(), of[:k].copy(), lits[:nl.value].copy())


# --------------------------------------------------------------------------
# Workloads.  Sizes, block sizes, sub-block counts and windows of every
# configuration used by the tests and the benchmark.

@dataclass(frozen=True)
class Workload:
    name: str
    kind: str          # "text2", "text3" (Markov order) or "csv"
    size: int          # decompressed bytes
    block_size: int
    n_sub: int         # K, sub-blocks per block
    window: int
    seed: int
    modes: tuple = ("mrr",)

    def data(self, size: int | None = None) -> np.ndarray:
        return make_data(self.kind, self.size if size is None else size, self.seed)


def make_data(kind: str, size: int, seed: int) -> np.ndarray:
    if kind == "text2":
        return markov_text(size, seed, order=2)
    if kind == "text3":
        return markov_text(size, seed, order=3)
    if kind == "csv":
        return csv_records(size, seed)
    raise ValueError(kind)


KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30

WORKLOADS = {
    # 1 MiB order-2 Markov text, 64 KiB blocks of 16 sub-blocks, 8 KiB window, MRR
    "text1m": Workload("text1m", "text2", 1 * MiB, 64 * KiB, 16, 8 * KiB, 1, ("mrr",)),
    # 256 MiB order-3 Markov text, 256 KiB blocks of 32 sub-blocks, 32 KiB window, MRR and DE
    "text256m": Workload("text256m", "text3", 256 * MiB, 256 * KiB, 32, 32 * KiB, 2, ("mrr", "de")),
    # 1 GiB CSV-like numeric records, 256 KiB blocks of 32 sub-blocks, 32 KiB window, MRR and DE
    "csv1g": Workload("csv1g", "csv", 1 * GiB, 256 * KiB, 32, 32 * KiB, 3, ("mrr", "de")),
}


def file_mix(seed: int, n_files: int = 4096, lo: int = 4 * KiB, hi: int = 16 * MiB,
             total_cap: int | None = None):
    """Batched workload: n_files sizes log-uniform in [lo, hi], content
    (Markov text / CSV records) and mode (MRR / DE) by seeded coins.  With
    total_cap, the seeded prefix of the list whose total stays within
    total_cap bytes.  Returns a list of (size, kind, mode, seed)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n_files)).astype(np.int64)
    kinds = np.where(rng.random(n_files) < 0.5, "text3", "csv")
    modes = np.where(rng.random(n_files) < 0.5, "mrr", "de")
    seeds = rng.integers(1, 2**62, n_files)
    out = []
    tot = 0
    for i in range(n_files):
        if total_cap is not None and tot + int(sizes[i]) > total_cap:
            break
        out.append((int(sizes[i]), str(kinds[i]), str(modes[i]), int(seeds[i])))
        tot += int(sizes[i])
    return out


def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """n arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def request_mix(seed: int, n: int, lo: int = 16 * KiB, hi: int = 64 * MiB):
    """Serving requests: sizes log-uniform in [lo, hi], mixed content and
    modes.  Returns a list of (size, kind, mode, seed)."""
    return file_mix(seed, n, lo, hi)
