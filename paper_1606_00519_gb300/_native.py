"""Build and load libgmp.so (the C-ABI library declared in include/gmp.h).

The library is compiled in-tree with nvcc for sm_103a only (CUDA kernels and
host runtime), into ``paper_1606_00519_gb300/_build/libgmp.so``.  Loading it
does not need a GPU; calling its CUDA entry points does.  There is no CPU
fallback: if the library is missing, every decode call raises.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
CSRC = os.path.join(_PKG, "csrc")
INCLUDE = os.path.join(_ROOT, "include")
BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(BUILD, "libgmp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["gmp_decode.cu", "gmp_host.cpp", "gmp_compress.cpp", "gmp_server.cpp", "gmp_noalloc.cu",
           "gmp_gpucompress.cu", "gmp_gpuencode.cu"]

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; libgmp.so cannot be built")
    return cand


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libgmp.so."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    deps = [os.path.join(CSRC, s) for s in srcs] + [os.path.join(CSRC, f) for f in os.listdir(CSRC)
                                                    if f.endswith(".h")] + [os.path.join(INCLUDE, "gmp.h")]
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB_PATH
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = [*ARCH, "-lineinfo", "-Xptxas", "-warn-spills"]
        else:
            cmd[1:1] = ["-x", "c++", "-Xcompiler", "-pthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class BlockRef(ctypes.Structure):
    _fields_ = [("comp_offset", ctypes.c_uint64), ("comp_bytes", ctypes.c_uint64),
                ("out_offset", ctypes.c_uint64), ("out_bytes", ctypes.c_uint64)]


class StreamInfo(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("block_size", ctypes.c_uint32),
                ("n_sub", ctypes.c_uint32), ("cwl", ctypes.c_uint32), ("window", ctypes.c_uint32),
                ("min_match", ctypes.c_uint32), ("max_match", ctypes.c_uint32),
                ("orig_size", ctypes.c_uint64), ("n_blocks", ctypes.c_uint64), ("stream_bytes", ctypes.c_uint64),
                ("max_block_out", ctypes.c_uint32), ("max_block_seq", ctypes.c_uint32)]


class CompressOpts(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_uint32), ("n_sub", ctypes.c_uint32), ("window", ctypes.c_uint32),
                ("cwl", ctypes.c_uint32), ("max_match", ctypes.c_uint32), ("chain_depth", ctypes.c_uint32),
                ("de", ctypes.c_uint32), ("n_threads", ctypes.c_uint32), ("lazy", ctypes.c_uint32),
                ("byte_mode", ctypes.c_uint32)]


class ContextOpts(ctypes.Structure):
    _fields_ = [("max_block_out", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("collect_stats", ctypes.c_uint32),
                ("max_files", ctypes.c_uint32), ("resolve", ctypes.c_uint32), ("concurrent", ctypes.c_uint32)]


class FileDesc(ctypes.Structure):
    _fields_ = [("comp", ctypes.c_uint64), ("comp_bytes", ctypes.c_uint64), ("index", ctypes.c_uint64),
                ("n_blocks", ctypes.c_uint64), ("out", ctypes.c_uint64), ("out_cap", ctypes.c_uint64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("n_lanes", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("max_block_out", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("d_out", ctypes.c_uint64),
                ("out_bytes", ctypes.c_uint64), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("t_gpu_ready", ctypes.c_double), ("t_gpu_done", ctypes.c_double)]


class GpuCompressTimes(ctypes.Structure):
    _fields_ = [("match_ms", ctypes.c_double), ("parse_ms", ctypes.c_double), ("encode_ms", ctypes.c_double),
                ("compressed_bytes", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("best_ms", ctypes.c_double),
                ("shapes_tried", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_uint64), ("rounds", ctypes.c_uint64), ("de_fallback_groups", ctypes.c_uint64),
                ("blocks", ctypes.c_uint64), ("max_rounds", ctypes.c_uint64),
                ("cycles_tables", ctypes.c_uint64), ("cycles_huffman", ctypes.c_uint64),
                ("cycles_lz77", ctypes.c_uint64), ("detail", ctypes.c_uint64 * 8),
                ("round_bytes", ctypes.c_uint64 * 8), ("round_groups", ctypes.c_uint64 * 8)]


def _declare(L):
    vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    P = ctypes.POINTER
    L.gmp_stream_info_parse.argtypes = [vp, sz, P(StreamInfo)]
    L.gmp_index_build.argtypes = [vp, sz, P(BlockRef), sz, P(sz), P(StreamInfo)]
    L.gmp_compress_opts_default.argtypes = [P(CompressOpts)]
    L.gmp_compress_opts_default.restype = None
    L.gmp_compress_bound.argtypes = [sz, P(CompressOpts)]
    L.gmp_compress_bound.restype = sz
    L.gmp_compress.argtypes = [vp, sz, P(CompressOpts), vp, sz, P(sz)]
    L.gmp_encode_tokens.argtypes = [vp, vp, vp, sz, vp, sz, P(CompressOpts), vp, sz, P(sz)]
    L.gmp_compress_gpu.argtypes = [i32, vp, sz, P(CompressOpts), vp, sz, P(sz)]
    L.gmp_compress_gpu_last_times.argtypes = [P(GpuCompressTimes)]
    L.gmp_compress_gpu_last_times.restype = None
    L.gmp_context_opts_default.argtypes = [P(ContextOpts)]
    L.gmp_context_opts_default.restype = None
    L.gmp_context_create.argtypes = [P(vp), i32, P(ContextOpts)]
    L.gmp_context_destroy.argtypes = [vp]
    L.gmp_context_destroy.restype = None
    L.gmp_context_set_launch.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
    L.gmp_context_set_input_wait.argtypes = [vp, ctypes.c_uint32]
    L.gmp_context_debug_drop_input_flag.argtypes = [vp, ctypes.c_int64]
    L.gmp_context_scratch_bytes.argtypes = [vp]
    L.gmp_context_scratch_bytes.restype = sz
    L.gmp_decompress.argtypes = [vp, vp, sz, vp, sz, vp, sz, vp, vp]
    L.gmp_decompress_batch.argtypes = [vp, vp, sz, vp, vp]
    L.gmp_batch_graph_create.argtypes = [vp, vp, sz, vp, vp, P(vp)]
    L.gmp_graph_launch.argtypes = [vp, vp]
    L.gmp_graph_destroy.argtypes = [vp]
    L.gmp_graph_destroy.restype = None
    L.gmp_autotune.argtypes = [vp, vp, sz, vp, vp, P(Tuning)]
    L.gmp_stats_reset.argtypes = [vp, vp]
    L.gmp_stats_read.argtypes = [vp, P(Stats)]
    L.gmp_decompress_host.argtypes = [vp, vp, sz, vp, sz, P(ctypes.c_int32), vp]
    L.gmp_decompress_host_batch.argtypes = [vp, sz, vp, vp, vp, vp, vp, vp]
    L.gmp_decompress_from_host_batch.argtypes = [vp, sz, vp, vp, vp, vp, vp, vp]
    L.gmp_server_opts_default.argtypes = [P(ServerOpts)]
    L.gmp_server_opts_default.restype = None
    L.gmp_server_create.argtypes = [P(vp), i32, P(ServerOpts)]
    L.gmp_server_submit.argtypes = [vp, vp, sz, P(ctypes.c_uint64)]
    L.gmp_server_poll.argtypes = [vp, P(Completion), sz, P(sz), i32]
    L.gmp_server_release.argtypes = [vp, ctypes.c_uint64]
    L.gmp_server_drain.argtypes = [vp]
    L.gmp_server_copy_out.argtypes = [vp, ctypes.c_uint64, vp, sz, i32]
    L.gmp_server_now.argtypes = [vp]
    L.gmp_server_now.restype = ctypes.c_double
    L.gmp_server_bytes_in_use.argtypes = [vp]
    L.gmp_server_bytes_in_use.restype = ctypes.c_uint64
    L.gmp_server_destroy.argtypes = [vp]
    L.gmp_server_destroy.restype = None
    L.gmp_decompress_noalloc.argtypes = [vp, sz, vp, sz, ctypes.c_uint32, vp, sz, vp, vp]
    L.gmp_noalloc_limits.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint64)]
    L.gmp_noalloc_limits.restype = None
    L.gmp_kernel_arch.argtypes = [P(ctypes.c_int), P(ctypes.c_int)]
    L.gmp_last_cuda_error.argtypes = []
    L.gmp_last_cuda_error.restype = ctypes.c_char_p


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libgmp.so is not built (run __graft_entry__.build() or "
                                   "paper_1606_00519_gb300._native.build()); there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib
