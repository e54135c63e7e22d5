"""GB300-native Gompresso-style decompression (arXiv:1606.00519).

Thin Python binding over libgmp.so (C ABI in include/gmp.h): argument
marshalling only.  Every decoding step runs in the library's CUDA kernels;
PyTorch provides device memory and streams.  There is no CPU fallback: if the
library is not built or no GPU is present, the decode calls raise.

Typical use::

    import paper_1606_00519_gb300 as gmp
    stream = gmp.compress(data, block_size=256 << 10, n_sub=32, window=32768, de=True)
    dev = gmp.DeviceStream(stream)               # stream + block index on the GPU
    ctx = gmp.Context()
    out, status = ctx.decompress(dev)            # torch.uint8 CUDA tensor
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native
from ._native import (BlockRef, Completion, CompressOpts, ContextOpts, FileDesc, ServerOpts, Stats, StreamInfo,
                      Tuning)

OK = 0
RESOLVE = {"auto": 0, "mrr": 1, "sc": 2}
STATUS_NAMES = {0: "OK", 1: "BAD_HEADER", 2: "CORRUPT_SYMBOL", 3: "BITSTREAM", 4: "BAD_OFFSET",
                5: "OUTPUT_OVERRUN", 6: "MRR_NO_PROGRESS", 7: "CAPACITY", 8: "INPUT_TIMEOUT"}
ERROR_NAMES = {-1: "INVALID_ARG", -2: "CAPACITY", -3: "CUDA", -4: "UNSUPPORTED", -5: "FORMAT", -6: "NOMEM"}


class GmpError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {ERROR_NAMES.get(code, code)}"
        if code == -3:
            msg += f" ({_native.lib().gmp_last_cuda_error().decode()})"
        super().__init__(msg)


def _check(rc: int, what: str):
    if rc != 0:
        raise GmpError(rc, what)


def _np_bytes(x) -> np.ndarray:
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x.reshape(-1).view(np.uint8))
    return np.frombuffer(bytes(x), dtype=np.uint8)


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _torch():
    import torch
    return torch


def _stream_handle(stream) -> ctypes.c_void_p:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


# --------------------------------------------------------------------------
# host side: compressor, header, block index

def compress(data, block_size: int = 256 << 10, n_sub: int = 32, window: int = 32768, cwl: int = 12,
             max_match: int = 64, chain_depth: int = 64, de: bool = False, n_threads: int = 0,
             lazy: bool = True, byte_mode: bool = False) -> np.ndarray:
    """Compress host bytes into the stream format of include/gmp.h (host,
    multi-threaded over blocks).  byte_mode: byte-level blocks (Gompresso/Byte,
    no Huffman coding; n_sub and cwl do not apply)."""
    L = _native.lib()
    src = _np_bytes(data)
    o = CompressOpts(block_size, n_sub, window, cwl, max_match, chain_depth, 1 if de else 0, n_threads,
                     1 if lazy else 0, 1 if byte_mode else 0)
    cap = L.gmp_compress_bound(src.size, ctypes.byref(o))
    out = np.empty(cap, np.uint8)
    n = ctypes.c_size_t()
    _check(L.gmp_compress(_ptr(src) if src.size else None, src.size, ctypes.byref(o), _ptr(out), cap,
                          ctypes.byref(n)), "gmp_compress")
    return out[:n.value]


def compress_gpu(data, block_size: int = 256 << 10, n_sub: int = 32, window: int = 32768, cwl: int = 12,
                 max_match: int = 64, de: bool = False, n_threads: int = 0, lazy: bool = True,
                 byte_mode: bool = False, device: int | None = None, chain_depth: int = 64) -> np.ndarray:
    """Compress host bytes on the GPU (gmp_compress_gpu: match search, parse
    and entropy coding on the device): same stream format as compress()."""
    L = _native.lib()
    src = _np_bytes(data)
    if device is None:
        device = _torch().cuda.current_device() if _torch().cuda.is_available() else 0
    o = CompressOpts(block_size, n_sub, window, cwl, max_match, chain_depth, 1 if de else 0, n_threads,
                     1 if lazy else 0, 1 if byte_mode else 0)
    cap = L.gmp_compress_bound(src.size, ctypes.byref(o))
    out = np.empty(cap, np.uint8)
    n = ctypes.c_size_t()
    _check(L.gmp_compress_gpu(device, _ptr(src) if src.size else None, src.size, ctypes.byref(o), _ptr(out), cap,
                              ctypes.byref(n)), "gmp_compress_gpu")
    return out[:n.value]


def compress_gpu_times() -> dict:
    """Device times (ms) of this thread's last compress_gpu call: match
    search, parse and entropy coding."""
    t = _native.GpuCompressTimes()
    _native.lib().gmp_compress_gpu_last_times(ctypes.byref(t))
    return {"match_ms": t.match_ms, "parse_ms": t.parse_ms, "encode_ms": t.encode_ms,
            "compressed_bytes": int(t.compressed_bytes)}


def encode_tokens(lit_len, match_len, dist, lits, block_size: int | None = None, n_sub: int = 32,
                  window: int = 32768, cwl: int = 12, max_match: int = 64, de: bool = False,
                  byte_mode: bool = False) -> np.ndarray:
    """One-block stream of the given LZ77 parse (sequence i: lit_len[i]
    literals from lits, then match_len[i] bytes at distance dist[i]).
    block_size defaults to the parse's output size."""
    L = _native.lib()
    ll = np.ascontiguousarray(lit_len, np.uint32)
    ml = np.ascontiguousarray(match_len, np.uint32)
    di = np.ascontiguousarray(dist, np.uint32)
    lt = _np_bytes(lits)
    total = int(ll.sum(dtype=np.int64) + ml.sum(dtype=np.int64))
    o = CompressOpts(block_size or max(total, 1), n_sub, window, cwl, max_match, 64, 1 if de else 0, 0, 1,
                     1 if byte_mode else 0)
    cap = 2 * lt.size + 5 * ll.size + 1280
    out = np.empty(cap, np.uint8)
    n = ctypes.c_size_t()
    _check(L.gmp_encode_tokens(_ptr(ll) if ll.size else None, _ptr(ml) if ml.size else None,
                               _ptr(di) if di.size else None, ll.size, _ptr(lt) if lt.size else None, lt.size,
                               ctypes.byref(o), _ptr(out), cap, ctypes.byref(n)), "gmp_encode_tokens")
    return out[:n.value]


def stream_info(stream) -> StreamInfo:
    s = _np_bytes(stream)
    info = StreamInfo()
    _check(_native.lib().gmp_stream_info_parse(_ptr(s), s.size, ctypes.byref(info)), "gmp_stream_info_parse")
    return info


def index_build(stream):
    """(index as an (n_blocks, 4) uint64 array, StreamInfo)."""
    L = _native.lib()
    s = _np_bytes(stream)
    n = ctypes.c_size_t()
    info = StreamInfo()
    _check(L.gmp_index_build(_ptr(s), s.size, None, 0, ctypes.byref(n), ctypes.byref(info)), "gmp_index_build")
    idx = np.zeros((max(n.value, 1), 4), np.uint64)
    _check(L.gmp_index_build(_ptr(s), s.size, idx.ctypes.data_as(ctypes.POINTER(BlockRef)), n.value,
                             ctypes.byref(n), ctypes.byref(info)), "gmp_index_build")
    return idx[:n.value], info


@dataclass
class DeviceStream:
    """A compressed stream and its block index resident on the GPU."""
    comp: object          # torch.uint8 CUDA tensor (16-byte aligned)
    index: object         # torch.uint64-as-int64 CUDA tensor, (n_blocks, 4)
    info: StreamInfo
    n_blocks: int
    comp_bytes: int

    def __init__(self, stream, device=None):
        torch = _torch()
        s = _np_bytes(stream)
        idx, info = index_build(s)
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.comp = torch.from_numpy(s.copy()).to(dev)
        self.index = torch.from_numpy(idx.view(np.int64).copy()).to(dev)
        self.info = info
        self.n_blocks = int(idx.shape[0])
        self.comp_bytes = int(s.size)

    @property
    def orig_size(self) -> int:
        return int(self.info.orig_size)

    def file_desc(self, out, out_cap: int | None = None) -> FileDesc:
        return FileDesc(self.comp.data_ptr(), self.comp_bytes, self.index.data_ptr(), self.n_blocks,
                        out.data_ptr(), out.numel() if out_cap is None else out_cap)


class Context:
    """A decoder context (scratch for one persistent launch) on one device."""

    def __init__(self, device: int | None = None, max_block_out: int = 256 << 10, warps_per_cta: int = 0,
                 ctas_per_sm: int = 0, collect_stats: bool = False, max_files: int = 65536, resolve: str = "auto",
                 concurrent: bool = False):
        """resolve: "auto" (DE streams in one pass, others by MRR), "mrr" (MRR
        always) or "sc" (sequential copying, the paper's baseline).
        concurrent: the context's launches run beside other kernels (warps take
        every block from the work counter instead of a fixed first block)."""
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the decoder runs only on the GPU")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._L = _native.lib()
        o = ContextOpts(max_block_out, warps_per_cta, ctas_per_sm, 1 if collect_stats else 0, max_files,
                        RESOLVE[resolve], 1 if concurrent else 0)
        h = ctypes.c_void_p()
        _check(self._L.gmp_context_create(ctypes.byref(h), self.device, ctypes.byref(o)), "gmp_context_create")
        self._h = h
        self.max_block_out = max_block_out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.gmp_context_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def set_launch(self, warps_per_cta: int, ctas_per_sm: int = 0):
        _check(self._L.gmp_context_set_launch(self._h, warps_per_cta, ctas_per_sm), "gmp_context_set_launch")

    def set_input_wait(self, ms: int):
        """Host-to-host calls: a warp's wait limit for a piece's input (ms;
        0 = the default 10 s)."""
        _check(self._L.gmp_context_set_input_wait(self._h, ms), "gmp_context_set_input_wait")

    def debug_drop_input_flag(self, piece: int):
        """Test hook: the next host-to-host call does not flag piece
        `piece`'s input (its waits run out; -1 clears)."""
        _check(self._L.gmp_context_debug_drop_input_flag(self._h, piece), "gmp_context_debug_drop_input_flag")

    def scratch_bytes(self) -> int:
        return int(self._L.gmp_context_scratch_bytes(self._h))

    def decompress_into(self, ds: DeviceStream, out, status, stream=None):
        """Asynchronous decode of `ds` into the uint8 CUDA tensor `out`;
        `status` is an int32 CUDA tensor of >= 1 element."""
        _check(self._L.gmp_decompress(self._h, ctypes.c_void_p(ds.comp.data_ptr()), ds.comp_bytes,
                                      ctypes.c_void_p(ds.index.data_ptr()), ds.n_blocks,
                                      ctypes.c_void_p(out.data_ptr()), out.numel(),
                                      ctypes.c_void_p(status.data_ptr()), _stream_handle(stream)),
               "gmp_decompress")

    def decompress(self, ds: DeviceStream, stream=None):
        """Decode into a new CUDA tensor; returns (out, status) where status is
        read after synchronising the stream."""
        torch = _torch()
        out = torch.empty(max(ds.orig_size, 16), dtype=torch.uint8, device=ds.comp.device)
        st = torch.zeros(1, dtype=torch.int32, device=ds.comp.device)
        self.decompress_into(ds, out, st, stream)
        status = int(st.item())
        return out[:ds.orig_size], status

    def decompress_batch(self, files_dev, n_files: int, status, stream=None):
        """files_dev: CUDA tensor holding n_files FileDesc records (see
        make_file_table); status: int32 CUDA tensor of n_files."""
        _check(self._L.gmp_decompress_batch(self._h, ctypes.c_void_p(files_dev.data_ptr()), n_files,
                                            ctypes.c_void_p(status.data_ptr()), _stream_handle(stream)),
               "gmp_decompress_batch")

    def batch_graph(self, files_dev, n_files: int, status) -> "Graph":
        g = ctypes.c_void_p()
        _check(self._L.gmp_batch_graph_create(self._h, ctypes.c_void_p(files_dev.data_ptr()), n_files,
                                              ctypes.c_void_p(status.data_ptr()), None, ctypes.byref(g)),
               "gmp_batch_graph_create")
        return Graph(self._L, g)

    def autotune(self, files_dev, n_files: int, status, stream=None) -> dict:
        """Time the batched decode of a sample under several launch shapes
        (gmp_autotune) and keep the fastest; returns the chosen shape."""
        t = Tuning()
        _check(self._L.gmp_autotune(self._h, ctypes.c_void_p(files_dev.data_ptr()), n_files,
                                    ctypes.c_void_p(status.data_ptr()), _stream_handle(stream), ctypes.byref(t)),
               "gmp_autotune")
        return {"warps_per_cta": t.warps_per_cta, "ctas_per_sm": t.ctas_per_sm, "best_ms": t.best_ms,
                "shapes_tried": t.shapes_tried}

    def stats_reset(self, stream=None):
        _check(self._L.gmp_stats_reset(self._h, _stream_handle(stream)), "gmp_stats_reset")

    def stats(self) -> dict:
        s = Stats()
        _check(self._L.gmp_stats_read(self._h, ctypes.byref(s)), "gmp_stats_read")
        arrays = ("detail", "round_bytes", "round_groups")
        d = {k: int(getattr(s, k)) for k, _ in Stats._fields_ if k not in arrays}
        for k in arrays:
            d[k] = [int(x) for x in getattr(s, k)]
        return d

    def decompress_host_batch(self, streams, outs=None, cuda_stream=None):
        """Host streams in, host bytes out: one pipelined call (input copies,
        decoding and copies back overlap; pinned buffers overlap best).
        Returns (outputs, statuses)."""
        ss = [_np_bytes(x) for x in streams]
        infos = [stream_info(x) for x in ss]
        if outs is None:
            outs = [np.empty(max(i.orig_size, 1), np.uint8) for i in infos]
        n = len(ss)
        ins = (ctypes.c_void_p * n)(*[x.ctypes.data for x in ss])
        sizes = (ctypes.c_size_t * n)(*[x.size for x in ss])
        optr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
        caps = (ctypes.c_size_t * n)(*[o.size for o in outs])
        st = (ctypes.c_int32 * n)()
        _check(self._L.gmp_decompress_host_batch(self._h, n, ins, sizes, optr, caps, st,
                                                 _stream_handle(cuda_stream)), "gmp_decompress_host_batch")
        return [o[:i.orig_size] for o, i in zip(outs, infos)], [int(x) for x in st]

    def decompress_from_host_batch(self, streams, outs=None, cuda_stream=None):
        """Host streams in, device bytes out (the paper's "(In)" mode): one
        pipelined call whose input copies overlap the decoding; outs are uint8
        CUDA tensors (allocated when None).  Returns (outputs, statuses)."""
        torch = _torch()
        ss = [_np_bytes(x) for x in streams]
        infos = [stream_info(x) for x in ss]
        if outs is None:
            outs = [torch.empty(max(i.orig_size, 1), dtype=torch.uint8, device=f"cuda:{self.device}") for i in infos]
        n = len(ss)
        ins = (ctypes.c_void_p * n)(*[x.ctypes.data for x in ss])
        sizes = (ctypes.c_size_t * n)(*[x.size for x in ss])
        optr = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        caps = (ctypes.c_size_t * n)(*[o.numel() for o in outs])
        st = (ctypes.c_int32 * n)()
        _check(self._L.gmp_decompress_from_host_batch(self._h, n, ins, sizes, optr, caps, st,
                                                      _stream_handle(cuda_stream)), "gmp_decompress_from_host_batch")
        return [o[:i.orig_size] for o, i in zip(outs, infos)], [int(x) for x in st]

    def decompress_host(self, stream, out: np.ndarray | None = None, cuda_stream=None):
        """Host stream in, host bytes out (H2D + decode + D2H, pipelined,
        synchronous)."""
        s = _np_bytes(stream)
        info = stream_info(s)
        if out is None:
            out = np.empty(max(info.orig_size, 1), np.uint8)
        st = ctypes.c_int32()
        _check(self._L.gmp_decompress_host(self._h, _ptr(s), s.size, _ptr(out), out.size, ctypes.byref(st),
                                           _stream_handle(cuda_stream)), "gmp_decompress_host")
        return out[:info.orig_size], st.value


class Graph:
    def __init__(self, L, h):
        self._L = L
        self._h = h

    def launch(self, stream=None):
        _check(self._L.gmp_graph_launch(self._h, _stream_handle(stream)), "gmp_graph_launch")

    def close(self):
        if self._h and self._h.value:
            self._L.gmp_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_file_table(descs, device=None):
    """Pack FileDesc records into a CUDA tensor for the batched calls."""
    torch = _torch()
    arr = (FileDesc * len(descs))(*descs)
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
    dev = torch.device("cuda") if device is None else torch.device(device)
    return torch.from_numpy(raw).to(dev)


class Server:
    """Continuous-batching decompression server (gmp_server_* in the C ABI).

    submit() takes a compressed stream in host memory (a numpy uint8 array,
    ideally pinned); the array is kept alive here until its request is
    released.  poll() returns completions as dicts with the request id,
    status, output size and the submit / launch / done timestamps."""

    def __init__(self, device: int | None = None, budget_bytes: int = 32 << 30, n_lanes: int = 8,
                 max_batch: int = 64, max_block_out: int = 256 << 10, warps_per_cta: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the server decodes only on the GPU")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._L = _native.lib()
        o = ServerOpts(budget_bytes, n_lanes, max_batch, max_block_out, warps_per_cta)
        h = ctypes.c_void_p()
        _check(self._L.gmp_server_create(ctypes.byref(h), self.device, ctypes.byref(o)), "gmp_server_create")
        self._h = h
        self._keep = {}

    def submit(self, stream) -> int:
        s = stream if isinstance(stream, np.ndarray) else _np_bytes(stream)
        rid = ctypes.c_uint64()
        _check(self._L.gmp_server_submit(self._h, _ptr(s), s.size, ctypes.byref(rid)), "gmp_server_submit")
        self._keep[rid.value] = s
        return rid.value

    def poll(self, max_n: int = 4096, wait_ms: int = 0) -> list:
        buf = (Completion * max_n)()
        n = ctypes.c_size_t()
        _check(self._L.gmp_server_poll(self._h, buf, max_n, ctypes.byref(n), wait_ms), "gmp_server_poll")
        return [{"id": buf[i].id, "status": buf[i].status, "out_bytes": buf[i].out_bytes,
                 "t_submit": buf[i].t_submit, "t_start": buf[i].t_start, "t_done": buf[i].t_done,
                 "t_gpu_ready": buf[i].t_gpu_ready, "t_gpu_done": buf[i].t_gpu_done}
                for i in range(n.value)]

    def copy_out(self, rid: int, dst) -> None:
        """Copy a completed request's output into a numpy array or a CUDA tensor."""
        if isinstance(dst, np.ndarray):
            _check(self._L.gmp_server_copy_out(self._h, rid, _ptr(dst), dst.size, 0), "gmp_server_copy_out")
        else:
            _check(self._L.gmp_server_copy_out(self._h, rid, ctypes.c_void_p(dst.data_ptr()), dst.numel(), 1),
                   "gmp_server_copy_out")

    def release(self, rid: int) -> None:
        _check(self._L.gmp_server_release(self._h, rid), "gmp_server_release")
        self._keep.pop(rid, None)

    def drain(self) -> None:
        _check(self._L.gmp_server_drain(self._h), "gmp_server_drain")

    def now(self) -> float:
        return float(self._L.gmp_server_now(self._h))

    def bytes_in_use(self) -> int:
        return int(self._L.gmp_server_bytes_in_use(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.gmp_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
