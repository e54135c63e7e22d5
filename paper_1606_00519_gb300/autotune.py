"""Autotuning of the decode path.

Two kinds of parameters decide decode speed:

* the launch shape (warps per CTA, CTAs per SM) of the persistent decode
  kernel: ``Context.autotune`` (native ``gmp_autotune``) times a sample batch
  under each shape and keeps the fastest;
* the stream format's block size and sub-blocks per block, which the
  compressor fixes: ``tune_format`` compresses a sample under each candidate,
  decodes it on the GPU, and picks the fastest whose compression ratio stays
  within ``max_ratio_loss`` of the best (smaller blocks and more sub-blocks
  give more parallelism and less compression, Sec. 3.1 and Sec. 5.3 of the
  paper).

``tune`` runs both and caches the result in a JSON file keyed by the GPU
name and a digest of the sample, so a later process reuses it.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

KiB = 1 << 10


def _gpu_key(device: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|sm{p.multi_processor_count}"


def _time_decode(gmp, ds, ctx, repeats: int) -> float:
    """Mean seconds of one decode of `ds`, timed with CUDA events."""
    import torch
    out = torch.empty(max(ds.orig_size, 16), dtype=torch.uint8, device=ds.comp.device)
    st = torch.zeros(1, dtype=torch.int32, device=ds.comp.device)
    ctx.decompress_into(ds, out, st)
    torch.cuda.synchronize()
    if int(st.item()) != 0:
        raise RuntimeError("autotune: sample did not decode")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(repeats):
        ctx.decompress_into(ds, out, st)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / repeats


def tune_format(sample, block_sizes=(64 * KiB, 128 * KiB, 256 * KiB), n_subs=(16, 32, 64), window: int = 32 * KiB,
                de: bool = True, max_ratio_loss: float = 0.02, repeats: int = 5, device: int | None = None) -> dict:
    """Block size and sub-block count for streams like `sample`: the fastest
    GPU decode among the candidates whose ratio is within max_ratio_loss of
    the best candidate's ratio."""
    import torch

    import paper_1606_00519_gb300 as gmp
    dev = torch.cuda.current_device() if device is None else device
    data = np.ascontiguousarray(sample, dtype=np.uint8)
    rows = []
    for bs in block_sizes:
        ctx = gmp.Context(device=dev, max_block_out=bs)
        for k in n_subs:
            stream = gmp.compress(data, bs, k, min(window, 32768), de=de)
            ds = gmp.DeviceStream(stream, device=f"cuda:{dev}")
            sec = _time_decode(gmp, ds, ctx, repeats)
            rows.append({"block_size": bs, "n_sub": k, "ratio": data.size / stream.size,
                         "gbs": data.size / sec / 1e9})
        ctx.close()
    best_ratio = max(r["ratio"] for r in rows)
    ok = [r for r in rows if r["ratio"] >= (1.0 - max_ratio_loss) * best_ratio]
    pick = max(ok, key=lambda r: r["gbs"])
    return {**pick, "candidates": rows}


def tune(sample, cache_path: str | None = None, device: int | None = None, **kw) -> dict:
    """tune_format plus the launch shape for the chosen format, cached."""
    import torch

    import paper_1606_00519_gb300 as gmp
    dev = torch.cuda.current_device() if device is None else device
    data = np.ascontiguousarray(sample, dtype=np.uint8)
    digest = hashlib.sha1(data.tobytes()).hexdigest()[:16]
    key = f"{_gpu_key(dev)}|{digest}|{json.dumps(kw, sort_keys=True)}"
    path = cache_path or os.environ.get("GMP_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "gmp_tune.json")
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        return {**cache[key], "cached": True}
    t0 = time.perf_counter()
    fmt = tune_format(data, device=dev, **kw)
    stream = gmp.compress(data, fmt["block_size"], fmt["n_sub"], 32 * KiB, de=kw.get("de", True))
    ds = gmp.DeviceStream(stream, device=f"cuda:{dev}")
    out = torch.empty(max(ds.orig_size, 16), dtype=torch.uint8, device=f"cuda:{dev}")
    table = gmp.make_file_table([ds.file_desc(out)], device=f"cuda:{dev}")
    status = torch.zeros(1, dtype=torch.int32, device=f"cuda:{dev}")
    ctx = gmp.Context(device=dev, max_block_out=fmt["block_size"])
    shape = ctx.autotune(table, 1, status)
    ctx.close()
    res = {"block_size": fmt["block_size"], "n_sub": fmt["n_sub"], "ratio": fmt["ratio"], "gbs": fmt["gbs"],
           "warps_per_cta": shape["warps_per_cta"], "ctas_per_sm": shape["ctas_per_sm"],
           "tune_seconds": time.perf_counter() - t0}
    cache[key] = res
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return {**res, "cached": False}
