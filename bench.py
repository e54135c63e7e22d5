#!/usr/bin/env python3
"""Decompression benchmark (decompressed GB/s, fraction of the HBM roofline).

One step = one pass of the whole decode path over the workload: Huffman
decoding of every sub-block, then LZ77 resolution of every block, for the
workload's MRR stream and its DE stream, in one persistent launch of the
batched decoder.  The default workload is the 1 GiB configuration: CSV-like
numeric records (csv1g), 256 KiB blocks of 32 sub-blocks, compressed once in
MRR and once in DE mode.  Inputs (compressed streams and block indexes) are
resident in device memory before the timed region; the decompressed output
(2 x 1 GiB) is larger than L2, so no flush is needed.

The same JSON line carries, for one GPU, sub-objects for the other
configurations: ``text256m`` (256 MiB Markov text, MRR + DE), ``batch_1gib``
(the seeded 1 GiB cut of the 4096-file mix in one CUDA-graph launch, against
one launch per file) and ``serving`` (Poisson arrivals under a 32 GiB budget:
closed-loop peak, p50/p99 at 25/50/90 % of it, against one call per request).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (the
slow, obviously correct serial decoder) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import datagen  # noqa: E402

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("gmp_decode.cu", "gmp_internal.h"):
        with open(os.path.join(ROOT, "paper_1606_00519_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_per_unit(fmt: str = "bit", workload: str = "csv1g"):
    """DRAM bytes per decompressed byte of the decode kernel from the committed
    ncu summary of the workload and stream format, if it was taken on the
    current kernel source."""
    name = f"decode_kernel_traffic_{workload}" + ("" if fmt == "bit" else f"_{fmt}") + ".json"
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            t = json.load(f)
        if t.get("kernel_source_sha256_16") == _kernel_source_hash():
            return float(t["dram_bytes_per_output_byte"]), t
    except Exception:
        pass
    return None, None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 20):
        self.proc = None
        # raw samples (the JSON line carries their summary)
        out_dir = os.environ.get("GMP_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", f"-lms", str(period_ms)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s, p in zip(sm, pw)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


def _dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return rank, world, local, dist
    return rank, world, local, None


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_workload(name: str, size: int | None = None, fmt: str = "bit"):
    """(workload, data, {mode: stream}) using the product compressor; fmt
    "bit" writes Huffman blocks (Gompresso/Bit), "byte" byte-level blocks
    (Gompresso/Byte)."""
    import paper_1606_00519_gb300 as gmp
    w = datagen.WORKLOADS[name]
    data = w.data(size)
    streams = {}
    for mode in ("mrr", "de"):
        streams[mode] = gmp.compress(data, w.block_size, w.n_sub, w.window, de=(mode == "de"),
                                     byte_mode=(fmt == "byte"))
    return w, data, streams


def cpu_oracle_sample(streams, budget_s: float, max_blocks: int | None = None):
    """Time the oracle's serial decoder on a bounded sample of blocks (taken
    round-robin from the streams, from the start).  Returns (bytes, seconds,
    description)."""
    import oracle
    infos = {m: oracle.stream_info(s) for m, s in streams.items()}
    done_bytes, t0, nblk = 0, time.perf_counter(), 0
    b = 0
    while True:
        progressed = False
        for m, s in streams.items():
            if b < infos[m].n_blocks:
                out = oracle.decompress_block(s, b)
                done_bytes += out.size
                nblk += 1
                progressed = True
        b += 1
        el = time.perf_counter() - t0
        if not progressed or el >= budget_s or (max_blocks and nblk >= max_blocks):
            break
    el = time.perf_counter() - t0
    desc = f"first {b} blocks of each of the {len(streams)} streams ({nblk} blocks, {done_bytes} bytes), 1 thread"
    return done_bytes, el, desc


def cpu_oracle_parallel(streams, budget_s: float, threads: int, max_blocks: int | None = None):
    """The oracle's serial block decoder run block-parallel on `threads` host
    threads (blocks are independent, Sec. 3.1; the paper's CPU baselines are
    parallel over blocks the same way).  The oracle's C calls release the
    GIL, so the threads decode concurrently.  Blocks are taken round-robin
    from the streams until the time budget or max_blocks runs out.  Returns
    (bytes, seconds, description)."""
    import threading

    import oracle
    infos = {m: oracle.stream_info(s) for m, s in streams.items()}
    order = []
    for b in range(max(i.n_blocks for i in infos.values())):
        for m in streams:
            if b < infos[m].n_blocks:
                order.append((m, b))
    if max_blocks:
        order = order[:max_blocks]
    lock = threading.Lock()
    state = {"next": 0, "bytes": 0, "blocks": 0}
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                k = state["next"]
                if k >= len(order) or time.perf_counter() - t0 >= budget_s:
                    return
                state["next"] = k + 1
            m, b = order[k]
            n = oracle.decompress_block(streams[m], b).size
            with lock:
                state["bytes"] += n
                state["blocks"] += 1

    ts = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    el = time.perf_counter() - t0
    desc = (f"{state['blocks']} blocks ({state['bytes']} bytes) taken round-robin from the {len(streams)} streams, "
            f"block-parallel on {threads} threads")
    return state["bytes"], el, desc


def _oracle_pool(w, fmt: str, pool_bytes: int, threads: int):
    """Streams for the reference arm, written by the oracle's own compressor
    (no product code on that path): the first pool_bytes of the workload in
    chunks of whole blocks, each chunk compressed as its own stream on a host
    thread (blocks are independent, Sec. 3.1, so the chunks' blocks are the
    blocks of one stream of the whole).  Returns {mode: [stream, ...]}."""
    import threading

    import oracle
    data = w.data(min(w.size, pool_bytes))
    chunk = max(w.block_size, (data.size // (4 * threads)) // w.block_size * w.block_size)
    pieces = [data[i:i + chunk] for i in range(0, data.size, chunk)]
    pool = {}
    for mode in ("mrr", "de"):
        prm = oracle.params(w.block_size, w.n_sub if fmt == "bit" else 1, w.window, de=(mode == "de"),
                            byte_mode=(fmt == "byte"))
        out = [None] * len(pieces)
        nxt = [0]
        lock = threading.Lock()

        def work():
            while True:
                with lock:
                    k = nxt[0]
                    nxt[0] += 1
                if k >= len(pieces):
                    return
                out[k] = oracle.compress(pieces[k], prm)

        ts = [threading.Thread(target=work) for _ in range(threads)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        pool[mode] = out
    return pool, data.size


def run_reference(args):
    """The reference arm: the CPU oracle's serial block decoder, run
    block-parallel on all host cores, on a bounded sample of the workload per
    step (args.ref_blocks blocks per thread)."""
    rank, world, local, dist = _dist_init(args)
    if rank != 0:
        return
    import oracle
    w = datagen.WORKLOADS[args.workload]
    threads = os.cpu_count() or 1
    pool, pool_bytes = _oracle_pool(w, args.format, args.ref_pool, threads)
    streams = {f"{m}{i}": st for m in pool for i, st in enumerate(pool[m])}
    per_step_blocks = args.ref_blocks * threads
    for _ in range(args.warmup):
        cpu_oracle_parallel(streams, 1e9, threads, max_blocks=threads)
    tot_b, tot_t = 0, 0.0
    for _ in range(args.steps):
        nb, el, desc = cpu_oracle_parallel(streams, 1e9, threads, max_blocks=per_step_blocks)
        tot_b += nb
        tot_t += el
    gbs = tot_b / tot_t / 1e9
    comp = sum(st.size for m in pool for st in pool[m])
    sample = (f"per step: {per_step_blocks} blocks ({per_step_blocks * w.block_size} bytes) of a pool of the first "
              f"{pool_bytes} bytes of the workload compressed by the oracle in MRR and DE mode (ratio "
              f"{2 * pool_bytes / comp:.3f}), block-parallel on {threads} threads")
    line = {"impl": "reference", "metric": "decompressed GB/s", "value": gbs, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": _config(w, args.format, world, args.size),
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(w, fmt="bit", world=1, size=None):
    """The workload as both arms describe it (the same keys and values)."""
    size = int(size or w.size)
    if fmt == "byte":
        coding = "Gompresso/Byte (byte-level records, no Huffman)"
    else:
        coding = f"K={w.n_sub} sub-blocks"
    return {"workload": f"{w.name}: {size / MiB:g} MiB {w.kind}, {w.block_size // KiB} KiB blocks, "
                        f"{coding}, {w.window // KiB} KiB window, MRR and DE streams",
            "format": fmt, "bytes_per_stream": size, "block_size": w.block_size,
            "n_sub": w.n_sub if fmt == "bit" else 0, "window": w.window, "cwl": 12 if fmt == "bit" else 0,
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"}


def measure_decode(args, w, data, streams, dev, dist=None, rank=0, clocks=False, extras=True):
    """Times `args.steps` batched launches decoding the workload's MRR and DE
    streams (one launch per step) after a byte-exact check; returns the
    figures of the JSON line.  extras: per-stream rates and the statistics
    launch with the cycle split of the decode kernel."""
    import torch
    import paper_1606_00519_gb300 as gmp

    local = dev.index or 0
    modes = ["mrr", "de"]
    ds = {m: gmp.DeviceStream(streams[m], device=dev) for m in modes}
    outs = {m: torch.empty(data.size, dtype=torch.uint8, device=dev) for m in modes}
    ctx = gmp.Context(device=local, max_block_out=w.block_size, warps_per_cta=args.warps_per_cta,
                      ctas_per_sm=args.ctas_per_sm, collect_stats=False)
    table = gmp.make_file_table([ds[m].file_desc(outs[m]) for m in modes], device=dev)
    status = torch.zeros(len(modes), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # launch shape for this workload from the autotuner (outside the timed
    # region), unless fixed on the command line
    tuned = None
    if not args.warps_per_cta:
        tuned = ctx.autotune(table, len(modes), status, stream)
    shape = {"warps_per_cta": tuned["warps_per_cta"] if tuned else args.warps_per_cta,
             "ctas_per_sm": tuned["ctas_per_sm"] if tuned else args.ctas_per_sm, "autotuned": tuned is not None}
    out_bytes = data.size * len(modes)
    comp_bytes = sum(ds[m].comp_bytes for m in modes)

    def step():
        ctx.decompress_batch(table, len(modes), status, stream)

    # correctness of the timed configuration (byte-exact against the input)
    for o in outs.values():
        o.fill_(0xA5)
    step()
    torch.cuda.synchronize()
    ref = torch.from_numpy(data).to(dev)
    st = status.cpu().numpy()
    ok = bool(np.all(st == 0)) and all(bool(torch.equal(outs[m], ref)) for m in modes)
    del ref
    if not ok:
        raise SystemExit(f"bench: {w.name} decoded output is not byte-exact (status {st.tolist()})")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if clocks else None
    _barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launch_ev = []
    ev0.record(stream)
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        launch_ev.append((a, b))
    ev1.record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    el_ms = ev0.elapsed_time(ev1)
    per_launch = [a.elapsed_time(b) for a, b in launch_ev]
    clk = sampler.stop() if sampler else None
    el_ms = _max_over_ranks(dist, el_ms)
    total_bytes = _sum_over_ranks(dist, float(out_bytes * args.steps))
    value = total_bytes / (el_ms / 1e3) / 1e9

    hbm_peak, peak_kind = _peaks()
    launch_avg_ms = float(np.mean(per_launch))
    algo_bytes = comp_bytes + out_bytes  # compressed read + decompressed written
    achieved = algo_bytes / (launch_avg_ms / 1e3) / 1e9
    tpu, _ = _traffic_per_unit(args.format, w.name)
    res = {
        "value": round(value, 3), "ms_per_step": round(el_ms / args.steps, 4), "unit": "GB/s",
        "launch_shape": shape,
        "streams": {"ratio_mrr": round(data.size / streams["mrr"].size, 4),
                    "ratio_de": round(data.size / streams["de"].size, 4), "compressed_bytes": int(comp_bytes),
                    "compressor": "gmp_compress (host, lazy parse)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "peak_kind": peak_kind,
                     "traffic": (round(tpu * out_bytes) if tpu else None),
                     "kernel": "gmp::decode_kernel (persistent; one launch per step)",
                     "algorithmic_bytes_per_launch": int(algo_bytes),
                     "launch_avg_ms": round(launch_avg_ms, 4),
                     "launch_median_ms": round(float(np.median(per_launch)), 4),
                     "launch_min_ms": round(float(np.min(per_launch)), 4),
                     "decompressed_frac_of_roofline": round(value / (hbm_peak * (out_bytes / algo_bytes)), 4)},
        "clocks": clk,
    }
    if extras:
        # per-mode throughput (each stream in its own launch), for context
        per_mode = {}
        for m in modes:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st1 = torch.zeros(1, dtype=torch.int32, device=dev)
            ctx.decompress_into(ds[m], outs[m], st1, stream)
            torch.cuda.synchronize()
            a.record(stream)
            reps = max(3, args.steps // 2)
            for _ in range(reps):
                ctx.decompress_into(ds[m], outs[m], st1, stream)
            b.record(stream)
            torch.cuda.synchronize()
            per_mode[m] = round(data.size * reps / (a.elapsed_time(b) / 1e3) / 1e9, 2)
        res["per_mode_gbs"] = per_mode
        # where the decode kernel spends its cycles (one extra launch with the
        # per-phase clock counters on, outside the timed region)
        sctx = gmp.Context(device=local, max_block_out=w.block_size, warps_per_cta=shape["warps_per_cta"],
                           ctas_per_sm=shape["ctas_per_sm"], collect_stats=True)
        sctx.stats_reset(stream)
        sctx.decompress_batch(table, len(modes), status, stream)
        torch.cuda.synchronize()
        phase = sctx.stats()
        sctx.close()
        cyc = phase["cycles_tables"] + phase["cycles_huffman"] + phase["cycles_lz77"]
        res["decode_kernel_cycles"] = {
            "tables": round(phase["cycles_tables"] / max(cyc, 1), 4),
            "huffman": round(phase["cycles_huffman"] / max(cyc, 1), 4),
            "lz77": round(phase["cycles_lz77"] / max(cyc, 1), 4),
            "cycles_per_block": round(cyc / max(phase["blocks"], 1)),
            "mrr_rounds_per_group": round(phase["rounds"] / max(phase["groups"], 1), 3),
            "max_rounds": phase["max_rounds"], "de_fallback_groups": phase["de_fallback_groups"]}
    ctx.close()
    return res, (ds, outs, comp_bytes, out_bytes)


def run_gmp(args):
    import torch
    import paper_1606_00519_gb300 as gmp

    rank, world, local, dist = _dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, data, streams = make_workload(args.workload, args.size, args.format)
    res, (ds, outs, comp_bytes, out_bytes) = measure_decode(args, w, data, streams, dev, dist, rank,
                                                            clocks=(rank == 0))
    modes = ["mrr", "de"]
    stream = torch.cuda.current_stream(dev)

    # end to end through the public host-to-host call: pinned host input,
    # H2D of the compressed streams, decode, D2H of the decompressed bytes,
    # one pipelined call per step for both streams
    e2e_ctx = gmp.Context(device=local, max_block_out=w.block_size,
                          warps_per_cta=res["launch_shape"]["warps_per_cta"],
                          ctas_per_sm=res["launch_shape"]["ctas_per_sm"])
    pin_in = [torch.from_numpy(streams[m].copy()).pin_memory().numpy() for m in modes]
    pin_out = [torch.empty(data.size, dtype=torch.uint8).pin_memory().numpy() for m in modes]
    e2e_ctx.decompress_host_batch(pin_in, pin_out, stream)  # staging allocated outside the timed region
    torch.cuda.synchronize()
    _barrier(dist)
    e2e_steps = max(2, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _, stv = e2e_ctx.decompress_host_batch(pin_in, pin_out, stream)
        if any(stv):
            raise SystemExit("bench: e2e decode failed")
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(dist, time.perf_counter() - t0)
    e2e_val = _sum_over_ranks(dist, float(out_bytes * e2e_steps)) / e2e_s / 1e9
    if not all(np.array_equal(o, data) for o in pin_out):
        raise SystemExit("bench: e2e output is not byte-exact")
    del pin_out
    # the paper's "(In)" mode: the same pinned input, H2D overlapped with the
    # decode, the output left in device memory (the outputs of the timed
    # launches are reused)
    dev_out = [outs[m] for m in modes]
    for o in dev_out:
        o.fill_(0x5A)
    e2e_ctx.decompress_from_host_batch(pin_in, dev_out, stream)
    torch.cuda.synchronize()
    _barrier(dist)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _, stv = e2e_ctx.decompress_from_host_batch(pin_in, dev_out, stream)
        if any(stv):
            raise SystemExit("bench: input-only end-to-end decode failed")
    torch.cuda.synchronize()
    in_s = _max_over_ranks(dist, time.perf_counter() - t0)
    in_val = _sum_over_ranks(dist, float(out_bytes * e2e_steps)) / in_s / 1e9
    ref_dev = torch.from_numpy(data).to(dev)
    if not all(torch.equal(o, ref_dev) for o in dev_out):
        raise SystemExit("bench: input-only end-to-end output is not byte-exact")
    del ref_dev, dev_out, pin_in
    e2e_ctx.close()
    del ds, outs
    torch.cuda.empty_cache()

    line = {
        "metric": "decompressed GB/s", "value": res["value"], "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": _config(w, args.format, world, data.size),
        "launch_shape": res["launch_shape"], "streams": res["streams"], "per_mode_gbs": res.get("per_mode_gbs"),
        "decode_kernel_cycles": res.get("decode_kernel_cycles"),
        "roofline": res["roofline"],
        "e2e": {"value": round(e2e_val, 3), "unit": "GB/s", "h2d_bytes_per_step": int(comp_bytes),
                "d2h_bytes_per_step": int(out_bytes),
                "input_only": {"value": round(in_val, 3), "unit": "GB/s", "h2d_bytes_per_step": int(comp_bytes),
                               "d2h_bytes_per_step": 0,
                               "call": "decompress_from_host_batch (output left in device memory)"}},
        "gpu_launches": 2 * args.steps,
        "clocks": res["clocks"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        nb, el, desc = cpu_oracle_parallel(streams, args.cpu_budget / 4, threads)
        nb1, el1, desc1 = cpu_oracle_sample(streams, args.cpu_budget * 3 / 4)
        line["cpu_baseline"] = {"value": round(nb / el / 1e9, 5), "unit": "GB/s", "cores": threads,
                                "kind": "oracle", "sample": desc,
                                "single_thread": {"value": round(nb1 / el1 / 1e9, 5), "cores": 1, "sample": desc1}}
    del streams, data
    # the other configurations, on one GPU (a scaling run reports the main
    # workload only)
    if world == 1 and not args.no_extras:
        tw = datagen.WORKLOADS["text256m"]
        if args.workload != "text256m":
            _, tdata, tstreams = make_workload("text256m", None, args.format)
            tres, bufs = measure_decode(args, tw, tdata, tstreams, dev, clocks=True, extras=False)
            del bufs, tdata, tstreams
            torch.cuda.empty_cache()
            line["text256m"] = {"workload": _config(tw, args.format, 1, tw.size)["workload"], **tres}
        line["batch_1gib"] = batch_result(args, GiB)
        torch.cuda.empty_cache()
        line["serving"] = serve_result(args)
    if rank == 0:
        print(json.dumps(line), flush=True)


def batch_result(args, cap):
    """Batched workload: many independent files of uneven sizes (log-uniform
    4 KiB..16 MiB, seeded text/CSV and MRR/DE coins; the seeded prefix of the
    4096-file list up to `cap` bytes, or all files for cap None) decoded in
    ONE persistent launch replayed from a CUDA graph, against one
    gmp_decompress launch per file on the same stream.  Block size and
    sub-blocks per block come from the format autotuner on a sample of the
    mix, the launch shape from the launch autotuner on the whole batch; with
    --warps-per-cta (a profiling run) neither tuner runs: 256 KiB blocks of
    32 sub-blocks and the given shape.  Returns the figures as a dict."""
    import torch
    import paper_1606_00519_gb300 as gmp
    from paper_1606_00519_gb300 import autotune

    mix = datagen.file_mix(seed=4, n_files=args.batch_files, lo=4 * KiB, hi=16 * MiB, total_cap=cap)
    # a sample large enough to fill the GPU (the tuner times throughput, not
    # the latency of a small input): the first files of the mix, 128 MiB
    fixed = args.warps_per_cta > 0
    t0 = time.perf_counter()
    if fixed:
        tuned = {"fixed": True, "block_size": 256 * KiB, "n_sub": 32}
    else:
        parts, got = [], 0
        for sz, kind, mode, sd in mix:
            if got >= 128 * MiB:
                break
            parts.append(datagen.make_data(kind, sz, sd))
            got += sz
        sample = np.concatenate(parts)
        tuned = autotune.tune(sample, block_sizes=(128 * KiB, 256 * KiB), n_subs=(32, 64), repeats=3)
    t_tune = time.perf_counter() - t0
    bs, k = tuned["block_size"], tuned["n_sub"]
    files, total, comp_total = [], 0, 0
    for size, kind, mode, sd in mix:
        data = datagen.make_data(kind, size, sd)
        st = gmp.compress(data, bs, k, 32 * KiB, de=(mode == "de"))
        ds = gmp.DeviceStream(st)
        ref = torch.from_numpy(data).cuda()
        out = torch.empty(max(size, 16), dtype=torch.uint8, device="cuda")
        files.append((ds, out, ref))
        total += size
        comp_total += st.size
    table = gmp.make_file_table([ds.file_desc(out, ds.orig_size) for ds, out, _ in files])
    status = torch.zeros(len(files), dtype=torch.int32, device="cuda")
    ctx = gmp.Context(max_block_out=bs, max_files=len(files))
    # the launch shape for the whole batch (the format tuner's shape was
    # chosen on its sample, a fraction of the batch's blocks)
    if fixed:
        ctx.set_launch(args.warps_per_cta, args.ctas_per_sm)
        shape = {"warps_per_cta": args.warps_per_cta, "ctas_per_sm": args.ctas_per_sm}
    else:
        shape = ctx.autotune(table, len(files), status)
    graph = ctx.batch_graph(table, len(files), status)
    stream = torch.cuda.current_stream()

    def check():
        torch.cuda.synchronize()
        assert int(status.abs().sum().item()) == 0, "batch: a file reported an error"
        for ds, out, ref in files:
            if not torch.equal(out[:ds.orig_size], ref):
                raise SystemExit("batch: output differs from the input")

    graph.launch(stream)
    check()
    for _ in range(args.warmup):
        graph.launch(stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        graph.launch(stream)
    b.record(stream)
    torch.cuda.synchronize()
    graph_ms = a.elapsed_time(b) / args.steps
    # one launch per file
    st1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    for ds, out, _ in files:
        ctx.decompress_into(ds, out, st1, stream)
    check()
    a.record(stream)
    for _ in range(args.steps):
        for ds, out, _ in files:
            ctx.decompress_into(ds, out, st1, stream)
    b.record(stream)
    torch.cuda.synchronize()
    per_file_ms = a.elapsed_time(b) / args.steps
    check()
    graph.close()
    ctx.close()
    return {"metric": "batched decompressed GB/s", "value": round(total / (graph_ms / 1e3) / 1e9, 3), "unit": "GB/s",
            "steps": args.steps, "ms_per_step": round(graph_ms, 4),
            "workload": f"batch: {len(files)} files, log-uniform 4 KiB..16 MiB, text/CSV and MRR/DE mixed"
                        + (f", seeded prefix up to {cap} bytes" if cap else ""),
            "total_bytes": total, "compressed_bytes": comp_total, "ratio": round(total / comp_total, 4),
            "tuned": tuned, "tune_seconds": round(t_tune, 2),
            "launch_shape": {"warps_per_cta": shape["warps_per_cta"], "ctas_per_sm": shape["ctas_per_sm"]},
            "one_launch_per_file": {"value": round(total / (per_file_ms / 1e3) / 1e9, 3), "unit": "GB/s",
                                    "ms_per_step": round(per_file_ms, 4)},
            "speedup_vs_one_launch_per_file": round(per_file_ms / graph_ms, 3)}


def run_batch(args):
    """The batched workload alone (bench.py --batch)."""
    import torch
    torch.cuda.set_device(0)
    r = batch_result(args, None if args.batch_cap == 0 else args.batch_cap)
    line = {"metric": r.pop("metric"), "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": 1,
            "steps": r.pop("steps"), "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"),
            "higher_is_better": True, "dtype": "u8", "data": "synthetic",
            "config": {"workload": r.pop("workload")}, **r}
    print(json.dumps(line), flush=True)


def _time_batch(ctx, table, n_files, status, stream, reps):
    """Mean ms of one batched launch over `reps` launches (CUDA events)."""
    import torch
    for _ in range(2):
        ctx.decompress_batch(table, n_files, status, stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        ctx.decompress_batch(table, n_files, status, stream)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _round_profile(gmp, table, n_files, status, stream, block_size, resolve):
    """Rounds per group, largest round count and mean bytes resolved per
    group in each round (rounds past 7 together) of one statistics launch."""
    import torch
    c = gmp.Context(max_block_out=block_size, collect_stats=True, resolve=resolve, max_files=max(n_files, 1))
    c.stats_reset(stream)
    c.decompress_batch(table, n_files, status, stream)
    torch.cuda.synchronize()
    st = c.stats()
    c.close()
    per_round = [round(b / g, 1) if g else 0.0 for b, g in zip(st["round_bytes"], st["round_groups"])]
    return {"rounds_per_group": round(st["rounds"] / max(st["groups"], 1), 3), "max_rounds": st["max_rounds"],
            "bytes_per_group_in_round": per_round}


def run_sweep(args):
    """Ablation of the LZ77 resolution strategies (Sec. 5.1): Sequential
    Copying (SC), Multi-Round Resolution (MRR) and Dependency Elimination
    (DE) on the text and CSV workloads in both stream formats, then MRR and SC
    against the back-reference nesting depth (1..32 dependent copies per
    32-sequence group; the nesting-depth data sets of Sec. 5.1, one 256 KiB
    block per file, as many files as --sweep-bytes holds).  Every decoded
    output is compared with the input before it is timed."""
    import torch
    import paper_1606_00519_gb300 as gmp

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    reps = max(3, args.steps)
    strategies = []
    for wl in ("text256m", "csv1g"):
        w = datagen.WORKLOADS[wl]
        data = w.data(min(w.size, args.sweep_bytes))
        ref = torch.from_numpy(data).cuda()
        for fmt in ("bit", "byte"):
            for mode in ("mrr", "de"):
                st = gmp.compress(data, w.block_size, w.n_sub, w.window, de=(mode == "de"), byte_mode=(fmt == "byte"))
                ds = gmp.DeviceStream(st)
                out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
                table = gmp.make_file_table([ds.file_desc(out)])
                status = torch.zeros(1, dtype=torch.int32, device="cuda")
                for resolve in (("sc", "mrr", "auto") if mode == "de" else ("sc", "mrr")):
                    ctx = gmp.Context(max_block_out=w.block_size, resolve=resolve)
                    out.zero_()
                    ctx.decompress_batch(table, 1, status, stream)
                    torch.cuda.synchronize()
                    if int(status.item()) != 0 or not torch.equal(out, ref):
                        raise SystemExit(f"sweep: {wl} {fmt} {mode} {resolve} is not byte-exact")
                    ms = _time_batch(ctx, table, 1, status, stream, reps)
                    ctx.close()
                    name = {"sc": "SC", "mrr": "MRR", "auto": "DE"}[resolve]
                    row = {"workload": wl, "bytes": int(data.size), "format": fmt, "stream": mode,
                           "strategy": name, "ms": round(ms, 3), "gbs": round(data.size / ms / 1e6, 2),
                           "ratio": round(data.size / st.size, 4)}
                    row.update(_round_profile(gmp, table, 1, status, stream, w.block_size, resolve))
                    strategies.append(row)
                    print(json.dumps(row), file=sys.stderr, flush=True)
                del ds, out, table
        del ref
    nesting = []
    # one block of at most 256 KiB per file: n_inst 17-byte instances after
    # m initial strings
    n_inst = ((256 * KiB - 17 * 33) // 17) // 32 * 32
    for m in (1, 2, 4, 8, 16, 32):
        for fmt in ("bit", "byte"):
            files, total = [], 0
            while total < args.sweep_bytes:
                ts = datagen.nesting_tokens(seed=1000 * m + len(files), m=m, n_inst=n_inst)
                st = gmp.encode_tokens(ts.lit_len, ts.mlen, ts.off, ts.lits, block_size=256 * KiB, n_sub=32,
                                       byte_mode=(fmt == "byte"))
                ds = gmp.DeviceStream(st)
                out = torch.empty(max(ds.orig_size, 16), dtype=torch.uint8, device="cuda")
                files.append((ds, out))
                total += ds.orig_size
            table = gmp.make_file_table([ds.file_desc(out, ds.orig_size) for ds, out in files])
            status = torch.zeros(len(files), dtype=torch.int32, device="cuda")
            first = None
            for resolve in ("mrr", "sc"):
                ctx = gmp.Context(max_block_out=256 * KiB, resolve=resolve, max_files=len(files))
                ctx.decompress_batch(table, len(files), status, stream)
                torch.cuda.synchronize()
                if int(status.abs().sum().item()) != 0:
                    raise SystemExit(f"sweep: nesting m={m} {fmt} {resolve} reported an error")
                # both strategies must give the same bytes (the GPU tests
                # compare these streams with the serial LZ77 decode)
                got = torch.cat([out[:ds.orig_size] for ds, out in files])
                if first is None:
                    first = got.clone()
                elif not torch.equal(got, first):
                    raise SystemExit(f"sweep: nesting m={m} {fmt}: strategies disagree")
                ms = _time_batch(ctx, table, len(files), status, stream, reps)
                ctx.close()
                row = {"depth": 32 // m, "strings": m, "format": fmt, "strategy": resolve.upper(),
                       "files": len(files), "bytes": total, "ms": round(ms, 3), "gbs": round(total / ms / 1e6, 2)}
                row.update(_round_profile(gmp, table, len(files), status, stream, 256 * KiB, resolve))
                nesting.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
            del files, table, first
    line = {"metric": "LZ77 resolution strategies: decompressed GB/s", "unit": "GB/s", "n_gpus": 1,
            "steps": reps, "higher_is_better": True, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "strategy ablation on text256m and csv1g (first "
                                   f"{args.sweep_bytes // MiB} MiB), nesting-depth sets of {args.sweep_bytes // MiB} MiB",
                       "launch": "one batched launch per measurement; single-stream launches for the strategies"},
            "strategies": strategies, "nesting": nesting}
    print(json.dumps(line), flush=True)


def run_compress(args):
    """Compression: the GPU compressor (gmp_compress_gpu: match search, parse
    and entropy coding on the device) against the host compressor
    (gmp_compress, all host threads), host buffer to host buffer, on the
    workload in both modes and formats; input GB/s and ratio, the GPU
    compressor's device time per stage (input GB/s of the device work alone
    and of its entropy coding), and the decoded stream checked against the
    input on the GPU."""
    import torch
    import paper_1606_00519_gb300 as gmp

    torch.cuda.set_device(0)
    w = datagen.WORKLOADS[args.workload]
    data = w.data(args.size)
    ctx = gmp.Context(max_block_out=w.block_size)
    rows = []
    for fmt in ("bit", "byte"):
        for mode in ("mrr", "de"):
            kw = dict(de=(mode == "de"), byte_mode=(fmt == "byte"))
            res = {}
            for name, fn in (("gpu", gmp.compress_gpu), ("host", gmp.compress)):
                fn(data[:1 << 20], w.block_size, w.n_sub, w.window, **kw)  # warm-up
                reps = max(1, min(args.steps, 3))
                t0 = time.perf_counter()
                for _ in range(reps):
                    st = fn(data, w.block_size, w.n_sub, w.window, **kw)
                sec = (time.perf_counter() - t0) / reps
                out, status = ctx.decompress(gmp.DeviceStream(st))
                if status != 0 or not np.array_equal(out.cpu().numpy(), data):
                    raise SystemExit(f"compress: {name} {fmt} {mode} stream does not decode to the input")
                res[name] = {"gbs": round(data.size / sec / 1e9, 3), "ratio": round(data.size / st.size, 4)}
                if name == "gpu":
                    t = gmp.compress_gpu_times()
                    dev_ms = t["match_ms"] + t["parse_ms"] + t["encode_ms"]
                    res[name]["device_ms"] = {k: round(t[k], 3) for k in ("match_ms", "parse_ms", "encode_ms")}
                    res[name]["device_gbs"] = round(data.size / dev_ms / 1e6, 3)
                    res[name]["encode_gbs"] = round(data.size / t["encode_ms"] / 1e6, 3)
            row = {"format": fmt, "stream": mode, **res}
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    line = {"metric": "compression input GB/s (host buffers)", "unit": "GB/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{w.name}: {data.size // MiB} MiB {w.kind}, {w.block_size // KiB} KiB blocks",
                       "host_threads": os.cpu_count()},
            "rows": rows}
    print(json.dumps(line), flush=True)


def _concurrency(spans):
    """Batched launches in flight at once, from each distinct launch's
    (start, end) on one clock (requests of one batch share their launch):
    the largest count over time and the time-weighted mean while any launch
    is in flight."""
    ev = sorted([(a, 1) for a, b in spans] + [(b, -1) for a, b in spans])
    cur = peak = 0
    busy = area = 0.0
    last = None
    for t, d in ev:
        if last is not None and cur > 0:
            busy += t - last
            area += cur * (t - last)
        cur += d
        peak = max(peak, cur)
        last = t
    return {"launches": len(spans), "max": peak, "mean": round(area / busy, 3) if busy > 0 else 0.0}


def serve_result(args):
    """Serving: Poisson arrivals of requests (16 KiB..64 MiB, mixed content
    and modes) admitted under a device-memory budget by the continuous-batching
    server; p50/p99 latency (submit -> completion) and served GB/s at 25/50/90 %
    of the closed-loop peak, next to the same arrivals served one launch per
    request.  Returns the figures as a dict."""
    import threading

    import torch
    import paper_1606_00519_gb300 as gmp

    # a seeded pool of distinct requests; the arrival sequence draws from it
    mix = datagen.request_mix(seed=5, n=args.serve_pool, lo=16 * KiB, hi=args.serve_max)
    pool = []
    for size, kind, mode, sd in mix:
        data = datagen.make_data(kind, size, sd)
        st = gmp.compress(data, 256 * KiB, 32, 32 * KiB, de=(mode == "de"))
        pin = torch.from_numpy(st.copy()).pin_memory().numpy()
        pool.append((size, pin, data))
    mean_size = float(np.mean([p[0] for p in pool]))
    rng = np.random.default_rng(11)

    def run(server, arrivals, picks):
        """Submit pool[picks[i]] at arrivals[i] (seconds); returns latencies,
        total bytes, wall seconds; checks every output's size and status, and
        after the run the bytes of a sample (every 97th request)."""
        lat, done, nbytes = [], 0, 0
        spans, gpu_spans = set(), set()
        ids = {}
        errors = []
        checked = []  # sampled requests whose bytes are compared after the run
        lock = threading.Lock()

        def collector():
            nonlocal done, nbytes
            while done < len(picks):
                for c in server.poll(wait_ms=5):
                    with lock:
                        i = ids.pop(c["id"])
                    if c["status"] != 0 or c["out_bytes"] != pool[picks[i]][0]:
                        errors.append((i, c["status"]))
                    lat.append(c["t_done"] - c["t_submit"])
                    spans.add((c["t_start"], c["t_done"]))
                    gpu_spans.add((c["t_gpu_ready"], c["t_gpu_done"]))
                    nbytes += c["out_bytes"]
                    if i % 97 == 0:
                        checked.append((i, c["id"], c["out_bytes"]))  # kept on the device until then
                    else:
                        server.release(c["id"])
                    done += 1

        th = threading.Thread(target=collector)
        th.start()
        t0 = time.perf_counter()
        for i, (ta, k) in enumerate(zip(arrivals, picks)):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            with lock:
                ids[server.submit(pool[k][1])] = i
        th.join()
        wall = time.perf_counter() - t0
        # the sampled outputs' bytes, outside the timed region (a synchronous
        # copy inside it held up the collector)
        for i, rid, nb in checked:
            buf = np.empty(nb, np.uint8)
            server.copy_out(rid, buf)
            if not np.array_equal(buf, pool[picks[i]][2]):
                errors.append((i, "bytes"))
            server.release(rid)
        if errors:
            raise SystemExit(f"serve: {len(errors)} bad results, e.g. {errors[:3]}")
        run.last_concurrency = _concurrency(spans)
        run.last_gpu_concurrency = _concurrency(gpu_spans)
        return np.array(lat), nbytes, wall

    n = args.serve_requests
    picks = rng.integers(0, len(pool), n)
    servers = {
        "batched": dict(budget_bytes=args.serve_budget, n_lanes=8, max_batch=64),
        "one_call_per_file": dict(budget_bytes=args.serve_budget, n_lanes=1, max_batch=1),
    }
    result = {"metric": "served decompressed GB/s and latency", "unit": "GB/s", "n_gpus": 1,
              "config": {"workload": f"serving: requests log-uniform 16 KiB..{args.serve_max // MiB} MiB, "
                                     "mixed text/CSV, MRR/DE, 256 KiB blocks, K=32",
                         "pool": len(pool), "requests_per_load": n, "budget_bytes": args.serve_budget,
                         "mean_request_bytes": int(mean_size)}}
    for name, kw in servers.items():
        srv = gmp.Server(**kw)
        # closed loop: every request at once (saturated peak; enough requests
        # that the first and last batches do not dominate), after one untimed
        # pass that warms the server's lanes up
        run(srv, np.zeros(n), picks)
        lat, nb, wall = run(srv, np.zeros(n), picks)
        peak = nb / wall / 1e9
        # launches in flight on the host clock (launch -> completion seen), and
        # decodes on the GPU's clock (inputs in and decode next -> decode end)
        out = {"peak_gbs": round(peak, 3), "peak_launches_in_flight": run.last_concurrency,
               "peak_decodes_on_gpu": run.last_gpu_concurrency}
        for load in (0.25, 0.5, 0.9):
            rate = load * peak * 1e9 / mean_size
            arr = datagen.poisson_arrivals(seed=int(load * 100), n=n, rate_per_s=rate)
            lat, nb, wall = run(srv, arr, picks)
            out[f"load_{int(load * 100)}"] = {"offered_req_per_s": round(rate, 1),
                                              "served_gbs": round(nb / wall / 1e9, 3),
                                              "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                                              "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                                              "launches_in_flight": run.last_concurrency,
                                              "decodes_on_gpu": run.last_gpu_concurrency}
        srv.close()
        result[name] = out
    result["value"] = result["batched"]["peak_gbs"]
    return result


def run_serve(args):
    """The serving benchmark alone (bench.py --serve)."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(serve_result(args)), flush=True)




def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gmp", choices=["gmp", "reference"])
    ap.add_argument("--workload", default="csv1g", choices=sorted(datagen.WORKLOADS))
    ap.add_argument("--size", type=int, default=None, help="override bytes per stream")
    ap.add_argument("--format", default="bit", choices=["bit", "byte"],
                    help="stream format: Huffman blocks (bit) or byte-level blocks (byte)")
    ap.add_argument("--warps-per-cta", type=int, default=0, help="fixed launch shape instead of the autotuner's")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="with --warps-per-cta: CTAs per SM (0: as many as fit)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle CPU baseline")
    ap.add_argument("--ref-blocks", type=int, default=16, help="oracle blocks per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the main workload (no text256m, batch_1gib and serving sub-objects)")
    ap.add_argument("--ref-pool", type=int, default=256 * MiB,
                    help="reference arm: bytes of the workload compressed by the oracle per mode")
    ap.add_argument("--batch", action="store_true", help="batched many-file benchmark instead of the decode step")
    ap.add_argument("--batch-files", type=int, default=4096)
    ap.add_argument("--batch-cap", type=int, default=GiB, help="seeded prefix of the file list up to this many bytes "
                                                                 "(0: all files)")
    ap.add_argument("--sweep", action="store_true", help="resolution strategies and nesting-depth sweep")
    ap.add_argument("--compress", action="store_true", help="GPU parse against host compressor")
    ap.add_argument("--sweep-bytes", type=int, default=256 * MiB)
    ap.add_argument("--serve", action="store_true", help="serving benchmark instead of the decode step")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-pool", type=int, default=96)
    ap.add_argument("--serve-max", type=int, default=64 * MiB)
    ap.add_argument("--serve-budget", type=int, default=32 * GiB)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.sweep:
        run_sweep(args)
    elif args.compress:
        run_compress(args)
    elif args.batch:
        run_batch(args)
    elif args.serve:
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gmp(args)


if __name__ == "__main__":
    main()
