"""GPU tests of the host-to-host calls (the paper's "(In/Out)" mode): streams
in host memory, copied in piece by piece while one persistent launch decodes
them, outputs copied back as pieces complete, byte for byte against the
oracle, with pinned and pageable buffers, many pieces on a small launch,
1 MiB blocks, more pieces than the flag arrays first hold, mixed formats, unaligned
buffers, groups larger than the ring, per-file error status, and a wait for
input that runs out (a flag dropped on the host)."""
import time

import numpy as np
import pytest

import datagen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600, method="thread")]

KiB, MiB = 1 << 10, 1 << 20


@pytest.fixture(scope="module")
def gmp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1606_00519_gb300 import _native
    _native.build()
    import paper_1606_00519_gb300 as g
    return g


def _pinned(torch, n):
    return torch.empty(max(n, 1), dtype=torch.uint8).pin_memory().numpy()


@pytest.mark.parametrize("size", [0, 1, 4095, 3 * MiB + 17])
def test_single_stream_sizes(gmp, size):
    data = datagen.markov_text(size, seed=size + 5, order=3) if size else np.zeros(0, np.uint8)
    s = gmp.compress(data, 64 * KiB, 16, 32 * KiB, de=True)
    ctx = gmp.Context(max_block_out=64 * KiB)
    out, st = ctx.decompress_host(s)
    assert st == 0 and np.array_equal(out, data)
    ctx.close()


def test_batch_of_mixed_streams_pinned_and_pageable(gmp):
    import torch
    streams, datas = [], []
    for i in range(7):
        kind = "csv" if i % 2 else "text3"
        data = datagen.make_data(kind, 700_000 + 99_999 * i, 50 + i)
        s = gmp.compress(data, 128 * KiB, 32, 32 * KiB, de=(i % 3 == 0), byte_mode=(i % 4 == 1))
        streams.append(s)
        datas.append(data)
    ctx = gmp.Context(max_block_out=128 * KiB, collect_stats=True)
    ctx.stats_reset()
    outs, sts = ctx.decompress_host_batch(streams)
    assert sts == [0] * len(streams)
    for o, d, s in zip(outs, datas, streams):
        assert np.array_equal(o, d) and np.array_equal(o, oracle.decompress(s))
    assert ctx.stats()["blocks"] == sum(gmp.stream_info(s).n_blocks for s in streams)
    # pinned inputs and outputs
    pin_in = []
    for s in streams:
        p = _pinned(torch, s.size)[:s.size]
        p[:] = s
        pin_in.append(p)
    pin_out = [_pinned(torch, d.size) for d in datas]
    outs, sts = ctx.decompress_host_batch(pin_in, pin_out)
    assert sts == [0] * len(streams)
    for o, d in zip(outs, datas):
        assert np.array_equal(o, d)
    ctx.close()


def test_many_pieces_small_launch(gmp):
    # a small launch shape (152 warp slots) and 4 KiB blocks: 1538 blocks in
    # 33 pieces of up to 49, each warp decoding blocks of many pieces
    streams, datas = [], []
    for i in range(3):
        data = datagen.csv_records(2 * MiB + 1000 * i, seed=70 + i)
        streams.append(gmp.compress(data, 4 * KiB, 8, 4 * KiB, de=(i == 1)))
        datas.append(data)
    ctx = gmp.Context(max_block_out=4 * KiB, warps_per_cta=1, ctas_per_sm=1)
    for _ in range(2):  # the staging, streams and events are reused
        outs, sts = ctx.decompress_host_batch(streams)
        assert sts == [0, 0, 0]
        for o, d in zip(outs, datas):
            assert np.array_equal(o, d)
    ctx.close()


def test_large_blocks_both_modes(gmp):
    # 1 MiB blocks of 64 sub-blocks (the Huffman phase takes them 32 at a
    # time) through both host calls, MRR and DE, against the oracle
    datas = [datagen.make_data("csv", 9 * MiB + 12345, 501), datagen.make_data("text3", 6 * MiB + 777, 502)]
    streams = [gmp.compress(d, 1 * MiB, 64, 32 * KiB, de=(i == 1)) for i, d in enumerate(datas)]
    ctx = gmp.Context(max_block_out=1 * MiB)
    outs, sts = ctx.decompress_host_batch(streams)
    assert sts == [0, 0]
    for o, d, st in zip(outs, datas, streams):
        assert np.array_equal(o, d) and np.array_equal(o, oracle.decompress(st))
    douts, sts = ctx.decompress_from_host_batch(streams)
    assert sts == [0, 0]
    for o, d in zip(douts, datas):
        assert np.array_equal(o.cpu().numpy(), d)
    ctx.close()


def test_more_pieces_than_flags(gmp):
    # 1100 small streams (one to three blocks, one piece each) are 1100
    # pieces, more than the 1024 flag words a context first allocates; the
    # next calls reuse the grown flags with fewer pieces, then more again
    import torch
    datas = [datagen.make_data("csv" if i % 2 else "text3", 3000 + 7 * i, 300 + i) for i in range(1100)]
    streams = [gmp.compress(d, 4 * KiB, 4, 4 * KiB, de=(i % 3 == 0)) for i, d in enumerate(datas)]
    ctx = gmp.Context(max_block_out=4 * KiB)
    for sel in (slice(0, 1100), slice(0, 5), slice(17, 1100)):
        outs, sts = ctx.decompress_host_batch(streams[sel])
        assert sts == [0] * len(outs)
        for o, d in zip(outs, datas[sel]):
            assert np.array_equal(o, d)
        douts, sts = ctx.decompress_from_host_batch(streams[sel])
        assert sts == [0] * len(douts)
        got = torch.cat([o for o in douts]).cpu().numpy()
        assert np.array_equal(got, np.concatenate(datas[sel]))
    ctx.close()


def test_per_file_status_and_capacity(gmp):
    good = datagen.markov_text(500_000, seed=81, order=2)
    s_good = gmp.compress(good, 64 * KiB, 16, 8 * KiB)
    bad_data = datagen.markov_text(500_000, seed=82, order=2)
    s_bad = oracle.compress(bad_data, oracle.params(64 * KiB, 16, 8 * KiB))
    bo = int(s_bad[64 + 8 * 2:72 + 8 * 2].view(np.uint64)[0])
    s_bad[bo + 8 + ord("e") // 2] ^= 0x0F if ord("e") % 2 == 0 else 0xF0  # block 2's code lengths break Kraft
    assert oracle.decompress_status(s_bad) == oracle.BAD_HEADER
    ctx = gmp.Context(max_block_out=64 * KiB)
    outs, sts = ctx.decompress_host_batch([s_good, s_bad, s_good])
    assert sts[0] == 0 and sts[2] == 0 and sts[1] == oracle.BAD_HEADER
    assert np.array_equal(outs[0], good) and np.array_equal(outs[2], good)
    with pytest.raises(gmp.GmpError):
        ctx.decompress_host_batch([s_good], [np.empty(good.size - 1, np.uint8)])
    small = gmp.Context(max_block_out=16 * KiB)
    with pytest.raises(gmp.GmpError):  # blocks larger than the context's max_block_out
        small.decompress_host(s_good)
    small.close()
    ctx.close()


def _pin_copy(torch, a, offset=0):
    p = _pinned(torch, a.size + offset)[offset:offset + a.size]
    p[:] = a
    return p


def test_pinned_buffers_edge_cases(gmp):
    import torch
    rng = np.random.default_rng(91)
    rnd = rng.integers(0, 256, 300_000).astype(np.uint8)  # long literal runs: groups larger than the ring
    datas = [datagen.markov_text(1_000_000, seed=92, order=3), rnd,
             np.concatenate([rnd[:50_000], datagen.csv_records(400_000, seed=93)]),
             np.zeros(0, np.uint8), datagen.csv_records(33_333, seed=94)]
    streams = [gmp.compress(datas[0], 64 * KiB, 16, 32 * KiB, de=True),
               gmp.compress(datas[1], 256 * KiB, 32, 32 * KiB),
               gmp.compress(datas[2], 1000, 4, 1000, byte_mode=True),  # blocks not a multiple of 16 bytes
               gmp.compress(datas[3], 64 * KiB, 16, 8 * KiB),
               gmp.compress(datas[4], 64 * KiB, 16, 8 * KiB)]
    ctx = gmp.Context(max_block_out=256 * KiB, collect_stats=True)
    pin_in = [_pin_copy(torch, s) for s in streams]
    for out_offset in (0, 1):  # outputs 16-byte aligned or not
        pin_out = [_pinned(torch, d.size + 1)[out_offset:out_offset + d.size] for d in datas]
        for o in pin_out:
            o[:] = 0xA5
        ctx.stats_reset()
        outs, sts = ctx.decompress_host_batch(pin_in, pin_out)
        assert sts == [0] * len(datas)
        for o, d in zip(outs, datas):
            assert np.array_equal(o, d)
        assert ctx.stats()["blocks"] == sum(gmp.stream_info(s).n_blocks for s in streams)
    # a stream that is not 16-byte aligned, or pageable outputs
    mixed_in = [_pin_copy(torch, streams[0], 1)] + pin_in[1:]
    outs, sts = ctx.decompress_host_batch(mixed_in, [_pinned(torch, d.size) for d in datas])
    assert sts == [0] * len(datas) and all(np.array_equal(o, d) for o, d in zip(outs, datas))
    outs, sts = ctx.decompress_host_batch(pin_in, [np.empty(d.size, np.uint8) for d in datas])
    assert sts == [0] * len(datas) and all(np.array_equal(o, d) for o, d in zip(outs, datas))
    # per-file status with pinned buffers
    bad = streams[4].copy()
    bo = int(bad[64:72].view(np.uint64)[0])
    bad[bo + 8 + ord("e") // 2] ^= 0x0F if ord("e") % 2 == 0 else 0xF0  # block 0's code lengths break Kraft
    assert oracle.decompress_status(bad) == oracle.BAD_HEADER
    outs, sts = ctx.decompress_host_batch([pin_in[0], _pin_copy(torch, bad)],
                                          [_pinned(torch, datas[0].size), _pinned(torch, datas[4].size)])
    assert sts == [0, oracle.BAD_HEADER] and np.array_equal(outs[0], datas[0])
    ctx.close()


def test_from_host_to_device_outputs(gmp):
    # the paper's "(In)" mode: host streams in, outputs left in device memory
    import torch
    datas = [datagen.make_data("csv" if i % 2 else "text3", 500_000 + 77_777 * i, 60 + i) for i in range(5)]
    streams = [gmp.compress(d, 128 * KiB, 32, 32 * KiB, de=(i % 2 == 0), byte_mode=(i == 3))
               for i, d in enumerate(datas)]
    for shape in ((0, 0), (1, 1)):  # default shape, and a launch of 152 warps
        ctx = gmp.Context(max_block_out=128 * KiB, warps_per_cta=shape[0], ctas_per_sm=shape[1])
        for pinned in (False, True):
            ins = [_pin_copy(torch, s) for s in streams] if pinned else streams
            outs, sts = ctx.decompress_from_host_batch(ins)
            assert sts == [0] * len(datas)
            for o, d in zip(outs, datas):
                assert o.is_cuda and np.array_equal(o.cpu().numpy(), d)
        ctx.close()
    # per-file status, and a device buffer that is too small
    bad = oracle.compress(datas[0], oracle.params(64 * KiB, 16, 8 * KiB))
    bo = int(bad[64 + 8:72 + 8].view(np.uint64)[0])
    bad[bo + 8 + ord("e") // 2] ^= 0x0F if ord("e") % 2 == 0 else 0xF0  # block 1's code lengths break Kraft
    assert oracle.decompress_status(bad) == oracle.BAD_HEADER
    ctx = gmp.Context(max_block_out=128 * KiB)
    outs, sts = ctx.decompress_from_host_batch([streams[1], bad])
    assert sts == [0, oracle.BAD_HEADER] and np.array_equal(outs[0].cpu().numpy(), datas[1])
    small = torch.empty(datas[1].size - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(gmp.GmpError):
        ctx.decompress_from_host_batch([streams[1]], [small])
    ctx.close()


def test_input_wait_runs_out(gmp):
    # fault injected on the host: piece 0's input is copied but its flag is
    # never written.  The warps waiting for it give up after the context's
    # limit (200 ms), its file reports INPUT_TIMEOUT, the other file decodes,
    # the kernel ends by itself, and the next call on the context is exact.
    datas = [datagen.make_data("csv", 3_000_000, 401), datagen.make_data("text3", 2_000_000, 402)]
    streams = [gmp.compress(d, 64 * KiB, 16, 32 * KiB) for d in datas]
    ctx = gmp.Context(max_block_out=64 * KiB)
    ctx.set_input_wait(200)
    for call in (ctx.decompress_host_batch, ctx.decompress_from_host_batch):
        ctx.debug_drop_input_flag(0)
        t0 = time.perf_counter()
        outs, sts = call(streams)
        assert time.perf_counter() - t0 < 5.0
        assert gmp.STATUS_NAMES[sts[0]] == "INPUT_TIMEOUT" and sts[1] == 0
        got = outs[1] if isinstance(outs[1], np.ndarray) else outs[1].cpu().numpy()
        assert np.array_equal(got, datas[1])
        outs, sts = call(streams)  # no flag dropped: the context is still usable
        assert sts == [0, 0]
        for o, d in zip(outs, datas):
            assert np.array_equal(o if isinstance(o, np.ndarray) else o.cpu().numpy(), d)
    ctx.close()
