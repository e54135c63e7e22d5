"""GPU batched decoding: many streams of uneven sizes, MRR and DE mixed, in
one persistent launch and replayed from a CUDA graph; every file byte-exact
against the oracle and its own status word.  Both ways of handing out work
items: a fixed first block per warp spread over the SMs (the default) and
the work counter alone (contexts marked concurrent), also with fewer warps
than blocks and with two launches overlapping on two streams."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

KiB = 1 << 10


@pytest.fixture(scope="module")
def gmp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1606_00519_gb300 import _native
    _native.build()
    import paper_1606_00519_gb300 as g
    return g


def _files(n, seed, lo=1, hi=600 * KiB):
    mix = datagen.file_mix(seed, n, lo=max(lo, 1), hi=hi)
    out = []
    for i, (size, kind, mode, s) in enumerate(mix):
        data = datagen.make_data(kind, size, s)
        bs = [16 * KiB, 64 * KiB, 256 * KiB][i % 3]
        stream = oracle.compress(data, oracle.params(bs, [8, 16, 32][i % 3], 32 * KiB, de=(mode == "de")))
        out.append((data, stream))
    return out


def _decode_batch(gmp, ctx, files, use_graph=False, replays=1):
    import torch
    ds = [gmp.DeviceStream(s) for _, s in files]
    outs = [torch.full((max(d.orig_size, 1),), 0x5A, dtype=torch.uint8, device="cuda") for d in ds]
    table = gmp.make_file_table([d.file_desc(o, d.orig_size) for d, o in zip(ds, outs)])
    status = torch.full((len(files),), -1, dtype=torch.int32, device="cuda")
    if use_graph:
        g = ctx.batch_graph(table, len(files), status)
        for _ in range(replays):
            for o in outs:
                o.fill_(0x5A)
            g.launch()
        torch.cuda.synchronize()
        g.close()
    else:
        ctx.decompress_batch(table, len(files), status)
        torch.cuda.synchronize()
    return [o[:d.orig_size].cpu().numpy() for d, o in zip(ds, outs)], status.cpu().numpy()


def test_batch_uneven_files(gmp):
    files = _files(40, seed=1)
    ctx = gmp.Context(max_block_out=256 * KiB)
    outs, st = _decode_batch(gmp, ctx, files)
    assert np.all(st == 0)
    for (data, _), got in zip(files, outs):
        assert np.array_equal(got, data)
    ctx.close()


def test_batch_graph_replay(gmp):
    files = _files(25, seed=2)
    ctx = gmp.Context(max_block_out=256 * KiB)
    outs, st = _decode_batch(gmp, ctx, files, use_graph=True, replays=3)
    assert np.all(st == 0)
    for (data, _), got in zip(files, outs):
        assert np.array_equal(got, data)
    ctx.close()


def test_batch_status_is_per_file(gmp):
    files = _files(6, seed=3, lo=100 * KiB)
    data, s = files[2]
    bad = s.copy()
    bad[16:20] = np.frombuffer(np.uint32(1).tobytes(), np.uint8)  # window 1: distances too large
    files[2] = (data, bad)
    ctx = gmp.Context(max_block_out=256 * KiB)
    outs, st = _decode_batch(gmp, ctx, files)
    assert st[2] == oracle.BAD_OFFSET
    for i, ((d, _), got) in enumerate(zip(files, outs)):
        if i != 2:
            assert st[i] == 0 and np.array_equal(got, d)
    ctx.close()


def test_batch_alone_equals_in_mix(gmp):
    files = _files(12, seed=4)
    ctx = gmp.Context(max_block_out=256 * KiB)
    mixed, st = _decode_batch(gmp, ctx, files)
    assert np.all(st == 0)
    for f, got in zip(files, mixed):
        alone, st1 = _decode_batch(gmp, ctx, [f])
        assert st1[0] == 0 and np.array_equal(alone[0], got)
    ctx.close()


@pytest.mark.parametrize("shape", [(0, 0), (1, 1)])
def test_batch_concurrent_contexts(gmp, shape):
    # (1, 1): 152 warps for hundreds of blocks, so most blocks come from the
    # work counter after a warp's first one
    import torch
    files = _files(30, seed=5)
    ctxs = [gmp.Context(max_block_out=256 * KiB, warps_per_cta=shape[0], ctas_per_sm=shape[1], concurrent=c)
            for c in (False, True)]
    for c in ctxs:
        outs, st = _decode_batch(gmp, c, files)
        assert np.all(st == 0)
        for (data, _), got in zip(files, outs):
            assert np.array_equal(got, data)
    # two launches at once on two streams, one per context
    ds = [gmp.DeviceStream(s) for _, s in files]
    res = []
    streams = [torch.cuda.Stream() for _ in ctxs]
    for c, cs in zip(ctxs, streams):
        outs = [torch.zeros(max(d.orig_size, 1), dtype=torch.uint8, device="cuda") for d in ds]
        table = gmp.make_file_table([d.file_desc(o, d.orig_size) for d, o in zip(ds, outs)])
        status = torch.full((len(ds),), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        c.decompress_batch(table, len(ds), status, cs)
        res.append((outs, status, table))
    torch.cuda.synchronize()
    for outs, status, _ in res:
        assert np.all(status.cpu().numpy() == 0)
        for (data, _), o, d in zip(files, outs, ds):
            assert np.array_equal(o[:d.orig_size].cpu().numpy(), data)
    for c in ctxs:
        c.close()
