"""GPU batched decoding: many streams of uneven sizes, MRR and DE mixed, in
one persistent launch and replayed from a CUDA graph; every file byte-exact
against the oracle and its own status word."""
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
