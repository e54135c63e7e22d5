"""GPU parity for Gompresso/Byte streams (Sec. 3.1 and 3.2: the LZ77
sequences coded at byte level, no Huffman trees): the CUDA decoder through
the C ABI against the CPU oracle, byte for byte, on streams from both
compressors, both dependency modes, edge sizes, long literal runs, nesting
depths, batches that mix Byte and Huffman files, and corrupt records (which
must give an error status, not a fault)."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

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


@pytest.fixture(scope="module")
def ctx(gmp):
    c = gmp.Context(max_block_out=256 * KiB, collect_stats=True)
    yield c
    c.close()


def gpu_decode(gmp, ctx, stream):
    ds = gmp.DeviceStream(stream)
    out, status = ctx.decompress(ds)
    return out.cpu().numpy(), status


def check_stream(gmp, ctx, stream, data=None):
    expect = oracle.decompress(stream)
    got, status = gpu_decode(gmp, ctx, stream)
    assert status == 0, gmp.STATUS_NAMES.get(status, status)
    assert got.size == expect.size
    if not np.array_equal(got, expect):
        i = int(np.flatnonzero(got != expect)[0])
        raise AssertionError(f"first differing byte {i} of {got.size}")
    if data is not None:
        assert np.array_equal(expect, data)


def byte_params(block_size, window, de=False, **kw):
    return oracle.params(block_size, 1, window, de=de, byte_mode=True, **kw)


@pytest.mark.parametrize("name", ["text1m", "text256m", "csv1g"])
@pytest.mark.parametrize("mode", ["mrr", "de"])
def test_oracle_byte_streams(gmp, ctx, name, mode):
    w = datagen.WORKLOADS[name]
    data = w.data(5 * w.block_size + 4321)  # several blocks, ragged tail
    s = oracle.compress(data, byte_params(w.block_size, w.window, de=(mode == "de")))
    check_stream(gmp, ctx, s, data)


@pytest.mark.parametrize("name", ["text1m", "text256m", "csv1g"])
@pytest.mark.parametrize("mode", ["mrr", "de"])
def test_product_byte_streams(gmp, ctx, name, mode):
    w = datagen.WORKLOADS[name]
    data = w.data(9 * w.block_size + 99)
    s = gmp.compress(data, w.block_size, w.n_sub, w.window, de=(mode == "de"), byte_mode=True)
    assert oracle.validate(s)["rc"] == 0
    check_stream(gmp, ctx, s, data)


@pytest.mark.parametrize("size", [0, 1, 2, 15, 16, 17, 1000, 1023, 1024, 65535, 65536, 65537])
def test_byte_sizes(gmp, ctx, size):
    data = datagen.csv_records(size, seed=size + 3) if size else np.zeros(0, np.uint8)
    check_stream(gmp, ctx, oracle.compress(data, byte_params(64 * KiB, 8 * KiB)), data)
    check_stream(gmp, ctx, gmp.compress(data, 64 * KiB, 1, 8 * KiB, byte_mode=True), data)


def test_byte_long_literal_runs_and_degenerate_data(gmp, ctx):
    rng = np.random.default_rng(6)
    rnd = rng.integers(0, 256, 600_000).astype(np.uint8)  # literal-only sequences of 1023 bytes
    zeros = np.zeros(600_000, np.uint8)                    # distance-1 overlapping copies
    two = np.tile(np.frombuffer(b"ab", np.uint8), 300_000)
    mixed = np.concatenate([rnd[:70_000], datagen.markov_text(200_000, seed=6, order=3), rnd[70_000:140_000]])
    for data in (rnd, zeros, two, mixed):
        for de in (False, True):
            check_stream(gmp, ctx, oracle.compress(data, byte_params(256 * KiB, 32 * KiB, de=de)), data)
            check_stream(gmp, ctx, gmp.compress(data, 256 * KiB, 1, 32 * KiB, de=de, byte_mode=True), data)


def test_byte_odd_block_sizes_and_small_windows(gmp, ctx):
    data = datagen.markov_text(50_000, seed=8, order=2)
    for bs, win, mm in [(1000, 1, 64), (4093, 4096, 3), (12345, 257, 17), (16, 8, 64)]:
        check_stream(gmp, ctx, oracle.compress(data, byte_params(bs, win, max_match=mm)), data)


def test_byte_de_streams_take_one_pass(gmp, ctx):
    w = datagen.WORKLOADS["text256m"]
    data = w.data(4 * w.block_size)
    s = oracle.compress(data, byte_params(w.block_size, w.window, de=True))
    ctx.stats_reset()
    check_stream(gmp, ctx, s, data)
    st = ctx.stats()
    assert st["de_fallback_groups"] == 0 and st["max_rounds"] == 1 and st["groups"] > 0


@pytest.mark.parametrize("m", [1, 4, 32])
def test_byte_nesting_depth_round_counts(gmp, ctx, m):
    ts = datagen.nesting_tokens(seed=200 + m, m=m, n_inst=32 * 40)
    s = oracle.encode_tokens(ts, byte_params(256 * KiB, 32 * KiB))
    ctx.stats_reset()
    check_stream(gmp, ctx, s)
    st = ctx.stats()
    assert st["rounds"] == int(oracle.mrr_rounds(ts.lit_len, ts.mlen, ts.off, ts.lits).sum())
    assert st["max_rounds"] == 32 // m


def test_batch_mixes_byte_and_huffman_files(gmp):
    import torch
    files, datas = [], []
    for i in range(12):
        data = datagen.markov_text(300_000 + 7777 * i, seed=40 + i, order=3)
        byte = i % 2 == 0
        s = gmp.compress(data, 64 * KiB, 16, 16 * KiB, de=(i % 3 == 0), byte_mode=byte)
        ds = gmp.DeviceStream(s)
        out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
        files.append((ds, out))
        datas.append(data)
    c = gmp.Context(max_block_out=64 * KiB)
    table = gmp.make_file_table([ds.file_desc(out) for ds, out in files])
    status = torch.full((len(files),), -1, dtype=torch.int32, device="cuda")
    c.decompress_batch(table, len(files), status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(files)
    for (ds, out), data in zip(files, datas):
        assert np.array_equal(out.cpu().numpy(), data)
    c.close()


# ---------------------------------------------------------------- corrupt input

def _byte_stream():
    data = datagen.markov_text(5 * 64 * KiB, seed=33, order=2)
    return data, oracle.compress(data, byte_params(64 * KiB, 8 * KiB))


def _block_offset(s, b):
    return int(s[64 + 8 * b:72 + 8 * b].view(np.uint64)[0])


def _records(s, b):
    bo = _block_offset(s, b)
    n_seq = int(s[bo:bo + 4].view(np.uint32)[0])
    return bo, s[bo + 16:bo + 16 + 4 * n_seq].view(np.uint32)


def test_byte_match_code_63_is_corrupt(gmp, ctx):
    data, s = _byte_stream()
    bad = s.copy()
    _, rec = _records(bad, 1)
    k = int(np.flatnonzero((rec >> 10) & 63)[5])
    rec[k] |= np.uint32(63 << 10)
    assert oracle.decompress_status(bad) == oracle.CORRUPT_SYMBOL
    assert gpu_decode(gmp, ctx, bad)[1] == oracle.CORRUPT_SYMBOL


def test_byte_distance_before_block_start(gmp, ctx):
    data, s = _byte_stream()
    bad = s.copy()
    _, rec = _records(bad, 2)
    k = int(np.flatnonzero((rec >> 10) & 63)[0])  # the block's first back-reference
    rec[k] = (rec[k] & np.uint32(0xffff)) | np.uint32(0xffff << 16)  # distance 65536
    assert oracle.decompress_status(bad) == oracle.BAD_OFFSET
    assert gpu_decode(gmp, ctx, bad)[1] == oracle.BAD_OFFSET


def test_byte_literal_count_mismatch(gmp, ctx):
    data, s = _byte_stream()
    bad = s.copy()
    bo = _block_offset(bad, 3)
    v = bad[bo + 8:bo + 12].view(np.uint32)
    v[0] -= 1  # one literal fewer than the records use
    assert oracle.decompress_status(bad) == oracle.OUTPUT_OVERRUN
    assert gpu_decode(gmp, ctx, bad)[1] == oracle.OUTPUT_OVERRUN


def test_byte_literal_length_overrun(gmp, ctx):
    data, s = _byte_stream()
    bad = s.copy()
    _, rec = _records(bad, 0)
    rec[-1] |= np.uint32(1023)  # the block's last record claims 1023 literals
    assert oracle.decompress_status(bad) != oracle.OK
    assert gpu_decode(gmp, ctx, bad)[1] in (oracle.OUTPUT_OVERRUN, oracle.BAD_HEADER)


def test_byte_random_bit_flips_never_fault(gmp, ctx):
    data, s = _byte_stream()
    rng = np.random.default_rng(78)
    start = _block_offset(s, 0)
    for _ in range(80):
        bad = s.copy()
        i = int(rng.integers(start, s.size - 17))
        bad[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        ost = oracle.decompress_status(bad)
        got, st = gpu_decode(gmp, ctx, bad)
        # both accept (and agree on the bytes) or both reject
        assert (ost == 0) == (st == 0), (i, ost, st)
        if ost == 0:
            assert np.array_equal(got, oracle.decompress(bad))
