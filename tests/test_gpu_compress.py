"""GPU tests of the compressor that runs on the GPU end to end
(gmp_compress_gpu; Sec. 3.1 block-parallel compression and the two Huffman
trees per block, Sec. 4.2 DE): every stream it writes passes the oracle's
validators (Kraft equality and code lengths within the limit for both trees
of every block, window and block bounds, sub-block sizes, the DE property
for DE streams), decodes to the input in the oracle and on the GPU, in both
formats and modes, at edge sizes and on degenerate data (single-symbol
alphabets, incompressible blocks that are one literal run); the output is
deterministic and the entropy coding ran on the device."""
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


@pytest.fixture(scope="module")
def ctx(gmp):
    c = gmp.Context(max_block_out=256 * KiB)
    yield c
    c.close()


def check(gmp, ctx, s, data, de):
    rep = oracle.validate(s)
    assert rep["rc"] == 0 and rep["offsets_ok"] and rep["blocks_ok"], rep
    if gmp.stream_info(s).flags & 2:
        assert rep["kraft_ok"] and rep["lengths_ok"] and rep["subblocks_ok"]
    if de:
        assert rep["de_weak_ok"]
    assert np.array_equal(oracle.decompress(s), data)
    got, st = ctx.decompress(gmp.DeviceStream(s))
    assert st == 0 and np.array_equal(got.cpu().numpy(), data)


@pytest.mark.parametrize("byte_mode", [False, True])
@pytest.mark.parametrize("mode", ["mrr", "de"])
@pytest.mark.parametrize("name", ["text256m", "csv1g"])
def test_workloads(gmp, ctx, name, mode, byte_mode):
    w = datagen.WORKLOADS[name]
    data = w.data(5 * w.block_size + 4321)
    de = mode == "de"
    s = gmp.compress_gpu(data, w.block_size, w.n_sub, w.window, de=de, byte_mode=byte_mode)
    check(gmp, ctx, s, data, de)
    # a real compressor: the ratio is within reach of the host compressor's
    ref = gmp.compress(data, w.block_size, w.n_sub, w.window, de=de, byte_mode=byte_mode)
    assert s.size < 1.35 * ref.size
    # deterministic
    assert np.array_equal(gmp.compress_gpu(data, w.block_size, w.n_sub, w.window, de=de, byte_mode=byte_mode), s)
    t = gmp.compress_gpu_times()
    assert t["match_ms"] > 0 and t["parse_ms"] > 0 and t["encode_ms"] > 0 and t["compressed_bytes"] == s.size


@pytest.mark.parametrize("cwl", [9, 10, 12])
def test_code_length_limit(gmp, ctx, cwl):
    """Skewed symbol frequencies whose unconstrained Huffman code is deeper
    than the limit: the lengths are cut to cwl bits and stay complete."""
    rng = np.random.default_rng(cwl)
    # literal frequencies falling geometrically (depth ~ 20 unconstrained)
    p = 0.6 ** np.arange(64)
    data = rng.choice(64, size=400_000, p=p / p.sum()).astype(np.uint8)
    for de in (False, True):
        s = gmp.compress_gpu(data, 64 * KiB, 16, 8 * KiB, cwl=cwl, de=de)
        rep = oracle.validate(s)
        assert rep["rc"] == 0 and rep["kraft_ok"] and rep["lengths_ok"], rep
        assert np.array_equal(oracle.decompress(s), data)
        got, st = ctx.decompress(gmp.DeviceStream(s))
        assert st == 0 and np.array_equal(got.cpu().numpy(), data)


@pytest.mark.parametrize("size", [0, 1, 2, 3, 31, 32, 33, 1000, 65535, 65536, 65537, 200_003])
def test_sizes(gmp, ctx, size):
    data = datagen.markov_text(size, seed=size + 9, order=2) if size else np.zeros(0, np.uint8)
    for byte_mode in (False, True):
        for de in (False, True):
            s = gmp.compress_gpu(data, 64 * KiB, 16, 8 * KiB, de=de, byte_mode=byte_mode)
            check(gmp, ctx, s, data, de)


def test_degenerate_data_and_small_parameters(gmp, ctx):
    rng = np.random.default_rng(11)
    rnd = rng.integers(0, 256, 300_000).astype(np.uint8)       # literal strings over 1023 bytes
    zeros = np.zeros(300_000, np.uint8)                         # distance-1 matches
    two = np.tile(np.frombuffer(b"ab", np.uint8), 150_000)
    for data in (rnd, zeros, two):
        for byte_mode in (False, True):
            for de in (False, True):
                s = gmp.compress_gpu(data, 128 * KiB, 32, 32 * KiB, de=de, byte_mode=byte_mode)
                check(gmp, ctx, s, data, de)
    data = datagen.csv_records(100_000, seed=4)
    for bs, win, mm in [(1000, 1, 64), (4093, 4096, 3), (12345, 257, 17)]:
        s = gmp.compress_gpu(data, bs, 4, win, max_match=mm)
        check(gmp, ctx, s, data, False)
