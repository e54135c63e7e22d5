"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
function include/gmp.h declares, parses stream headers and block indexes, and
its compressor writes streams that the oracle validates and decodes back to
the input."""
import ctypes
import os
import re

import numpy as np
import pytest

import datagen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "gmp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gmp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_00519_gb300 import _native
    _native.build()
    return _native.lib()


def test_library_exports_every_declared_function(lib):
    names = _declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.gpu
def test_decode_kernel_is_compiled_for_sm103(lib):
    """The runtime's own report of the loaded kernel's code: machine code and
    virtual architecture both 10.3 (a library built for another arch would
    report that arch, or fail to load the kernel at all)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    b, p = ctypes.c_int(), ctypes.c_int()
    assert lib.gmp_kernel_arch(ctypes.byref(b), ctypes.byref(p)) == 0, lib.gmp_last_cuda_error()
    assert b.value == 103 and p.value == 103, (b.value, p.value)


def test_compressor_streams_validate_and_roundtrip(lib):
    import paper_1606_00519_gb300 as gmp
    for name, w in datagen.WORKLOADS.items():
        data = w.data(3 * w.block_size + 777)
        for mode in w.modes:
            s = gmp.compress(data, w.block_size, w.n_sub, w.window, de=(mode == "de"))
            assert np.array_equal(oracle.decompress(s), data)
            r = oracle.validate(s)
            assert r["rc"] == 0 and r["kraft_ok"] and r["offsets_ok"] and r["subblocks_ok"] and r["blocks_ok"]
            if mode == "de":
                assert r["de_weak_ok"]


def test_compressor_byte_streams_validate_and_roundtrip(lib):
    import paper_1606_00519_gb300 as gmp
    rnd = np.random.default_rng(9).integers(0, 256, 5000).astype(np.uint8)  # literal strings over 1023 bytes
    for data in (datagen.csv_records(700_000, seed=5), datagen.markov_text(300_000, seed=6, order=3), rnd):
        for de in (False, True):
            s = gmp.compress(data, 64 * 1024, 16, 8192, de=de, byte_mode=True)
            info = gmp.stream_info(s)
            assert info.flags == (1 if de else 0) and info.n_sub == 0 and info.cwl == 0
            r = oracle.validate(s)
            assert r["rc"] == 0 and r["offsets_ok"] and r["blocks_ok"]
            assert np.array_equal(oracle.decompress(s), data)
            if de:
                assert r["de_weak_ok"]


def test_index_and_header_checks_for_byte_streams(lib):
    import paper_1606_00519_gb300 as gmp
    data = datagen.csv_records(300_000, seed=8)
    s = gmp.compress(data, 64 * 1024, 16, 8192, byte_mode=True)
    idx, info = gmp.index_build(s)
    assert info.n_blocks == 5 and info.n_sub == 0 and info.cwl == 0 and not info.flags & 2
    assert np.all(idx[:, 0] % 16 == 0) and list(idx[:, 3]) == [65536] * 4 + [300_000 - 4 * 65536]
    assert np.all(idx[:-1, 0] + idx[:-1, 1] == idx[1:, 0])
    # a Byte header must not claim sub-blocks or a code length limit
    for off, val in ((12, 16), (14, 12)):
        bad = s.copy()
        bad[off] = val
        with pytest.raises(gmp.GmpError):
            gmp.index_build(bad)
    # and a Huffman header must claim both
    h = gmp.compress(data, 64 * 1024, 16, 8192)
    bad = h.copy()
    bad[12:14] = 0
    with pytest.raises(gmp.GmpError):
        gmp.index_build(bad)


def test_host_compressor_options(lib):
    import paper_1606_00519_gb300 as gmp
    data = datagen.markov_text(400_000, seed=12, order=3)
    sizes = {}
    for lazy in (False, True):
        for depth in (1, 8, 64):
            s = gmp.compress(data, 128 * 1024, 32, 32768, chain_depth=depth, lazy=lazy)
            assert np.array_equal(oracle.decompress(s), data)
            sizes[(lazy, depth)] = s.size
    # deeper search and lazy evaluation never make this input larger
    assert sizes[(False, 64)] <= sizes[(False, 1)] and sizes[(True, 64)] <= sizes[(False, 64)]
    with pytest.raises(gmp.GmpError):
        gmp.compress(data, 128 * 1024, 32, 32768, cwl=8)  # 319 symbols need 9 bits


def test_encode_tokens_matches_oracle(lib):
    import paper_1606_00519_gb300 as gmp
    for m in (1, 4, 32):
        ts = datagen.nesting_tokens(seed=300 + m, m=m, n_inst=32 * 20)
        expect = oracle.lz77_decode(ts.lit_len, ts.mlen, ts.off, ts.lits, 32768)
        for byte_mode in (False, True):
            s = gmp.encode_tokens(ts.lit_len, ts.mlen, ts.off, ts.lits, n_sub=16, byte_mode=byte_mode)
            assert np.array_equal(oracle.decompress(s), expect)
            # the same parse: the oracle reads back exactly the sequences given
            got = oracle.block_tokens(s, 0)
            assert np.array_equal(got.mlen[got.mlen > 0], ts.mlen[ts.mlen > 0])
            assert np.array_equal(got.off[got.mlen > 0], ts.off[ts.mlen > 0])


def test_encode_tokens_rejects_bad_parses(lib):
    import paper_1606_00519_gb300 as gmp
    lits = np.frombuffer(b"abcdef", np.uint8)
    with pytest.raises(gmp.GmpError):  # distance before the block start
        gmp.encode_tokens([3, 3], [4, 0], [5, 0], lits)
    with pytest.raises(gmp.GmpError):  # match shorter than 3
        gmp.encode_tokens([3, 3], [2, 0], [1, 0], lits)
    with pytest.raises(gmp.GmpError):  # a Huffman block's sequence without a back-reference before the end
        gmp.encode_tokens([3, 3], [0, 0], [0, 0], lits)
    with pytest.raises(gmp.GmpError):  # literals left over
        gmp.encode_tokens([3, 2], [3, 0], [1, 0], lits)
    s = gmp.encode_tokens([3, 3], [0, 0], [0, 0], lits, byte_mode=True)  # fine in Byte blocks
    assert bytes(oracle.decompress(s)) == b"abcdef"


def test_compressor_tiny_inputs(lib):
    import paper_1606_00519_gb300 as gmp
    for data in (b"", b"x", b"xy", b"aaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaa", bytes(range(256)) * 3):
        for de in (False, True):
            s = gmp.compress(np.frombuffer(data, np.uint8), block_size=64, n_sub=4, window=32, de=de)
            assert bytes(oracle.decompress(s)) == data


def test_index_build_matches_header(lib):
    import paper_1606_00519_gb300 as gmp
    data = datagen.markov_text(300_000, seed=3, order=2)
    s = oracle.compress(data, oracle.params(65536, 16, 8192))
    idx, info = gmp.index_build(s)
    assert info.n_blocks == 5 and info.orig_size == 300_000 and info.n_sub == 16
    assert np.all(idx[:, 0] % 16 == 0)
    assert list(idx[:, 2]) == [0, 65536, 131072, 196608, 262144]
    assert list(idx[:, 3]) == [65536] * 4 + [300_000 - 4 * 65536]
    assert np.all(idx[:-1, 0] + idx[:-1, 1] == idx[1:, 0])
    assert 0 < info.max_block_seq <= 65536 // 3 + 1 and info.max_block_out == 65536


def test_index_build_rejects_bad_headers(lib):
    import paper_1606_00519_gb300 as gmp
    s = oracle.compress(datagen.markov_text(50_000, seed=1), oracle.params(16384, 8, 4096))
    bad = s.copy()
    bad[0:4] = np.frombuffer(b"XXXX", np.uint8)
    with pytest.raises(gmp.GmpError):
        gmp.index_build(bad)
    bad = s.copy()
    bad[64:72] = np.frombuffer(np.uint64(3).tobytes(), np.uint8)  # misaligned block offset
    with pytest.raises(gmp.GmpError):
        gmp.index_build(bad)
    with pytest.raises(gmp.GmpError):
        gmp.index_build(s[:40])


def test_decode_calls_fail_loudly_without_gpu(lib):
    import torch
    import paper_1606_00519_gb300 as gmp
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        gmp.Context()


def test_entry_points_reject_null_arguments(lib):
    # argument checks come before any CUDA call, so they hold on a machine
    # without a GPU: a null context or null buffers give GMP_ERR_INVALID_ARG
    INVALID = -1
    z = ctypes.c_size_t(0)
    assert lib.gmp_decompress(None, None, 0, None, 0, None, 0, None, None) == INVALID
    assert lib.gmp_decompress_batch(None, None, 1, None, None) == INVALID
    assert lib.gmp_decompress_host_batch(None, 1, None, None, None, None, None, None) == INVALID
    assert lib.gmp_decompress_from_host_batch(None, 1, None, None, None, None, None, None) == INVALID
    assert lib.gmp_decompress_host(None, None, 0, None, 0, None, None) == INVALID
    assert lib.gmp_stats_reset(None, None) == INVALID
    assert lib.gmp_context_set_input_wait(None, ctypes.c_uint32(100)) == INVALID
    assert lib.gmp_context_debug_drop_input_flag(None, ctypes.c_int64(0)) == INVALID
    assert lib.gmp_index_build(None, 0, None, 0, ctypes.byref(z), None) == INVALID


@pytest.mark.parametrize("name,cls,expect", [
    ("gmp_context_opts_default", "ContextOpts",
     dict(max_block_out=256 << 10, warps_per_cta=0, ctas_per_sm=0, collect_stats=0, max_files=65536, resolve=0,
          concurrent=0)),
    ("gmp_server_opts_default", "ServerOpts", None),
    ("gmp_compress_opts_default", "CompressOpts", None),
])
def test_option_structs_match_the_binding(lib, name, cls, expect):
    # the C default-setter writes every field of the binding's struct (each
    # starts as a 0xAB pattern) and nothing past its end, so the two layouts
    # have the same size and fields
    from paper_1606_00519_gb300 import _native
    S = getattr(_native, cls)
    size = ctypes.sizeof(S)
    buf = (ctypes.c_uint8 * (size + 64))(*([0xAB] * (size + 64)))
    getattr(lib, name)(ctypes.cast(buf, ctypes.POINTER(S)))
    assert bytes(buf[size:]) == b"\xab" * 64
    o = S.from_buffer(buf)
    for f, t in S._fields_:
        v = getattr(o, f)
        pattern = int.from_bytes(b"\xab" * ctypes.sizeof(t), "little")
        assert v != pattern, f"{cls}.{f} not written by {name}"
        if expect is not None:
            assert v == expect[f], (f, v)
