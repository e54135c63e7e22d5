"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the paper's
worked examples (golden fixtures with citations), closed forms, a textbook
Huffman construction, brute force on tiny inputs, and round trips on seeded
synthetic data.  No GPU is needed.
"""
import heapq
import itertools

import numpy as np
import pytest

import datagen
import oracle
from conftest import read_golden, read_golden_rows


def _ints(s):
    return [int(x) for x in s.split()]


# ---------------------------------------------------------------- Fig. 1

def test_fig1_example_decodes():
    g = read_golden("fig1_lz77_example.txt")
    out = oracle.lz77_decode(_ints(g["lit_len"]), _ints(g["mlen"]), _ints(g["off"]),
                             np.frombuffer(g["lits"].encode(), np.uint8))
    assert bytes(out) == g["expect"].encode()


def test_fig1_example_roundtrips_through_a_stream():
    g = read_golden("fig1_lz77_example.txt")
    ts = datagen.TokenStream(np.array(_ints(g["lit_len"]), np.uint32), np.array(_ints(g["mlen"]), np.uint32),
                             np.array(_ints(g["off"]), np.uint32), np.frombuffer(g["lits"].encode(), np.uint8))
    s = oracle.encode_tokens(ts, oracle.params(block_size=64, n_sub=1, window=8))
    assert bytes(oracle.decompress(s)) == g["expect"].encode()


# ---------------------------------------------------------------- MRR (Sec. 4.1)

def test_mrr_three_sequence_example_takes_two_rounds():
    g = read_golden("mrr_three_sequences.txt")
    args = (_ints(g["lit_len"]), _ints(g["mlen"]), _ints(g["off"]), np.frombuffer(g["lits"].encode(), np.uint8))
    assert bytes(oracle.lz77_decode(*args)) == g["expect"].encode()
    rounds = oracle.mrr_rounds(*args)
    assert list(rounds) == [int(g["rounds"])]
    # the one-pass DE schedule must refuse this stream (T2, T3 depend on T1)
    with pytest.raises(oracle.OracleError):
        oracle.mrr_rounds(*args, de_single_pass=True)


def test_mrr_independent_references_take_one_round():
    # Sec. 4.1: back-references that do not depend on data produced by other
    # back-references of the same warp resolve in one round.
    rng = np.random.default_rng(7)
    lits = rng.integers(0, 256, 4096).astype(np.uint8)
    ll = np.full(32, 64, np.uint32)
    ll[0] = 2048
    ml = np.full(32, 8, np.uint32)
    # every copy reads from the first literal string only
    pos = np.cumsum(ll + ml) - ml  # write positions
    off = (pos - rng.integers(0, 2000, 32)).astype(np.uint32)
    rounds = oracle.mrr_rounds(ll, ml, off, lits[:int(ll.sum())])
    assert list(rounds) == [1]


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32])
def test_nesting_depth_rounds(m):
    # Sec. 5.1: one repeated string gives nesting depth 32 (32 rounds), two
    # strings 16, four 8, and so on.
    ts = datagen.nesting_tokens(seed=11 + m, m=m, n_inst=32 * 8)
    rounds = oracle.mrr_rounds(ts.lit_len, ts.mlen, ts.off, ts.lits)
    full = [r for i, r in enumerate(rounds) if (i + 1) * 32 <= ts.n_seq]
    assert full and all(r == 32 // m for r in full), rounds


@pytest.mark.parametrize("m", [1, 2, 8])
def test_nesting_data_has_the_described_shape(m):
    # 17-byte instances: a digit separator, then a 16-letter string that
    # differs from the previous instance of the same string in one byte,
    # alternately the first and the last.
    ts = datagen.nesting_tokens(seed=5, m=m, n_inst=200)
    data = bytes(oracle.lz77_decode(ts.lit_len, ts.mlen, ts.off, ts.lits))
    assert len(data) == 17 * (m + 200)
    inst = [data[17 * k:17 * k + 17] for k in range(m + 200)]
    assert all(x[0:1].isdigit() and x[1:].isalpha() for x in inst)
    for k in range(m, m + 200):
        a, b = inst[k - m][1:], inst[k][1:]
        diff = [i for i in range(16) if a[i] != b[i]]
        assert diff == ([0] if (k // m) % 2 else [15])


# ---------------------------------------------------------------- offset code

def test_offset_code_matches_deflate_table():
    for sym, ne, lo, hi in read_golden_rows("deflate_distance_codes.txt"):
        assert oracle.offset_nextra(sym) == ne
        for d in {lo, hi, (lo + hi) // 2}:
            s, n, e = oracle.offset_encode(d)
            assert (s, n) == (sym, ne) and 0 <= e < (1 << n)
            assert oracle.offset_decode(s, e) == d
        assert oracle.offset_decode(sym, 0) == lo
        assert oracle.offset_decode(sym, (1 << ne) - 1) == hi


def test_offset_code_roundtrip_all():
    prev = -1
    for d in range(1, 32769):
        s, n, e = oracle.offset_encode(d)
        assert s >= prev and s < 30
        prev = s
        assert oracle.offset_decode(s, e) == d
    with pytest.raises(oracle.OracleError):
        oracle.offset_encode(0)
    with pytest.raises(oracle.OracleError):
        oracle.offset_encode(32769)


# ---------------------------------------------------------------- Huffman

def test_canonical_codes_rfc1951_example():
    g = read_golden("canonical_rfc1951.txt")
    lengths = _ints(g["lengths"])
    codes = [int(c, 2) for c in g["codes"].split()]
    assert list(oracle.canonical_codes(lengths)) == codes


def _huffman_cost(freq):
    """Textbook Huffman (heap merge): total cost sum(f * depth)."""
    f = [x for x in freq if x > 0]
    if len(f) <= 1:
        return sum(f)
    h = list(f)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def _max_huffman_depth(freq):
    f = [(x, i) for i, x in enumerate(freq) if x > 0]
    h = [(w, i, 0) for w, i in f]
    heapq.heapify(h)
    k = len(f)
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        heapq.heappush(h, (a[0] + b[0], k, max(a[2], b[2]) + 1))
        k += 1
    return h[0][2]


def test_package_merge_equals_huffman_when_unconstrained():
    rng = np.random.default_rng(3)
    for trial in range(60):
        n = int(rng.integers(2, 320))
        freq = rng.integers(0, 1000, n) * (rng.random(n) < 0.8)
        if (freq > 0).sum() < 2:
            continue
        if _max_huffman_depth(freq) > 12:
            continue
        ln = oracle.package_merge(freq, 12)
        cost = int((ln.astype(np.int64) * freq).sum())
        assert cost == _huffman_cost(freq), trial


def test_package_merge_is_optimal_by_brute_force():
    rng = np.random.default_rng(4)
    for trial in range(40):
        n = int(rng.integers(2, 7))
        limit = int(rng.integers(max(1, (n - 1).bit_length()), 5))
        freq = rng.integers(1, 50, n)
        freq[0] = 1000  # skewed, so the limit binds
        ln = oracle.package_merge(freq, limit)
        assert ln.max() <= limit
        assert oracle.kraft_scaled(ln, limit) == 1 << limit
        best = min(sum(int(f) * l for f, l in zip(freq, ls))
                   for ls in itertools.product(range(1, limit + 1), repeat=n)
                   if sum(2 ** (limit - l) for l in ls) <= 2 ** limit)
        assert int((ln.astype(np.int64) * freq).sum()) == best, (freq, limit)


def test_package_merge_kraft_equality_and_limit():
    rng = np.random.default_rng(5)
    for trial in range(100):
        n = int(rng.integers(2, 320))
        freq = (rng.pareto(0.7, n) * 10).astype(np.int64) * (rng.random(n) < 0.9)
        if (freq > 0).sum() < 2:
            freq[:2] = [1, 1]
        for limit in (9, 10, 12):
            if (freq > 0).sum() > (1 << limit):
                continue
            ln = oracle.package_merge(freq, limit)
            assert ln.max() <= limit
            assert np.all((ln > 0) == (freq > 0))
            assert oracle.kraft_scaled(ln, limit) == 1 << limit


def test_single_symbol_alphabet_gets_a_dummy():
    ln = oracle.package_merge([0, 0, 5, 0], 12)
    assert list(ln) == [1, 0, 1, 0]
    ln = oracle.package_merge([7, 0, 0], 12)
    assert list(ln) == [1, 1, 0]


def test_canonical_codes_are_prefix_free_and_ordered():
    rng = np.random.default_rng(6)
    for trial in range(30):
        n = int(rng.integers(2, 320))
        freq = rng.integers(1, 10000, n)
        ln = oracle.package_merge(freq, 12)
        codes = oracle.canonical_codes(ln)
        words = sorted((format(int(c), f"0{int(l)}b"), s) for s, (c, l) in enumerate(zip(codes, ln)))
        for (a, _), (b, _) in zip(words, words[1:]):
            assert not b.startswith(a)
        # canonical: ordered by (length, symbol) means codes increase in that order
        order = sorted(range(n), key=lambda s: (ln[s], s))
        vals = [int(codes[s]) << (12 - int(ln[s])) for s in order]
        assert vals == sorted(vals) and len(set(vals)) == n


# ---------------------------------------------------------------- round trips

@pytest.mark.parametrize("name", ["text1m", "text256m", "csv1g"])
def test_roundtrip_and_validators(name):
    w = datagen.WORKLOADS[name]
    data = w.data(w.block_size * 3 + 1234)  # several blocks and a ragged tail
    for mode in w.modes:
        p = oracle.params(w.block_size, w.n_sub, w.window, de=(mode == "de"))
        s = oracle.compress(data, p)
        assert np.array_equal(oracle.decompress(s), data)
        r = oracle.validate(s)
        assert r["rc"] == 0
        for k in ("kraft_ok", "lengths_ok", "offsets_ok", "blocks_ok", "subblocks_ok", "subblocks_even", "mrr_ok"):
            assert r[k] == 1, k
        assert r["n_blocks"] == 4
        if mode == "de":
            assert r["de_weak_ok"] == 1
        # every block is decodable on its own
        for b in range(r["n_blocks"]):
            lo = b * w.block_size
            assert np.array_equal(oracle.decompress_block(s, b), data[lo:lo + w.block_size])


def test_empty_and_tiny_inputs():
    p = oracle.params(block_size=16, n_sub=4, window=8)
    for data in (b"", b"a", b"ab", b"aaaa", b"abcabcabcabcabcabc"):
        s = oracle.compress(np.frombuffer(data, np.uint8), p)
        info = oracle.stream_info(s)
        assert info.orig_size == len(data)
        assert bytes(oracle.decompress(s)) == data


def test_stream_shape():
    data = datagen.markov_text(100_000, seed=9, order=2)
    p = oracle.params(block_size=16384, n_sub=8, window=4096)
    s = oracle.compress(data, p)
    info = oracle.stream_info(s)
    assert s[:4].tobytes() == b"GMP1"
    assert info.n_blocks == 7 and info.orig_size == 100_000 and info.stream_bytes == s.size
    offs = s[64:64 + 8 * 7].view(np.uint64)
    assert np.all(offs % 16 == 0) and np.all(np.diff(offs.astype(np.int64)) > 0)
    assert np.all(s[-16:] == 0)


def test_corruptions_are_reported():
    data = datagen.markov_text(40_000, seed=10, order=2)
    s = oracle.compress(data, oracle.params(block_size=16384, n_sub=8, window=4096))
    assert oracle.decompress_status(s) == oracle.OK
    bad = s.copy()
    bad[0] ^= 1  # magic
    assert oracle.decompress_status(bad) == oracle.BAD_HEADER
    # flip a bit in the middle of a bitstream: any error code, never silent success
    rng = np.random.default_rng(1)
    hits = 0
    for _ in range(40):
        bad = s.copy()
        i = int(rng.integers(int(s[64:72].view(np.uint64)[0]) + 400, s.size - 32))
        bad[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        # a flip can also turn one literal into another of the same code
        # length (the format has no checksum); most flips must be detected
        if oracle.decompress_status(bad) != oracle.OK:
            hits += 1
    assert hits >= 8


# ---------------------------------------------------------------- Gompresso/Byte

@pytest.mark.parametrize("name", ["text1m", "text256m", "csv1g"])
def test_byte_mode_roundtrip_and_validators(name):
    # Sec. 3.1 / 3.2: byte-level encoding without Huffman trees, same LZ77
    w = datagen.WORKLOADS[name]
    data = w.data(3 * w.block_size + 321)
    for de in (False, True):
        s = oracle.compress(data, oracle.params(w.block_size, 1, w.window, de=de, byte_mode=True))
        info = oracle.stream_info(s)
        assert not (info.flags & 2) and info.n_sub == 0 and info.cwl == 0
        assert np.array_equal(oracle.decompress(s), data)
        r = oracle.validate(s)
        assert r["rc"] == 0 and r["offsets_ok"] and r["mrr_ok"] and r["blocks_ok"]
        if de:
            assert r["de_weak_ok"]


def test_byte_record_layout_fig1():
    # The Fig. 1 sequence (3 literals, copy of 3 bytes at distance 3) as one
    # Byte record: literal length in bits 0-9, match code m = length - 2 in
    # bits 10-15, distance - 1 in bits 16-31.
    g = read_golden("fig1_lz77_example.txt")
    ts = datagen.TokenStream(np.array(_ints(g["lit_len"]), np.uint32), np.array(_ints(g["mlen"]), np.uint32),
                             np.array(_ints(g["off"]), np.uint32), np.frombuffer(g["lits"].encode(), np.uint8))
    s = oracle.encode_tokens(ts, oracle.params(block_size=64, n_sub=1, window=8, byte_mode=True))
    bo = int(s[64:72].view(np.uint64)[0])
    n_seq, out_bytes, n_lit = (int(x) for x in s[bo:bo + 12].view(np.uint32))
    assert (n_seq, out_bytes, n_lit) == (1, 6, 3)
    assert int(s[bo + 16:bo + 20].view(np.uint32)[0]) == 3 | ((3 - 2) << 10) | ((3 - 1) << 16)
    assert bytes(s[bo + 32:bo + 35]) == b"aac"
    assert bytes(oracle.decompress(s)) == g["expect"].encode()


def test_byte_mode_long_literal_runs():
    rng = np.random.default_rng(12)
    data = rng.integers(0, 256, 200_000).astype(np.uint8)  # incompressible: long literal runs
    s = oracle.compress(data, oracle.params(65536, 1, 8192, byte_mode=True))
    assert np.array_equal(oracle.decompress(s), data)
    for b in range(oracle.stream_info(s).n_blocks):
        t = oracle.block_tokens(s, b)
        assert t.lit_len.max() <= 1023
