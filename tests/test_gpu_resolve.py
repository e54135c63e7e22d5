"""GPU tests of the back-reference resolution strategies (Sec. 4 and the
ablation of Sec. 5.1): Sequential Copying, Multi-Round Resolution forced on
any stream, and the default (DE streams in one pass) all give the oracle's
bytes; their round counts and the bytes-per-round statistics match what the
strategy and the stream fix."""
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
def ctxs(gmp):
    cs = {r: gmp.Context(max_block_out=256 * KiB, collect_stats=True, resolve=r) for r in ("auto", "mrr", "sc")}
    yield cs
    for c in cs.values():
        c.close()


def decode(gmp, ctx, stream):
    ctx.stats_reset()
    out, status = ctx.decompress(gmp.DeviceStream(stream))
    return out.cpu().numpy(), status, ctx.stats()


@pytest.mark.parametrize("byte_mode", [False, True])
@pytest.mark.parametrize("mode", ["mrr", "de"])
def test_strategies_give_the_oracle_bytes(gmp, ctxs, byte_mode, mode):
    for name in ("text256m", "csv1g"):
        w = datagen.WORKLOADS[name]
        data = w.data(3 * w.block_size + 1234)
        s = gmp.compress(data, w.block_size, w.n_sub, w.window, de=(mode == "de"), byte_mode=byte_mode)
        expect = oracle.decompress(s)
        assert np.array_equal(expect, data)
        rep = oracle.validate(s)
        for r, c in ctxs.items():
            got, st, stats = decode(gmp, c, s)
            assert st == 0 and np.array_equal(got, expect), (name, r)
            # every back-reference byte is copied exactly once, in some round
            assert sum(stats["round_bytes"]) == rep["match_bytes"], (name, r)
            if r == "sc":
                # one back-reference per round
                assert stats["rounds"] == rep["n_matches"]
            elif r == "mrr" or mode == "mrr":
                # MRR resolves at least one back-reference per round
                assert stats["groups"] <= stats["rounds"] <= rep["n_matches"]
            else:
                assert stats["rounds"] == stats["groups"] and stats["max_rounds"] == 1


@pytest.mark.parametrize("m", [1, 2, 8, 32])
@pytest.mark.parametrize("byte_mode", [False, True])
def test_nesting_depth_rounds_and_bytes_per_round(gmp, ctxs, m, byte_mode):
    ts = datagen.nesting_tokens(seed=400 + m, m=m, n_inst=32 * 50)
    s = gmp.encode_tokens(ts.lit_len, ts.mlen, ts.off, ts.lits, n_sub=32, byte_mode=byte_mode)
    expect = oracle.lz77_decode(ts.lit_len, ts.mlen, ts.off, ts.lits)
    rounds = oracle.mrr_rounds(ts.lit_len, ts.mlen, ts.off, ts.lits)
    got, st, stats = decode(gmp, ctxs["mrr"], s)
    assert st == 0 and np.array_equal(got, expect)
    assert stats["rounds"] == int(rounds.sum()) and stats["max_rounds"] == 32 // m
    # depth 32 / m: in each of the first 32 / m rounds every group copies m
    # back-references (the first group's first round also copies the ones
    # that need nothing from the group)
    n_full = int(np.sum(rounds == 32 // m))
    depth = 32 // m
    for r in range(min(depth, 8)):
        assert stats["round_groups"][r] >= n_full
    got, st, stats = decode(gmp, ctxs["sc"], s)
    assert st == 0 and np.array_equal(got, expect)
    assert stats["rounds"] == int(np.count_nonzero(ts.mlen))


def test_sc_on_overlapping_and_far_copies(gmp, ctxs):
    zeros = np.zeros(400_000, np.uint8)  # distance-1 copies
    rnd = np.random.default_rng(3).integers(0, 256, 300_000).astype(np.uint8)
    mixed = np.concatenate([rnd[:100_000], datagen.csv_records(300_000, seed=2), rnd[:100_000]])
    for data in (zeros, mixed):
        for de in (False, True):
            s = gmp.compress(data, 256 * KiB, 32, 32 * KiB, de=de)
            for r in ("mrr", "sc"):
                got, st, _ = decode(gmp, ctxs[r], s)
                assert st == 0 and np.array_equal(got, data)



@pytest.mark.parametrize("byte_mode", [False, True])
def test_chain_of_exactly_adjacent_copies(gmp, ctxs, byte_mode):
    # each copy's source is exactly the previous copy's output (distance =
    # previous copy's length + one literal): every 32-sequence group is a
    # dependency chain of depth 32, the worst case for MRR
    n = 32 * 40
    ll = np.ones(n, np.uint32)
    ml = np.full(n, 16, np.uint32)
    off = np.full(n, 17, np.uint32)
    ll[0] = 17  # the first copy takes 16 of the first 17 literals
    lits = np.random.default_rng(9).integers(0, 256, int(ll.sum())).astype(np.uint8)
    s = gmp.encode_tokens(ll, ml, off, lits, n_sub=32, byte_mode=byte_mode)
    expect = oracle.lz77_decode(ll, ml, off, lits)
    rounds = oracle.mrr_rounds(ll, ml, off, lits)
    for r in ("auto", "mrr"):
        got, st, stats = decode(gmp, ctxs[r], s)
        assert st == 0 and np.array_equal(got, expect), r
        assert stats["rounds"] == int(rounds.sum()) and stats["max_rounds"] == 32, r
        assert sum(stats["round_bytes"]) == int(ml.sum()), r
        # rounds after the 8th land in the last bin
        assert stats["round_groups"] == [n // 32] * 7 + [25 * (n // 32)], r
    got, st, stats = decode(gmp, ctxs["sc"], s)
    assert st == 0 and np.array_equal(got, expect) and stats["rounds"] == n
