"""CPU checks of the seeded synthetic inputs against their stated recipe: the
Markov text (English-like letters, about 18 % spaces, a little noise outside
letters and punctuation, compression ratio near the calibrated 2.5-3), the CSV-like
rows (8 fields: two integer ids below 1e6, two prices with 2 decimals, two
ISO dates in a 5-year range, two of 20 lowercase tokens), the nesting-depth
token streams, the batched file mix (log-uniform sizes) and the Poisson
arrivals; every generator is deterministic in its seed."""
import re

import numpy as np

import datagen
import oracle

KiB, MiB = 1 << 10, 1 << 20


def test_generators_are_deterministic_in_the_seed():
    for f in (lambda s: datagen.markov_text(50_000, s, order=2), lambda s: datagen.markov_text(50_000, s, order=3),
              lambda s: datagen.csv_records(50_000, s)):
        a, b, c = f(7), f(7), f(8)
        assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert datagen.file_mix(4, 100) == datagen.file_mix(4, 100)
    t1, t2 = datagen.nesting_tokens(3, 4, 320), datagen.nesting_tokens(3, 4, 320)
    assert np.array_equal(t1.lits, t2.lits) and np.array_equal(t1.off, t2.off)


def test_markov_text_letter_statistics_and_ratio():
    for order, name in ((2, "text1m"), (3, "text256m")):
        data = datagen.markov_text(1 * MiB, seed=11, order=order)
        hist = np.bincount(data, minlength=256) / data.size
        assert 0.10 < hist[ord(" ")] < 0.26                   # spaces
        letters = hist[ord("a"):ord("z") + 1].sum()
        assert letters > 0.6                                  # mostly lowercase letters
        # noise: about 1.5 % of the bytes lie outside letters, space and
        # punctuation (the sampling table quantises the noise floor, so only
        # part of the 256 values occur)
        base = set(range(ord("a"), ord("z") + 1)) | set(range(ord("A"), ord("Z") + 1)) | {32, 44, 46, 10}
        other = sum(hist[i] for i in range(256) if i not in base)
        assert 0.003 < other < 0.04 and np.count_nonzero(hist) > 60
        w = datagen.WORKLOADS[name]
        s = oracle.compress(data, oracle.params(w.block_size, w.n_sub, w.window))
        ratio = data.size / s.size
        assert 2.3 < ratio < 3.2, ratio


def test_csv_rows_have_the_stated_fields():
    data = datagen.csv_records(400_000, seed=12)
    text = bytes(data).decode("ascii")
    rows = text.split("\n")[1:-1]  # the first and last rows may be cut by the size
    assert len(rows) > 3000
    tokens = set()
    year_lo, year_hi = 10_000, 0
    pat = re.compile(r"^(\d+),(\d+),(\d+)\.(\d\d),(\d+)\.(\d\d),(\d{4})-(\d\d)-(\d\d),(\d{4})-(\d\d)-(\d\d),"
                     r"([a-z]{4,12}),([a-z]{4,12})$")
    for r in rows:
        m = pat.match(r)
        assert m, r
        g = m.groups()
        assert int(g[0]) < 1_000_000 and int(g[1]) < 1_000_000
        for y, mo, d in ((g[6], g[7], g[8]), (g[9], g[10], g[11])):
            assert 1 <= int(mo) <= 12 and 1 <= int(d) <= 31
            year_lo, year_hi = min(year_lo, int(y)), max(year_hi, int(y))
        tokens.update(g[12:14])
    assert year_hi - year_lo <= 5
    assert 10 <= len(tokens) <= 20
    # about 10 % of the rows repeat a recent row with one field changed
    repeats = 0
    seen = []
    for r in rows:
        f = r.split(",")
        if any(sum(a != b for a, b in zip(f, p)) == 1 for p in seen[-64:]):
            repeats += 1
        seen.append(f)
    assert 0.05 < repeats / len(rows) < 0.2, repeats / len(rows)


def test_nesting_tokens_depth_and_lengths():
    for m in (1, 2, 4, 8, 16, 32):
        ts = datagen.nesting_tokens(seed=m, m=m, n_inst=32 * 10)
        out = oracle.lz77_decode(ts.lit_len, ts.mlen, ts.off, ts.lits)
        assert out.size == ts.out_bytes
        rounds = oracle.mrr_rounds(ts.lit_len, ts.mlen, ts.off, ts.lits)
        assert int(rounds.max()) == 32 // m
        assert set(np.unique(ts.mlen[ts.mlen > 0])) == {15} and set(np.unique(ts.off[ts.mlen > 0])) == {17 * m}


def test_file_mix_sizes_are_log_uniform():
    mix = datagen.file_mix(seed=4, n_files=4096, lo=4 * KiB, hi=16 * MiB)
    sizes = np.array([m[0] for m in mix], dtype=np.float64)
    assert sizes.size == 4096 and sizes.min() >= 4 * KiB and sizes.max() <= 16 * MiB
    # log-uniform: the log sizes are uniform, so their quartiles are evenly spaced
    q = np.quantile(np.log(sizes), [0.25, 0.5, 0.75])
    span = np.log(16 * MiB) - np.log(4 * KiB)
    expect = np.log(4 * KiB) + span * np.array([0.25, 0.5, 0.75])
    assert np.all(np.abs(q - expect) < 0.05 * span)
    kinds = {m[1] for m in mix}
    modes = {m[2] for m in mix}
    assert kinds == {"text3", "csv"} and modes == {"mrr", "de"}
    cut = datagen.file_mix(seed=4, n_files=4096, lo=4 * KiB, hi=16 * MiB, total_cap=1 << 30)
    assert cut == mix[:len(cut)] and sum(m[0] for m in cut) <= 1 << 30


def test_poisson_arrivals_rate():
    t = datagen.poisson_arrivals(seed=5, n=20_000, rate_per_s=1000.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1e-3) < 0.05e-3           # mean inter-arrival 1 / rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential: coefficient of variation 1
