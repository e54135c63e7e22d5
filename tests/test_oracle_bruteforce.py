"""Brute force over every tiny input: the oracle's compressor must round-trip
and keep the window, block and DE rules (Sec. 3.1, Sec. 4.2) for every string
up to length 14 over {a, b} and up to length 9 over {a, b, c}."""
import itertools

import numpy as np
import pytest

import oracle


def _all_strings(alphabet, max_len):
    for n in range(1, max_len + 1):
        for t in itertools.product(alphabet, repeat=n):
            yield "".join(t).encode()


@pytest.mark.parametrize("alphabet,max_len", [("ab", 14), ("abc", 9)])
@pytest.mark.parametrize("block_size", [16, 8])
@pytest.mark.parametrize("byte_mode", [False, True])
def test_every_tiny_input(alphabet, max_len, block_size, byte_mode):
    p_mrr = oracle.params(block_size=block_size, n_sub=3, window=8, byte_mode=byte_mode)
    p_de = oracle.params(block_size=block_size, n_sub=3, window=8, de=True, byte_mode=byte_mode)
    n_matches = 0
    for data in _all_strings(alphabet, max_len):
        arr = np.frombuffer(data, np.uint8)
        for p in (p_mrr, p_de):
            s = oracle.compress(arr, p)
            assert bytes(oracle.decompress(s)) == data
            r = oracle.validate(s)
            assert r["rc"] == 0 and r["offsets_ok"] and r["kraft_ok"] and r["blocks_ok"] and r["mrr_ok"]
            assert r["subblocks_ok"] and (byte_mode or r["subblocks_even"])
            if p.de:
                assert r["de_weak_ok"], data
            n_matches += r["n_matches"]
    assert n_matches > 0
