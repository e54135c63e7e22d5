"""GPU autotuning: the launch-shape tuner picks a valid shape and the decoder
stays byte-exact under it; the format tuner returns a candidate of its grid
and respects the ratio bound; results are cached."""
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


def test_launch_shape_autotune_keeps_output_exact(gmp):
    import torch
    data = datagen.csv_records(6 * MiB, seed=44)
    s = gmp.compress(data, 256 * KiB, 32, 32 * KiB, de=True)
    ds = gmp.DeviceStream(s)
    out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    table = gmp.make_file_table([ds.file_desc(out)])
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx = gmp.Context(max_block_out=256 * KiB)
    t = ctx.autotune(table, 1, status)
    assert t["warps_per_cta"] in (1, 2, 4, 8, 16) and t["ctas_per_sm"] >= 1 and t["shapes_tried"] >= 4
    assert t["best_ms"] > 0
    got, st = ctx.decompress(ds)
    assert st == 0 and np.array_equal(got.cpu().numpy(), data)
    ctx.close()


def test_format_tuner_and_cache(gmp, tmp_path):
    from paper_1606_00519_gb300 import autotune
    data = datagen.markov_text(4 * MiB, seed=3, order=3)
    res = autotune.tune(data, cache_path=str(tmp_path / "tune.json"), block_sizes=(64 * KiB, 256 * KiB),
                        n_subs=(16, 32), repeats=2)
    assert res["block_size"] in (64 * KiB, 256 * KiB) and res["n_sub"] in (16, 32)
    assert not res["cached"]
    again = autotune.tune(data, cache_path=str(tmp_path / "tune.json"), block_sizes=(64 * KiB, 256 * KiB),
                          n_subs=(16, 32), repeats=2)
    assert again["cached"] and again["block_size"] == res["block_size"]
    # the chosen format still round-trips through the oracle
    s = gmp.compress(data, res["block_size"], res["n_sub"], 32 * KiB, de=True)
    assert np.array_equal(oracle.decompress(s), data)
