"""GPU parity at the benchmark's full sizes and launch configuration: the
256 MiB text and 1 GiB CSV workloads, MRR and DE streams from the product
compressor, decoded in one batched launch under the launch shape the
autotuner picks (as bench.py does) and under both kernel register budgets.
Every output byte is compared with the input, and a sample of blocks with
the oracle's own decode of each block."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(1200, method="thread")]

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


def _check_full(gmp, name, byte_mode=False, shapes=("tuned",)):
    import torch
    w = datagen.WORKLOADS[name]
    data = w.data()
    streams = [gmp.compress(data, w.block_size, w.n_sub, w.window, de=de, byte_mode=byte_mode) for de in (False, True)]
    ds = [gmp.DeviceStream(s) for s in streams]
    outs = [torch.empty(data.size, dtype=torch.uint8, device="cuda") for _ in ds]
    table = gmp.make_file_table([d.file_desc(o) for d, o in zip(ds, outs)])
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    ref = torch.from_numpy(data).cuda()
    rng = np.random.default_rng(len(name))
    for shape in shapes:
        if shape == "tuned":
            ctx = gmp.Context(max_block_out=w.block_size)
            ctx.autotune(table, 2, status)
        else:
            ctx = gmp.Context(max_block_out=w.block_size, warps_per_cta=shape[0], ctas_per_sm=shape[1])
        for o in outs:
            o.fill_(0xA5)
        ctx.decompress_batch(table, 2, status)
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0, 0], shape
        for o in outs:
            assert torch.equal(o, ref), shape
        # sampled blocks against the oracle's decode of the same stream
        for s, o in zip(streams, outs):
            nb = gmp.stream_info(s).n_blocks
            for b in list(rng.choice(nb - 1, 6, replace=False)) + [nb - 1]:
                expect = oracle.decompress_block(s, int(b))
                got = o[int(b) * w.block_size:int(b) * w.block_size + expect.size].cpu().numpy()
                assert np.array_equal(got, expect), (shape, int(b))
        ctx.close()


def test_text256m_full_size(gmp):
    # the tuned shape, the 128-register kernel (16 warps x 1 CTA) and the
    # 96-register kernel (4 warps x 5 CTAs per SM)
    _check_full(gmp, "text256m", shapes=("tuned", (16, 1), (4, 5)))


def test_text256m_full_size_byte_streams(gmp):
    _check_full(gmp, "text256m", byte_mode=True)


def test_csv1g_full_size(gmp):
    _check_full(gmp, "csv1g", shapes=("tuned", (4, 5)))
