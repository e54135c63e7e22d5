"""gmp_decompress_noalloc through the C ABI, against the context path.

Callers that cannot call cudaMalloc (host callbacks that must not re-enter
the allocator, applications whose memory manager owns the device) use
gmp_decompress_noalloc, which decodes with a fixed scratch array inside the
library instead of a context's allocation.  Its output must equal
gmp_decompress's byte for byte (the tolerance of every decoder test here),
call after call, since every call reuses the same array; and the calls after
the first in a context (which looks up the array's address) must leave the
device's free memory unchanged.  The file name sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1606_00519_gb300 import _native
    _native.build()
    import paper_1606_00519_gb300 as gmp
    return torch, gmp, _native.lib()


def _noalloc(L, torch, ds, out, status, max_block_out):
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    return L.gmp_decompress_noalloc(ctypes.c_void_p(ds.comp.data_ptr()), ds.comp_bytes,
                                    ctypes.c_void_p(ds.index.data_ptr()), ds.n_blocks, max_block_out,
                                    ctypes.c_void_p(out.data_ptr()), out.numel(),
                                    ctypes.c_void_p(status.data_ptr()), stream)


@pytest.mark.parametrize("mode", ["mrr", "de"])
def test_noalloc_equals_context_path_on_consecutive_calls(env, mode):
    torch, gmp, L = env
    w = datagen.WORKLOADS["text256m"]
    data = w.data(3 * MiB + 4321)  # 13 blocks, ragged tail
    s = oracle.compress(data, oracle.params(w.block_size, w.n_sub, w.window, de=(mode == "de")))
    ds = gmp.DeviceStream(s)
    ctx = gmp.Context(max_block_out=w.block_size)
    ref, st = ctx.decompress(ds)
    assert st == 0 and np.array_equal(ref.cpu().numpy(), data)
    outs = [torch.full((data.size,), 0x33, dtype=torch.uint8, device="cuda") for _ in range(2)]
    statuses = [torch.full((1,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
    # the first call in this context may look up the array's address
    assert _noalloc(L, torch, ds, outs[0], statuses[0], ds.info.max_block_out) == 0
    torch.cuda.synchronize()
    for call in range(2):
        outs[call].fill_(0x33)
        statuses[call].fill_(-1)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        assert _noalloc(L, torch, ds, outs[call], statuses[call], ds.info.max_block_out) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, call
        assert int(statuses[call].item()) == 0, call
        assert torch.equal(outs[call], ref), call
    ctx.close()


def test_noalloc_limits_are_enforced(env):
    torch, gmp, L = env
    mbo, warps, nbytes = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
    L.gmp_noalloc_limits(ctypes.byref(mbo), ctypes.byref(warps), ctypes.byref(nbytes))
    assert mbo.value == 256 * KiB and warps.value == 32 and nbytes.value < 64 * MiB
    data = datagen.csv_records(1 * MiB + 10, seed=77)
    s = gmp.compress(data, 512 * KiB, 32, 32 * KiB)
    ds = gmp.DeviceStream(s)
    out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # the host check: a stated block size above the limit is refused
    assert _noalloc(L, torch, ds, out, status, 512 * KiB) == -2
    # a stream whose blocks are larger than stated: the kernel reports it
    assert _noalloc(L, torch, ds, out, status, 256 * KiB) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 7
