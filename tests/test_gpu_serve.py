"""GPU serving loop: continuous batching under a device-memory budget.
Requests of mixed sizes and modes are submitted while others run; every
output must equal the request decoded alone (tolerance: 0 bytes) and the
original data, and admission must respect the budget."""
import time

import numpy as np
import pytest

import datagen

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300, method="thread")]

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
def requests(gmp):
    mix = datagen.request_mix(seed=9, n=24, lo=16 * KiB, hi=6 * MiB)
    out = []
    for size, kind, mode, s in mix:
        data = datagen.make_data(kind, size, s)
        out.append((data, gmp.compress(data, 256 * KiB, 32, 32 * KiB, de=(mode == "de"))))
    return out


def _run(gmp, server, reqs, spacing_s=0.0):
    ids = {}
    results = {}
    for i, (data, s) in enumerate(reqs):
        ids[server.submit(s)] = i
        if spacing_s:
            time.sleep(spacing_s)
        for c in server.poll():
            results[c["id"]] = c
    server.drain()
    for c in server.poll():
        results[c["id"]] = c
    outs = {}
    for rid, c in results.items():
        i = ids[rid]
        buf = np.empty(max(c["out_bytes"], 1), np.uint8)
        server.copy_out(rid, buf)
        outs[i] = (c, buf[:c["out_bytes"]])
        server.release(rid)
    return outs


def test_serving_mixed_requests(gmp, requests):
    srv = gmp.Server(budget_bytes=512 * MiB, n_lanes=3, max_batch=8)
    outs = _run(gmp, srv, requests, spacing_s=0.001)
    assert len(outs) == len(requests)
    for i, (data, _) in enumerate(requests):
        c, got = outs[i]
        assert c["status"] == 0
        assert c["t_submit"] <= c["t_start"] <= c["t_done"]
        assert 0.0 <= c["t_gpu_ready"] <= c["t_gpu_done"]
        assert np.array_equal(got, data)
    assert srv.bytes_in_use() == 0
    srv.close()


def test_alone_equals_in_mix(gmp, requests):
    srv = gmp.Server(budget_bytes=512 * MiB, n_lanes=4, max_batch=16)
    mixed = _run(gmp, srv, requests)
    for i, r in enumerate(requests[:8]):
        alone = _run(gmp, srv, [r])
        assert np.array_equal(alone[0][1], mixed[i][1])
    srv.close()


def test_budget_admission(gmp, requests):
    # a budget that holds only a few requests at a time: the rest are admitted
    # as completed requests are released
    biggest = max(d.size + s.size for d, s in requests)
    srv = gmp.Server(budget_bytes=int(biggest * 1.5) + 1 * MiB, n_lanes=2, max_batch=4)
    pending = {}
    done = 0
    for i, (data, s) in enumerate(requests):
        pending[srv.submit(s)] = i
    peak = 0
    deadline = time.time() + 120
    while done < len(requests) and time.time() < deadline:
        peak = max(peak, srv.bytes_in_use())
        for c in srv.poll(wait_ms=50):
            i = pending.pop(c["id"])
            buf = np.empty(max(c["out_bytes"], 1), np.uint8)
            srv.copy_out(c["id"], buf)
            assert c["status"] == 0 and np.array_equal(buf[:c["out_bytes"]], requests[i][0])
            srv.release(c["id"])
            done += 1
    assert done == len(requests)
    assert peak <= int(biggest * 1.5) + 1 * MiB
    srv.close()


def test_request_larger_than_budget_is_refused(gmp, requests):
    data, s = max(requests, key=lambda r: r[0].size)
    srv = gmp.Server(budget_bytes=data.size // 2, n_lanes=1)
    with pytest.raises(gmp.GmpError):
        srv.submit(s)
    srv.close()


def test_serving_shape_of_the_load_configuration(gmp):
    """The serving configuration's request shape: sizes log-uniform from
    16 KiB to 64 MiB, mixed content and modes, arriving while others run,
    under a budget that holds only some of them (2 GiB here instead of 32).
    Several lanes must be busy at the same time (their batches' intervals
    overlap on the host's and on the GPU's clock), and every output must equal
    the input and the same request decoded alone (tolerance: 0 bytes)."""
    mix = datagen.request_mix(seed=21, n=40, lo=16 * KiB, hi=64 * MiB)
    reqs = []
    for size, kind, mode, sd in mix:
        data = datagen.make_data(kind, size, sd)
        reqs.append((data, gmp.compress(data, 256 * KiB, 32, 32 * KiB, de=(mode == "de"))))
    assert max(d.size for d, _ in reqs) > 32 * MiB
    srv = gmp.Server(budget_bytes=2 << 30, n_lanes=4, max_batch=8)
    mixed = _run(gmp, srv, reqs, spacing_s=0.0005)
    assert len(mixed) == len(reqs)
    spans, gpu_spans = [], []
    for i, (data, _) in enumerate(reqs):
        c, got = mixed[i]
        assert c["status"] == 0 and np.array_equal(got, data)
        spans.append((c["t_start"], c["t_done"]))
        gpu_spans.append((c["t_gpu_ready"], c["t_gpu_done"]))
    # distinct launches (requests of one batch share theirs) whose launch-to-
    # completion intervals overlap: batches of different lanes in flight at
    # the same time, on the host's clock and on the GPU's (from the inputs
    # being in to the decode's end)
    for sp in (spans, gpu_spans):
        launches = sorted(set(sp))
        overlaps = sum(1 for a, b in zip(launches, launches[1:]) if b[0] < a[1])
        assert len(launches) >= 2 and overlaps >= 1
    # the largest requests again, alone
    for i in sorted(range(len(reqs)), key=lambda k: -reqs[k][0].size)[:4]:
        alone = _run(gmp, srv, [reqs[i]])
        assert np.array_equal(alone[0][1], mixed[i][1])
    assert srv.bytes_in_use() == 0
    srv.close()
