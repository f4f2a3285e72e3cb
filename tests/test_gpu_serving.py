"""Serving loop (continuous batching, §3.4 analog): requests arriving while others run are
admitted into new batches on free streams within the accumulator budget; every answer equals
the same key answered alone, and both servers' answers reconstruct the record."""
import threading
import time

import numpy as np
import pytest

import paper_2509_06514_gb300 as impir
from paper_2509_06514_gb300 import workloads

pytestmark = pytest.mark.gpu

DBS = [(1 << 14, 64), (1 << 16, 256), (1 << 17, 512)]


@pytest.fixture(scope="module")
def dbs():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()
    out = []
    for i, (n, b) in enumerate(DBS):
        db = workloads.make_db(n, b, seed=500 + i)
        out.append((impir.impir_db_load(db, n, b), db, n, b))
    yield out
    for h, *_ in out:
        impir.impir_db_free(h)


def make_requests(dbs, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for t in range(count):
        d = int(rng.integers(0, len(dbs)))
        h, db, n, b = dbs[d]
        m = n.bit_length() - 1
        a = int(rng.integers(0, n))
        k0, k1 = impir.dpf_gen(a, m, t % 2, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
        reqs.append((t, d, a, k0, k1))
    return reqs


def serve_all(server, dbs, reqs, rate):
    """Submit from a client thread at Poisson times while the main thread takes results."""
    rng = np.random.default_rng(1)
    gaps = rng.exponential(1.0 / rate, len(reqs))

    def client():
        t0 = time.perf_counter()
        due = 0.0
        for (tag, d, a, k0, k1), g in zip(reqs, gaps):
            due += g
            while time.perf_counter() - t0 < due:
                pass
            impir.impir_server_submit(server, dbs[d][0], k0, tag)

    th = threading.Thread(target=client)
    th.start()
    got = {}
    deadline = time.time() + 120
    while len(got) < len(reqs) and time.time() < deadline:
        r = impir.impir_server_take(server, 200_000)
        if r is not None:
            got[r["tag"]] = r
    th.join()
    return got


def test_results_equal_alone_and_in_the_mix(dbs):
    reqs = make_requests(dbs, 300, seed=3)
    server = impir.impir_server_create(max_batch=64, streams=4, max_record_bytes=512,
                                       accumulator_budget=4 * 64 * 512)
    try:
        got = serve_all(server, dbs, reqs, rate=20000)
        stats = impir.impir_server_stats(server)
    finally:
        impir.impir_server_destroy(server)
    assert len(got) == len(reqs)
    for tag, d, a, k0, k1 in reqs:
        h, db, n, b = dbs[d]
        r = got[tag]
        assert r["db"] == h and len(r["answer"]) == b
        alone0 = impir.impir_answer(h, k0, 1, b)[0].tobytes()
        assert r["answer"] == alone0, tag
        alone1 = impir.impir_answer(h, k1, 1, b)[0].tobytes()
        assert bytes(x ^ y for x, y in zip(r["answer"], alone1)) == db[a].tobytes()
    assert stats["queries"] == len(reqs)
    assert stats["batches"] < len(reqs)            # requests were batched together
    assert stats["max_inflight_batches"] >= 2      # batches overlapped on the device
    assert max(r["batch"] for r in got.values()) > 1


def test_admission_respects_accumulator_budget(dbs):
    reqs = make_requests(dbs, 60, seed=4)
    # room for the accumulators of two 512-byte queries at a time
    server = impir.impir_server_create(max_batch=64, streams=4, max_record_bytes=512, accumulator_budget=2 * 512)
    try:
        got = serve_all(server, dbs, reqs, rate=50000)
        stats = impir.impir_server_stats(server)
    finally:
        impir.impir_server_destroy(server)
    assert len(got) == len(reqs)
    for tag, d, a, k0, k1 in reqs:
        h, db, n, b = dbs[d]
        assert got[tag]["batch"] <= 2 * 512 // (((b + 15) // 16) * 16)
        assert got[tag]["answer"] == impir.impir_answer(h, k0, 1, b)[0].tobytes()
    assert stats["queries"] == len(reqs)


def test_take_times_out_and_bad_key_is_rejected(dbs):
    server = impir.impir_server_create(max_batch=8, streams=2, max_record_bytes=512, accumulator_budget=1 << 20)
    try:
        t0 = time.perf_counter()
        assert impir.impir_server_take(server, 20_000) is None
        assert time.perf_counter() - t0 < 5
        k0, _ = impir.dpf_gen(1, 14, 0, bytes(32))
        bad = bytearray(k0)
        bad[0] = 3
        with pytest.raises(impir.ImpirError) as e:
            impir.impir_server_submit(server, dbs[0][0], bytes(bad), 1)
        assert e.value.status == impir.IMPIR_EINVAL
        with pytest.raises(impir.ImpirError):
            impir.impir_server_submit(server, 999, k0, 2)
    finally:
        impir.impir_server_destroy(server)
