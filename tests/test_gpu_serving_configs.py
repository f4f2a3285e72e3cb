"""Serving at the full database shapes of the serving workload (three resident databases:
2^18 x 64 B, 2^22 x 256 B, 2^24 x 512 B; Poisson arrivals, uniform database choice and
target, continuous batching within an accumulator budget), with every served answer of one
server compared with the CPU oracle bit for bit and every request reconstructed with the
other server's answer, also served."""
import os
import threading
import time

import numpy as np
import pytest

import paper_2509_06514_gb300 as impir
from paper_2509_06514_gb300 import workloads

pytestmark = pytest.mark.gpu

CORES = os.cpu_count() or 1
N_REQ = 288      # requests of server 0 checked against the oracle (>= 256)
RATE = 20_000    # offered requests per second


@pytest.fixture(scope="module")
def dbs():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()
    out = []
    for i, (n, b) in enumerate(workloads.SERVING_DBS):
        db = workloads.make_db(n, b, seed=900 + i)
        out.append((impir.impir_db_load(db, n, b), db, n, b))
    yield out
    for h, *_ in out:
        impir.impir_db_free(h)


def test_served_answers_equal_oracle_at_full_db_shapes(dbs, orc):
    arr = workloads.poisson_arrivals(RATE, N_REQ, seed=13)
    reqs = []   # (tag, db index, alpha, key of server 0, key of server 1)
    for i in range(N_REQ):
        d = int(arr.db[i])
        n = dbs[d][2]
        k0, k1 = impir.dpf_gen(int(arr.alpha[i]), n.bit_length() - 1, impir.IMPIR_PRF_AES_KEYED, arr.seeds[i])
        reqs.append((i, d, int(arr.alpha[i]), k0, k1))
    assert {d for _, d, *_ in reqs} == {0, 1, 2}
    # the benchmark's server shape: 4 streams, batches of up to 256, accumulators of 4 full
    # batches of the widest record
    server = impir.impir_server_create(max_batch=256, streams=4, max_record_bytes=512,
                                       accumulator_budget=4 * 256 * 512)
    got = {}
    try:
        def client():
            t0 = time.perf_counter()
            for i, (tag, d, a, k0, k1) in enumerate(reqs):
                while time.perf_counter() - t0 < float(arr.t[i]):
                    time.sleep(1e-5)
                # both servers' keys go through the same loop, server 1 tagged + N_REQ
                impir.impir_server_submit(server, dbs[d][0], k0, tag)
                impir.impir_server_submit(server, dbs[d][0], k1, tag + N_REQ)

        th = threading.Thread(target=client)
        th.start()
        deadline = time.time() + 300
        while len(got) < 2 * N_REQ and time.time() < deadline:
            r = impir.impir_server_take(server, 200_000)
            if r is not None:
                got[r["tag"]] = r
        th.join()
        stats = impir.impir_server_stats(server)
    finally:
        impir.impir_server_destroy(server)
    assert len(got) == 2 * N_REQ
    assert stats["batches"] < 2 * N_REQ               # requests were batched together
    assert stats["max_inflight_batches"] >= 2          # and batches overlapped on the device
    for tag, d, a, k0, k1 in reqs:
        h, db, n, b = dbs[d]
        r0, r1 = got[tag]["answer"], got[tag + N_REQ]["answer"]
        assert got[tag]["db"] == h and len(r0) == b and len(r1) == b
        assert bytes(x ^ y for x, y in zip(r0, r1)) == db[a].tobytes(), tag
        assert r0 == orc.answer(k0, db, n, b, threads=CORES), (tag, d)
