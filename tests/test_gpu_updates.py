"""Bulk database updates (§3.3: updates applied in windows when the database is idle):
answers after an update see the new records, and under serving traffic every answer is
computed on one whole version of the database (the one it reports)."""
import threading
import time

import numpy as np
import pytest

import paper_2509_06514_gb300 as impir
from paper_2509_06514_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()


def test_sync_update_changes_answers(built, orc):
    N, B, m = 1 << 14, 48, 14
    db = workloads.make_db(N, B, seed=61)
    h = impir.impir_db_load(db, N, B)
    rng = np.random.default_rng(61)
    try:
        assert impir.impir_db_version(h) == 0
        alphas = [150, 700, 9000]
        pairs = [impir.dpf_gen(a, m, i % 2, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
                 for i, a in enumerate(alphas)]
        blob0 = b"".join(p[0] for p in pairs)
        blob1 = b"".join(p[1] for p in pairs)
        new = rng.integers(0, 256, (1000, B), dtype=np.uint8)
        impir.impir_db_update(h, 100, new)
        assert impir.impir_db_version(h) == 1
        db2 = db.copy()
        db2[100:1100] = new
        r0 = impir.impir_answer(h, blob0, 3, B)
        r1 = impir.impir_answer(h, blob1, 3, B)
        for i, a in enumerate(alphas):
            assert np.array_equal(r0[i] ^ r1[i], db2[a])
            assert r0[i].tobytes() == orc.answer(pairs[i][0], db2, N, B)
        with pytest.raises(impir.ImpirError):
            impir.impir_db_update(h, N - 5, new[:10])
    finally:
        impir.impir_db_free(h)


def test_server_answers_on_whole_versions(built, orc):
    specs = [(1 << 13, 32), (1 << 14, 64)]
    dbs, snaps = [], []
    for i, (n, b) in enumerate(specs):
        d = workloads.make_db(n, b, seed=70 + i)
        dbs.append((impir.impir_db_load(d, n, b), n, b))
        snaps.append([d.copy()])
    rng = np.random.default_rng(7)
    reqs = []
    for t in range(240):
        d = int(rng.integers(0, 2))
        h, n, b = dbs[d]
        m = n.bit_length() - 1
        reqs.append((t, d, impir.dpf_gen(int(rng.integers(0, n)), m, 0, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())[0]))
    server = impir.impir_server_create(max_batch=16, streams=3, max_record_bytes=64, accumulator_budget=1 << 20)
    try:
        def client():
            for tag, d, k in reqs:
                impir.impir_server_submit(server, dbs[d][0], k, tag)
                time.sleep(0.0002)

        def updater():
            urng = np.random.default_rng(8)
            for _ in range(6):
                time.sleep(0.006)
                d = int(urng.integers(0, 2))
                h, n, b = dbs[d]
                first = int(urng.integers(0, n - 500))
                cnt = int(urng.integers(1, 500))
                rec = urng.integers(0, 256, (cnt, b), dtype=np.uint8)
                nxt = snaps[d][-1].copy()
                nxt[first:first + cnt] = rec
                snaps[d].append(nxt)             # version len-1 of database d
                impir.impir_server_update(server, h, first, rec)

        tc, tu = threading.Thread(target=client), threading.Thread(target=updater)
        tc.start()
        tu.start()
        got = {}
        deadline = time.time() + 120
        while len(got) < len(reqs) and time.time() < deadline:
            r = impir.impir_server_take(server, 200_000)
            if r is not None:
                got[r["tag"]] = r
        tc.join()
        tu.join()
    finally:
        impir.impir_server_destroy(server)
        for h, *_ in dbs:
            impir.impir_db_free(h)
    assert len(got) == len(reqs)
    seen = set()
    for tag, d, k in reqs:
        r = got[tag]
        v = r["version"]
        seen.add((d, v))
        h, n, b = dbs[d]
        assert r["answer"] == orc.answer(k, snaps[d][v], n, b), (tag, d, v)
    assert len({v for _, v in seen}) > 1          # answers spanned several versions
