"""Host-side thread safety: several threads calling the synchronous XOR and additive answers and
the streamed answer at once, on shared and separate databases, get exactly the answers a single
thread gets (the synchronous and streamed paths serialise on their own locks; the binding
releases the interpreter lock during every call)."""
import threading

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


def test_concurrent_calls_match_single_threaded(built):
    rng = np.random.default_rng(606)
    dbs = [(40000, 64), (70000, 48)]
    data = [workloads.make_db(n, b, seed=600 + i) for i, (n, b) in enumerate(dbs)]
    handles = [impir.impir_db_load(d, n, b) for d, (n, b) in zip(data, dbs)]
    try:
        jobs = []
        for i, (n, b) in enumerate(dbs):
            for m in (15, 16, 17):
                keys = [impir.dpf_gen(int(rng.integers(0, min(n, 1 << m))), m, int(j % 2),
                                      rng.integers(0, 256, 32, dtype=np.uint8).tobytes())[0] for j in range(5)]
                blob = b"".join(keys)
                jobs.append(("xor", i, blob, len(keys)))
                jobs.append(("add", i, blob, len(keys)))
            jobs.append(("streamed", i, blob, len(keys)))

        def run(job):
            kind, i, blob, nq = job
            n, b = dbs[i]
            if kind == "xor":
                return impir.impir_answer(handles[i], blob, nq, b)
            if kind == "add":
                return impir.impir_answer_add32(handles[i], blob, nq, b)
            return impir.impir_answer_streamed(data[i], n, b, blob, nq, 1 << 20)[0]

        want = [run(j) for j in jobs]
        errors, got = [], {}

        def worker(t):
            try:
                for rep in range(3):
                    for k in range(t, len(jobs) + t):
                        idx = k % len(jobs)
                        got[(t, rep, idx)] = run(jobs[idx])
            except Exception as e:  # surfaced below
                errors.append(repr(e))

        threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(300)
        assert not errors, errors
        assert len(got) == 4 * 3 * len(jobs)
        for (t, rep, idx), r in got.items():
            assert np.array_equal(r, want[idx]), (t, rep, jobs[idx][0])
    finally:
        for h in handles:
            impir.impir_db_free(h)
