"""The seeded input generator: the C helper equals its numpy restatement, and records can
be regenerated alone."""
import numpy as np

from paper_2509_06514_gb300 import workloads


def test_stream_matches_numpy():
    for seed in (0, 1, 2**63 + 5):
        for off, n in ((0, 1000), (3, 77), (13, 4096), (8, 8)):
            assert np.array_equal(workloads.stream_bytes(n, seed, off), workloads.stream_bytes_numpy(n, seed, off))
    big = workloads.stream_bytes(3 << 20, 7, 5, threads=4)
    assert np.array_equal(big, workloads.stream_bytes_numpy(3 << 20, 7, 5))


def test_record_regeneration():
    db = workloads.make_db(1000, 33, seed=4)
    for j in (0, 1, 500, 999):
        assert workloads.record(1000, 33, 4, j) == db[j].tobytes()


def test_workload_shapes():
    w = workloads.uneven_8gib()
    assert w.n_queries == 1024
    assert all(1 <= len(b.ms) <= 512 for b in w.batches)
    assert set(m for b in w.batches for m in b.ms) <= {23, 24, 25}
    for b in w.batches:
        assert all(0 <= a < (1 << m) for a, m in zip(b.alphas, b.ms))
    # the documented split of the benchmark workload (seeded)
    assert [len(b.ms) for b in w.batches] == [416, 178, 379, 51]


def test_batched_4gib_record_sizes():
    for b in (32, 256, 1024, 4096):
        w = workloads.batched_4gib(record_bytes=b)
        assert w.n_records * w.record_bytes == 4 << 30 and w.n_queries == 256
        assert set(w.batches[0].ms) == {workloads.log2_exact(w.n_records)}
    # the default (1 KiB records) workload is the one the GPU configuration test answers
    d = workloads.batched_4gib()
    assert (d.n_records, d.record_bytes, d.name) == (1 << 22, 1024, "batched: N=2^22 x 1 KiB, m=22, Q=256")
    assert d.batches[0].alphas == workloads.batched_4gib(record_bytes=1024).batches[0].alphas
