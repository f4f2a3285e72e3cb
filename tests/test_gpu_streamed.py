"""Databases larger than device memory (§3.3, chunked evaluation): streaming the records
from host memory in chunks gives the same answers as the resident database, bit for bit,
for ragged sizes, chunks smaller than a warp tile, mixed domains, and pinned host memory."""
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


def keys_for(rng, N, ms, prf=0):
    return [impir.dpf_gen(int(rng.integers(0, min(N, 1 << m))), m, prf, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
            for m in ms]


@pytest.mark.parametrize("N,B,chunk_bytes,ms", [
    (1 << 20, 256, 16 << 20, [20] * 24 + [19, 18, 12, 3]),
    (300001, 40, 5 << 20, [19, 19, 17, 12, 19]),
    (70000, 1024, 1, [17, 16, 10]),          # chunk rounded up to one warp tile
    (5000, 64, 1 << 30, [13, 12, 5]),        # chunk larger than the DB
    (1 << 20, 64, 0, [20, 19, 11]),          # the default chunk size
])
def test_streamed_equals_resident(built, orc, N, B, chunk_bytes, ms):
    rng = np.random.default_rng(N + B)
    db = workloads.make_db(N, B, seed=N)
    pairs = keys_for(rng, N, ms, prf=int(B == 40))
    blob0 = b"".join(p[0] for p in pairs)
    got, cfg = impir.impir_answer_streamed(db, N, B, blob0, len(pairs), chunk_bytes)
    h = impir.impir_db_load(db, N, B)
    try:
        want = impir.impir_answer(h, blob0, len(pairs), B)
    finally:
        impir.impir_db_free(h)
    assert np.array_equal(got, want)
    for i in (0, len(pairs) - 1):
        assert got[i].tobytes() == orc.answer(pairs[i][0], db, N, B, threads=8)


def test_streamed_from_pinned_memory_reconstructs(built):
    import torch
    N, B = 1 << 19, 64
    db = workloads.make_db(N, B, seed=9)
    pinned = torch.empty(N * B, dtype=torch.uint8, pin_memory=True)
    pinned.copy_(torch.from_numpy(db.reshape(-1)))
    rng = np.random.default_rng(9)
    alphas = [0, 12345, N - 1]
    pairs = [impir.dpf_gen(a, 19, 0, rng.integers(0, 256, 32, dtype=np.uint8).tobytes()) for a in alphas]
    r0, _ = impir.impir_answer_streamed(pinned.data_ptr(), N, B, b"".join(p[0] for p in pairs), 3, 4 << 20)
    r1, _ = impir.impir_answer_streamed(pinned.data_ptr(), N, B, b"".join(p[1] for p in pairs), 3, 4 << 20)
    for i, a in enumerate(alphas):
        assert np.array_equal(r0[i] ^ r1[i], db[a])


def test_streamed_buffer_reuse_across_layouts(built):
    """The staging buffers are kept between calls: a padded layout (40 B records, 48 B rows),
    then whole 48 B rows that overwrite the padding, then the padded layout again; every call
    equals the resident answers."""
    rng = np.random.default_rng(77)
    for N, B in ((90000, 40), (90000, 48), (90000, 40), (1 << 16, 256), (90000, 40)):
        db = workloads.make_db(N, B, seed=N + B + 1)
        pairs = keys_for(rng, N, [17, 16, 14])
        blob = b"".join(p[0] for p in pairs)
        got, _ = impir.impir_answer_streamed(db, N, B, blob, len(pairs), 1 << 20)
        h = impir.impir_db_load(db, N, B)
        try:
            assert np.array_equal(got, impir.impir_answer(h, blob, len(pairs), B)), (N, B)
        finally:
            impir.impir_db_free(h)
