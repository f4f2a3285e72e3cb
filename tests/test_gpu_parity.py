"""GPU parity: every answer of the CUDA path (through the C ABI) equals the CPU oracle's,
bit for bit (the method is GF(2) and integer work only), on seeded inputs that span many
warp tiles and a ragged tail, over both PRFs, record sizes with and without padding,
domains smaller and larger than the database, mixed-domain batches, every launch shape,
and the one-query-per-launch form."""
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
    return True


def random_key(rng, m, prf):
    """A well-formed key with uniform random codewords (not from Gen)."""
    kb = 8 + 64 * (m + 1)
    k = np.zeros(kb, np.uint8)
    k[0], k[1], k[2] = 1, prf, m
    k[8:] = rng.integers(0, 256, kb - 8, dtype=np.uint8)
    for t, x in ((0, 1), (1, 0), (1, 1)):
        o = 8 + t * 32 * (m + 1) + (x * (m + 1)) * 16
        k[o:o + 16] = 0
    return k.tobytes()


def oracle_answers(orc, keys, db, N, B):
    return np.stack([np.frombuffer(orc.answer(k, db, N, B, threads=8), np.uint8) for k in keys])


def gpu_answers(dbh, keys, B):
    blob, _ = impir.pack_keys(keys)
    return impir.impir_answer(dbh, blob, len(keys), B)


@pytest.mark.parametrize("prf", [0, 1])
@pytest.mark.parametrize("N,B,ms", [
    (1 << 12, 32, [12, 12, 12, 12, 12]),          # domain = N, 2-word records
    (3000, 17, [12, 11, 12, 10]),                  # ragged N, padded records, mixed domains
    (5000, 1, [13, 12, 7, 3, 1]),                  # domain > N, 1-byte records, tiny domains
    (1 << 10, 1024, [10, 10, 10]),                 # multi-pass-free wide records (64 words)
    (777, 33, [10, 9, 4, 2]),                      # odd sizes everywhere
    (1 << 14, 256, [14, 14, 13, 12, 14, 14, 14, 14, 14]),  # > 8 queries: several groups
    (600, 4100, [10, 9]),                          # > 4 KiB records: column passes
])
def test_answer_matches_oracle(built, orc, prf, N, B, ms):
    rng = np.random.default_rng(N + B + prf)
    db = workloads.make_db(N, B, seed=N * 7 + B)
    keys = [random_key(rng, m, prf) for m in ms]
    dbh = impir.impir_db_load(db, N, B)
    try:
        want = oracle_answers(orc, keys, db, N, B)
        got = gpu_answers(dbh, keys, B)
        assert np.array_equal(got, want)
    finally:
        impir.impir_db_free(dbh)


@pytest.mark.parametrize("cfg", [
    dict(lane_bits=0, queries_per_warp=1), dict(lane_bits=1, queries_per_warp=2), dict(lane_bits=3, queries_per_warp=8),
    dict(lane_bits=5, queries_per_warp=4), dict(lane_bits=6, queries_per_warp=2, warps_per_cta=8),
    dict(lane_bits=7, queries_per_warp=8), dict(lane_bits=9, queries_per_warp=2), dict(lane_bits=10, queries_per_warp=1),
    dict(lane_bits=4, queries_per_warp=4, queries_per_launch=1), dict(lane_bits=6, queries_per_warp=16),
    dict(lane_bits=2, queries_per_warp=16, warps_per_cta=4),
    dict(lane_bits=7, queries_per_warp=8, warps_per_cta=20), dict(lane_bits=4, queries_per_warp=2, warps_per_cta=20),
])
def test_every_launch_shape_matches_oracle(built, orc, cfg):
    N, B = 20000, 64
    rng = np.random.default_rng(sum(cfg.values()))
    db = workloads.make_db(N, B, seed=11)
    ms = [15, 15, 14, 12, 15, 9, 15, 15, 15, 6, 15]
    keys = [random_key(rng, m, int(i % 2)) for i, m in enumerate(ms)]
    dbh = impir.impir_db_load(db, N, B)
    try:
        impir.impir_set_config(dbh, **cfg)
        got = gpu_answers(dbh, keys, B)
        want = oracle_answers(orc, keys, db, N, B)
        assert np.array_equal(got, want)
    finally:
        impir.impir_db_free(dbh)


@pytest.mark.parametrize("prf", [0, 1])
def test_reconstruction_two_servers(built, orc, prf):
    """r_A ^ r_B = D[alpha] for keys from the library's own Gen, and both answers equal the oracle's."""
    N, B, m = 50000, 48, 16
    db = workloads.make_db(N, B, seed=21)
    rng = np.random.default_rng(3 + prf)
    alphas = [int(a) for a in rng.integers(0, N, 6)]
    pairs = [impir.dpf_gen(a, m, prf, rng.integers(0, 256, 32, dtype=np.uint8).tobytes()) for a in alphas]
    dbh = impir.impir_db_load(db, N, B)
    try:
        r0 = gpu_answers(dbh, [p[0] for p in pairs], B)
        r1 = gpu_answers(dbh, [p[1] for p in pairs], B)
        for i, a in enumerate(alphas):
            assert bytes(r0[i] ^ r1[i]) == db[a].tobytes()
        assert np.array_equal(r0[:2], oracle_answers(orc, [p[0] for p in pairs[:2]], db, N, B))
    finally:
        impir.impir_db_free(dbh)


def test_async_path_with_torch_memory_and_bad_key(built, orc):
    import torch
    N, B = 4096, 32
    db = workloads.make_db(N, B, seed=5)
    rng = np.random.default_rng(8)
    keys = [random_key(rng, 12, 0) for _ in range(5)]
    bad = bytearray(keys[3])
    bad[0] = 9                         # wrong version: rejected on the device
    keys[3] = bytes(bad)
    blob, offs = impir.pack_keys(keys)
    d_db = torch.zeros((N, 32), dtype=torch.uint8, device="cuda")
    d_db.copy_(torch.from_numpy(db))
    dbh = impir.impir_db_attach(d_db, N, B, 32)
    try:
        d_keys = torch.from_numpy(np.frombuffer(blob, np.uint8).copy()).cuda()
        d_off = torch.from_numpy(offs.astype(np.int32)).cuda()
        d_out = torch.zeros((len(keys), B), dtype=torch.uint8, device="cuda")
        wsb = impir.impir_workspace_bytes(len(keys), 32)
        d_ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        impir.impir_answer_async(dbh, d_keys, d_off, len(keys), d_out, d_ws, wsb, s)
        s.synchronize()
        got = d_out.cpu().numpy()
        assert impir.impir_workspace_status(d_ws) == (1, 3)
        for i, k in enumerate(keys):
            if i == 3:
                assert not got[i].any()
            else:
                assert got[i].tobytes() == orc.answer(k, db, N, B)
        with pytest.raises(impir.ImpirError):      # the synchronous path rejects before launching
            impir.impir_answer(dbh, blob, len(keys), B)
    finally:
        impir.impir_db_free(dbh)


def test_empty_batch_and_single_record(built, orc):
    db = workloads.make_db(1, 5, seed=1)
    dbh = impir.impir_db_load(db, 1, 5)
    try:
        assert impir.impir_answer(dbh, b"", 0, 5).shape == (0, 5)
        k0, k1 = impir.dpf_gen(0, 1, 0, bytes(32))
        r0 = gpu_answers(dbh, [k0], 5)
        r1 = gpu_answers(dbh, [k1], 5)
        assert bytes(r0[0] ^ r1[0]) == db[0].tobytes()
        assert r0[0].tobytes() == orc.answer(k0, db, 1, 5)
    finally:
        impir.impir_db_free(dbh)


@pytest.mark.parametrize("prf", [0, 1])
def test_large_domains_over_small_database(built, orc, prf):
    """Domains of 2^27..2^40 leaves over a 5000-record DB: only the prefix min(2^m, N) counts."""
    N, B = 5000, 40
    db = workloads.make_db(N, B, seed=4040)
    rng = np.random.default_rng(400 + prf)
    keys = [random_key(rng, m, prf) for m in (27, 33, 40, 40)]
    pairs = [impir.dpf_gen(a, 40, prf, rng.integers(0, 256, 32, dtype=np.uint8).tobytes()) for a in (0, 4999)]
    dbh = impir.impir_db_load(db, N, B)
    try:
        got = gpu_answers(dbh, keys + [p[0] for p in pairs], B)
        for i, k in enumerate(keys + [p[0] for p in pairs]):
            assert got[i].tobytes() == orc.answer_points(k, db, N, B), i
        other = gpu_answers(dbh, [p[1] for p in pairs], B)
        assert bytes(got[4] ^ other[0]) == db[0].tobytes()
        assert bytes(got[5] ^ other[1]) == db[4999].tobytes()
    finally:
        impir.impir_db_free(dbh)


@pytest.mark.parametrize("cfg", [None, dict(lane_bits=3, queries_per_warp=4)])
def test_every_domain_size_in_one_batch(built, orc, cfg):
    """One batch holding a key of every domain size 2^1 .. 2^40 (both PRFs, both parties):
    40 groups and segments, domains far smaller and far larger than N."""
    N, B = 3000, 24
    db = workloads.make_db(N, B, seed=4141)
    rng = np.random.default_rng(4141)
    keys = []
    for m in range(1, 41):
        k = bytearray(random_key(rng, m, m % 2))
        k[3] = (m // 2) % 2
        keys.append(bytes(k))
    order = rng.permutation(len(keys))
    keys = [keys[i] for i in order]
    dbh = impir.impir_db_load(db, N, B)
    try:
        if cfg:
            impir.impir_set_config(dbh, **cfg)
        got = gpu_answers(dbh, keys, B)
        for i, k in enumerate(keys):
            assert got[i].tobytes() == orc.answer_points(k, db, N, B), (i, k[2])
    finally:
        impir.impir_db_free(dbh)


def test_large_batch_reconstructs(built, orc):
    """12000 queries in one batch (domains 2^8 .. 2^13 over a 6000-record DB): every query's two
    answers reconstruct its record, and a sample equals the oracle's answer."""
    N, B = 6000, 16
    db = workloads.make_db(N, B, seed=12000)
    rng = np.random.default_rng(12000)
    ms = [int(m) for m in rng.integers(8, 14, 12000)]
    alphas = [int(rng.integers(0, min(N, 1 << m))) for m in ms]
    pairs = [impir.dpf_gen(a, m, i % 2, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
             for i, (a, m) in enumerate(zip(alphas, ms))]
    dbh = impir.impir_db_load(db, N, B)
    try:
        r0 = gpu_answers(dbh, [p[0] for p in pairs], B)
        r1 = gpu_answers(dbh, [p[1] for p in pairs], B)
        assert np.array_equal(r0 ^ r1, db[alphas])
        for i in rng.choice(len(pairs), 40, replace=False):
            assert r0[i].tobytes() == orc.answer(pairs[i][0], db, N, B), i
    finally:
        impir.impir_db_free(dbh)


@pytest.mark.parametrize("B", [1040, 2064, 4100])
@pytest.mark.parametrize("cfg", [dict(lane_bits=4, queries_per_warp=8), dict(lane_bits=3, queries_per_warp=4),
                                 dict(lane_bits=5, queries_per_warp=2)])
def test_wide_records_in_column_passes(built, orc, B, cfg):
    """Records above 512 bytes with up to 8 queries per warp: the scan covers each record in
    several column passes of 16 / queries_per_warp words per lane (ragged last pass)."""
    N = 3000
    db = workloads.make_db(N, B, seed=B + cfg["queries_per_warp"])
    rng = np.random.default_rng(B)
    ms = [12, 12, 12, 11, 12, 12, 12, 12, 12, 10]
    keys = [random_key(rng, m, int(i % 2)) for i, m in enumerate(ms)]
    dbh = impir.impir_db_load(db, N, B)
    try:
        impir.impir_set_config(dbh, **cfg)
        got = gpu_answers(dbh, keys, B)
        for i, k in enumerate(keys):
            assert got[i].tobytes() == orc.answer(k, db, N, B), i
    finally:
        impir.impir_db_free(dbh)
