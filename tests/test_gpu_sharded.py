"""Row shards on one GPU: a database split into three row shards (one handle each) answers
every query with partial answers whose combination (XOR, or sum mod 2^32 for the additive
answer) equals the whole database's answer and the oracle's, bit for bit, for domains that
cover all, some or one of the shards, tiny domains, both PRFs, padded records and several
launch shapes; bad shard bounds are rejected; bulk updates address rows within the shard."""
import numpy as np
import pytest

import paper_2509_06514_gb300 as impir
from paper_2509_06514_gb300 import workloads
from paper_2509_06514_gb300.sharding import combine, shard_rows

pytestmark = pytest.mark.gpu

N = 100000


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()
    return torch


def load_shards(db, B, world=3):
    blocks = shard_rows(N, world)
    assert [n for _, n in blocks] == [32768, 32768, N - 65536]
    return [impir.impir_db_load_rows(db[lo:lo + n], n, B, lo, N) for lo, n in blocks]


def keys_for(rng, ms, prf_of=lambda i: i % 2):
    """(targets, key pairs) for domains ms."""
    alphas = [int(rng.integers(0, min(N, 1 << m))) for m in ms]
    pairs = [impir.dpf_gen(a, m, prf_of(i), rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
             for i, (a, m) in enumerate(zip(alphas, ms))]
    return alphas, pairs


MS = [17, 16, 15, 10, 4, 17, 3]


@pytest.mark.parametrize("B", [40, 64])
@pytest.mark.parametrize("cfg", [None, (10, 1, 16), (3, 2, 16), (7, 8, 20)])
def test_sharded_xor_answers_combine_to_the_whole(torch_cuda, orc, B, cfg):
    torch = torch_cuda
    db = workloads.make_db(N, B, seed=B + 1)
    rng = np.random.default_rng(B)
    alphas, pairs = keys_for(rng, MS)
    blob0, _ = impir.pack_keys([p[0] for p in pairs])
    blob1, _ = impir.pack_keys([p[1] for p in pairs])
    whole = impir.impir_db_load(db, N, B)
    shards = load_shards(db, B)
    try:
        if cfg:
            for h in shards:
                impir.impir_set_config(h, *cfg, 0)
        combined = []
        for blob in (blob0, blob1):
            parts = np.stack([impir.impir_answer(h, blob, len(pairs), B) for h in shards])
            got = combine(torch.from_numpy(parts).cuda(), 0).cpu().numpy()
            assert np.array_equal(got, impir.impir_answer(whole, blob, len(pairs), B))
            assert np.array_equal(got, np.bitwise_xor.reduce(parts, axis=0))
            combined.append(got)
        for i in (0, 2, 4):
            assert combined[0][i].tobytes() == orc.answer(pairs[i][0], db, N, B), i
        # every query reconstructs from the two servers' combined answers
        assert np.array_equal(combined[0] ^ combined[1], db[alphas])
        # domains inside the first shard: the other shards' partials are zero
        parts0 = [impir.impir_answer(h, blob0, len(pairs), B) for h in shards]
        for i, m in enumerate(MS):
            if (1 << m) <= 32768:
                assert not parts0[1][i].any() and not parts0[2][i].any(), m
    finally:
        impir.impir_db_free(whole)
        for h in shards:
            impir.impir_db_free(h)


def test_sharded_device_path_and_additive(torch_cuda, orc):
    torch = torch_cuda
    B = 48
    db = workloads.make_db(N, B, seed=4848)
    rng = np.random.default_rng(4848)
    _, pairs = keys_for(rng, MS, prf_of=lambda i: 0)
    keys0 = [p[0] for p in pairs]
    blob, offs = impir.pack_keys(keys0)
    n = len(keys0)
    whole = impir.impir_db_load(db, N, B)
    shards = load_shards(db, B)
    try:
        assert [impir.impir_db_rows(h) for h in shards] == [(0, N), (32768, N), (65536, N)]
        d_keys = torch.from_numpy(np.frombuffer(blob, np.uint8).copy()).cuda()
        d_off = torch.from_numpy(offs.view(np.int32).copy()).cuda()
        parts = torch.zeros((len(shards), n, B), dtype=torch.uint8, device="cuda")
        wsb = impir.impir_workspace_bytes(n, B)
        d_ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        for r, h in enumerate(shards):
            impir.impir_answer_async(h, d_keys, d_off, n, parts[r], d_ws, wsb, s)
        out = combine(parts, 0, s)
        s.synchronize()
        assert np.array_equal(out.cpu().numpy(), impir.impir_answer(whole, blob, n, B))
        # additive answer: shard partial sums add up to the whole database's answer
        add_parts = np.stack([impir.impir_answer_add32(h, blob, n, B) for h in shards])
        add = combine(torch.from_numpy(add_parts).cuda(), 1).cpu().numpy()
        assert np.array_equal(add, impir.impir_answer_add32(whole, blob, n, B))
        for i in (0, 3):
            assert add[i].tobytes() == orc.answer_add32(keys0[i], db, N, B), i
    finally:
        impir.impir_db_free(whole)
        for h in shards:
            impir.impir_db_free(h)


def test_combine_kernel_paths(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(5)
    for nparts, nbytes, mode in ((3, 15, 0), (2, 12, 1), (5, 4096, 0), (4, 4096, 1), (1, 33, 0)):
        parts = rng.integers(0, 256, (nparts, nbytes), dtype=np.uint8)
        out = combine(torch.from_numpy(parts).cuda(), mode).cpu().numpy()
        if mode == 0:
            want = np.bitwise_xor.reduce(parts, axis=0)
        else:
            w = parts.view("<u4").astype(np.uint64).sum(axis=0) % (1 << 32)
            want = w.astype("<u4").view(np.uint8)
        assert np.array_equal(out, want), (nparts, nbytes, mode)
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(impir.ImpirError):
        impir.impir_combine_partials(1, d, 2, 6, torch.zeros(6, dtype=torch.uint8, device="cuda"))  # not 4-byte sized
    with pytest.raises(impir.ImpirError):
        impir.impir_combine_partials(0, d, 2, 16, d[8:])                                           # overlap
    with pytest.raises(impir.ImpirError):
        impir.impir_combine_partials(2, d, 2, 16, torch.zeros(16, dtype=torch.uint8, device="cuda"))


def test_bad_shard_bounds_and_shard_updates(torch_cuda, orc):
    B = 32
    db = workloads.make_db(N, B, seed=3232)
    for lo, n in ((1000, 40000), (32768, 1000), (65536, N), (0, 0), (N, 1)):
        with pytest.raises(impir.ImpirError):
            impir.impir_db_load_rows(db[:max(n, 1)], n, B, lo, N)
    shards = load_shards(db, B)
    whole = impir.impir_db_load(db, N, B)
    try:
        rng = np.random.default_rng(32)
        new = rng.integers(0, 256, (100, B), dtype=np.uint8)
        impir.impir_db_update(shards[1], 500, new)               # global rows 33268 .. 33367
        impir.impir_db_update(whole, 32768 + 500, new)
        upd = db.copy()
        upd[32768 + 500:32768 + 600] = new
        _, pairs = keys_for(rng, [17, 16])
        blob, _ = impir.pack_keys([p[0] for p in pairs])
        parts = np.stack([impir.impir_answer(h, blob, 2, B) for h in shards])
        got = np.bitwise_xor.reduce(parts, axis=0)
        assert np.array_equal(got, impir.impir_answer(whole, blob, 2, B))
        assert got[0].tobytes() == orc.answer(pairs[0][0], upd, N, B)
    finally:
        impir.impir_db_free(whole)
        for h in shards:
            impir.impir_db_free(h)
