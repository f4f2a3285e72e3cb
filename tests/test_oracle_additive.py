"""Pins for the oracle's additive (inner-product) answer over Z_{2^32} (§2.2's linear
combination, reconstructed as r_0 + r_1): brute-force share sums over tiny domains,
reconstruction of the target record, and linearity in the database."""
import numpy as np
import pytest

from paper_2509_06514_gb300 import workloads


def low32(leaves):
    return leaves[:, :4].copy().view("<u4").reshape(-1).astype(np.uint64)


@pytest.mark.parametrize("prf", [0, 1])
def test_shares_sum_to_one_hot(orc, prf):
    """(-1)^0 low32(R_0(m,j)) + (-1)^1 low32(R_1(m,j)) = [j == alpha] mod 2^32 for all j."""
    rng = np.random.default_rng(30 + prf)
    for m in range(1, 9):
        for a in (range(1 << m) if m <= 3 else rng.integers(0, 1 << m, 3)):
            k0, k1 = orc.gen(int(a), m, prf, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
            assert k0[3] == 0 and k1[3] == 1
            s = (low32(orc.eval_all(k0)) - low32(orc.eval_all(k1))) % (1 << 32)
            want = np.zeros(1 << m, np.uint64)
            want[int(a)] = 1
            assert np.array_equal(s, want), (m, a)


@pytest.mark.parametrize("prf", [0, 1])
@pytest.mark.parametrize("m,N,B", [(8, 256, 32), (10, 700, 12), (6, 1000, 4), (12, 4096, 64)])
def test_additive_reconstruction(orc, prf, m, N, B):
    db = workloads.make_db(N, B, seed=m + N + B)
    rng = np.random.default_rng(m * N)
    for _ in range(3):
        a = int(rng.integers(0, min(N, 1 << m)))
        k0, k1 = orc.gen(a, m, prf, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
        r0 = orc.answer_add32(k0, db, N, B)
        r1 = orc.answer_add32(k1, db, N, B)
        assert orc.reconstruct_add32(r0, r1) == db[a].tobytes()
        # the XOR answer of the same keys is unaffected by the party index
        assert orc.reconstruct(orc.answer(k0, db, N, B), orc.answer(k1, db, N, B)) == db[a].tobytes()


def test_additive_answer_is_linear(orc):
    rng = np.random.default_rng(5)
    N, B, m = 300, 16, 9
    d1 = rng.integers(0, 256, (N, B), dtype=np.uint8)
    d2 = rng.integers(0, 256, (N, B), dtype=np.uint8)
    s = (d1.view("<u4").astype(np.uint64) + d2.view("<u4").astype(np.uint64)) % (1 << 32)
    d12 = s.astype("<u4").view(np.uint8).reshape(N, B)
    k0, _ = orc.gen(17, m, 0, bytes(range(32)))
    a1 = np.frombuffer(orc.answer_add32(k0, d1, N, B), "<u4").astype(np.uint64)
    a2 = np.frombuffer(orc.answer_add32(k0, d2, N, B), "<u4").astype(np.uint64)
    a12 = np.frombuffer(orc.answer_add32(k0, d12, N, B), "<u4").astype(np.uint64)
    assert np.array_equal(a12, (a1 + a2) % (1 << 32))


def test_party_byte_validation(orc):
    k0, k1 = orc.gen(3, 4, 0, bytes(32))
    assert orc.key_check(k1) == 0
    bad = bytearray(k1)
    bad[3] = 2
    assert orc.key_check(bytes(bad)) != 0
