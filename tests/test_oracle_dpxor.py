"""Pins for the oracle's dpXOR (§2.3, §3.3): the worked example of Fig. 2, linearity,
special selections, reconstruction D[alpha] = r1 ^ r2, and the threaded subtree split."""
import numpy as np
import pytest

from conftest import golden_lines
from paper_2509_06514_gb300 import workloads


def test_fig2_worked_example(orc):
    g = {r[0]: r[1:] for r in golden_lines("fig2_dpxor.txt")}
    db = np.array([[int(s, 2)] for s in g["db"]], np.uint8)      # 2-bit strings as integers
    v1 = np.array([int(b) for b in g["v1"]], np.uint8)
    v2 = np.array([int(b) for b in g["v2"]], np.uint8)
    r1 = orc.dpxor(db, v1, 1)
    r2 = orc.dpxor(db, v2, 1)
    assert r1[0] == int(g["r1"][0], 2)
    assert r2[0] == int(g["r2"][0], 2)
    item = orc.reconstruct(r1, r2)
    assert item[0] == int(g["item"][0], 2) == db[int(g["target"][0]), 0]
    assert list(v1 ^ v2) == [1 if i == int(g["target"][0]) else 0 for i in range(4)]


def test_dpxor_special_cases(orc):
    rng = np.random.default_rng(3)
    for B in (1, 3, 17, 32, 33):
        db = rng.integers(0, 256, (37, B), dtype=np.uint8)
        zero = np.zeros(37, np.uint8)
        ones = np.ones(37, np.uint8)
        assert orc.dpxor(db, zero, B) == bytes(B)
        want = np.bitwise_xor.reduce(db, axis=0).tobytes()
        assert orc.dpxor(db, ones, B) == want
        assert orc.dpxor(np.zeros_like(db), ones, B) == bytes(B)
        e = np.zeros(37, np.uint8)
        e[5] = 1
        assert orc.dpxor(db, e, B) == db[5].tobytes()


def test_answer_linear_in_database(orc):
    rng = np.random.default_rng(4)
    m, N, B = 7, 100, 24
    k0, _ = orc.gen(17, m, 0, bytes(range(32)))
    d1 = rng.integers(0, 256, (N, B), dtype=np.uint8)
    d2 = rng.integers(0, 256, (N, B), dtype=np.uint8)
    a1 = np.frombuffer(orc.answer(k0, d1, N, B), np.uint8)
    a2 = np.frombuffer(orc.answer(k0, d2, N, B), np.uint8)
    a12 = np.frombuffer(orc.answer(k0, d1 ^ d2, N, B), np.uint8)
    assert np.array_equal(a12, a1 ^ a2)


@pytest.mark.parametrize("prf", [0, 1])
@pytest.mark.parametrize("m,N,B", [(6, 64, 32), (8, 200, 17), (5, 1000, 3), (10, 1024, 1), (9, 300, 64)])
def test_reconstruction(orc, prf, m, N, B):
    db = workloads.make_db(N, B, seed=m * 31 + B)
    rng = np.random.default_rng(m + N)
    for _ in range(3):
        a = int(rng.integers(0, min(N, 1 << m)))
        k0, k1 = orc.gen(a, m, prf, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
        r0 = orc.answer(k0, db, N, B)
        r1 = orc.answer(k1, db, N, B)
        assert orc.reconstruct(r0, r1) == db[a].tobytes()


def test_target_beyond_database_reconstructs_zero(orc):
    """A domain larger than N: leaves j >= N select nothing, so alpha >= N gives 0."""
    m, N, B = 6, 40, 8
    db = workloads.make_db(N, B, seed=9)
    k0, k1 = orc.gen(50, m, 0, bytes(32))
    assert orc.reconstruct(orc.answer(k0, db, N, B), orc.answer(k1, db, N, B)) == bytes(B)


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_subtree_split_matches(orc, threads):
    rng = np.random.default_rng(threads)
    for m, N, B in ((12, 4096, 32), (12, 3000, 5), (9, 5000, 64), (4, 16, 16)):
        db = workloads.make_db(N, B, seed=m + N)
        k0, _ = orc.gen(int(rng.integers(0, min(N, 1 << m))), m, 1 if B == 5 else 0,
                        rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
        assert orc.answer(k0, db, N, B, threads=threads) == orc.answer(k0, db, N, B)


@pytest.mark.parametrize("prf", [0, 1])
def test_pointwise_answer_matches_level_by_level(orc, prf):
    """The branch-parallel answer equals the level-by-level one (and works for m = 40)."""
    rng = np.random.default_rng(40 + prf)
    for m, N, B in ((10, 1000, 9), (12, 3000, 16), (8, 100, 3)):
        db = workloads.make_db(N, B, seed=m)
        k0, k1 = orc.gen(int(rng.integers(0, min(N, 1 << m))), m, prf, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
        assert orc.answer_points(k0, db, N, B) == orc.answer(k0, db, N, B)
    N, B, m, a = 200, 8, 40, 123
    db = workloads.make_db(N, B, seed=7)
    k0, k1 = orc.gen(a, m, prf, bytes(range(32)))
    r0, r1 = orc.answer_points(k0, db, N, B), orc.answer_points(k1, db, N, B)
    assert orc.reconstruct(r0, r1) == db[a].tobytes()
