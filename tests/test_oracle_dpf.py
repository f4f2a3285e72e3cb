"""Pins for the oracle's GGM tree (Eqs. (1)-(3), §3.2) and its key generator (§3.1):
the two evaluation orders agree, a closed form with a library AES fixes the wire layout,
and brute force over tiny domains shows the DPF property of §2.3."""
import numpy as np
import pytest


def random_key(rng, m, prf):
    """A well-formed key with uniform random codewords (any such key evaluates)."""
    kb = 8 + 64 * (m + 1)
    k = np.zeros(kb, np.uint8)
    k[0], k[1], k[2] = 1, prf, m
    c = rng.integers(0, 256, kb - 8, dtype=np.uint8)
    k[8:] = c
    # column 0: only C_0[0][0] (the root) may be nonzero
    def off(t, x, d):
        return 8 + t * 32 * (m + 1) + (x * (m + 1) + d) * 16
    for t, x in ((0, 1), (1, 0), (1, 1)):
        k[off(t, x, 0):off(t, x, 0) + 16] = 0
    return k.tobytes()


@pytest.mark.parametrize("prf", [0, 1])
def test_branch_parallel_equals_level_by_level(orc, prf):
    rng = np.random.default_rng(100 + prf)
    for m in (1, 2, 3, 5, 8, 10):
        key = random_key(rng, m, prf)
        leaves = orc.eval_all(key)
        js = range(1 << m) if m <= 8 else rng.integers(0, 1 << m, 64)
        for j in js:
            assert orc.eval_point(key, int(j)) == leaves[int(j)].tobytes()


@pytest.mark.parametrize("prf", [0, 1])
def test_closed_form_depth_two_with_library_aes(orc, prf):
    """R(2, j) spelled out with a library AES and explicit wire offsets."""
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")

    def aes(k, b):
        e = ciphers.Cipher(ciphers.algorithms.AES(k), ciphers.modes.ECB()).encryptor()
        return e.update(b) + e.finalize()

    mmo = [b"IM-PIR MMO key 0", b"IM-PIR MMO key 1"]

    def f(s, x):
        if prf == 0:
            return aes(s, bytes([x]) + bytes(15))
        return bytes(a ^ b for a, b in zip(aes(mmo[x], s), s))

    m = 2
    key = random_key(np.random.default_rng(5 + prf), m, prf)

    def C(t, x, d):
        o = 8 + t * 32 * (m + 1) + (x * (m + 1) + d) * 16
        return key[o:o + 16]

    def xor(a, b):
        return bytes(u ^ v for u, v in zip(a, b))

    root = C(0, 0, 0)
    for j in range(4):
        p = xor(f(root, j >> 1), C(root[0] & 1, j >> 1, 1))
        leaf = xor(f(p, j & 1), C(p[0] & 1, j & 1, 2))
        assert orc.eval_point(key, j) == leaf


@pytest.mark.parametrize("prf", [0, 1])
def test_dpf_property_brute_force(orc, prf):
    """Eval(k0, j) ^ Eval(k1, j) = [j == alpha] as 128-bit values, every j: every alpha for
    domains up to 2^10, 16 random alphas for 2^11 and 2^12."""
    one = bytes([1]) + bytes(15)
    rng = np.random.default_rng(11 + prf)
    for m in range(1, 13):
        alphas = range(1 << m) if m <= 10 else rng.integers(0, 1 << m, 16)
        for a in alphas:
            seed = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
            k0, k1 = orc.gen(int(a), m, prf, seed)
            l0, l1 = orc.eval_all(k0), orc.eval_all(k1)
            x = l0 ^ l1
            want = np.zeros_like(x)
            want[int(a)] = np.frombuffer(one, np.uint8)
            assert np.array_equal(x, want), (m, a)


def test_gen_key_shape(orc):
    m, a = 9, 300
    k0, k1 = orc.gen(a, m, 0, bytes(range(32)))
    assert len(k0) == len(k1) == 8 + 64 * (m + 1) == orc.key_bytes(m)
    assert k0[:8] == bytes([1, 0, m, 0, 0, 0, 0, 0])
    assert orc.key_check(k0) == 0 and orc.key_check(k1) == 0
    def off(t, x, d):
        return 8 + t * 32 * (m + 1) + (x * (m + 1) + d) * 16
    # the roots differ and their control bits differ
    assert k0[off(0, 0, 0)] & 1 != k1[off(0, 0, 0)] & 1
    # columns 1..m are shared by both keys
    for t in (0, 1):
        for x in (0, 1):
            for d in range(1, m + 1):
                assert k0[off(t, x, d):off(t, x, d) + 16] == k1[off(t, x, d):off(t, x, d) + 16]
    # deterministic in the seed
    assert orc.gen(a, m, 0, bytes(range(32))) == (k0, k1)


def test_key_validation(orc):
    k0, _ = orc.gen(3, 4, 0, bytes(32))
    bad = bytearray(k0)
    bad[0] = 2
    assert orc.key_check(bytes(bad)) != 0
    bad = bytearray(k0)
    bad[8 + 16] = 1  # C_0[0][1]... is column 1 of row 0: allowed; use C_0[1][0] instead
    assert orc.key_check(bytes(bad)) == 0
    bad = bytearray(k0)
    bad[8 + (1 * 5 + 0) * 16] = 1  # C_0[1][0] must be zero
    assert orc.key_check(bytes(bad)) != 0
    bad = bytearray(k0)
    bad[2] = 41
    assert orc.key_check(bytes(bad)) != 0
