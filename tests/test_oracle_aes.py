"""Pins for the oracle's AES-128 (the PRF of §3.2 / §4): FIPS-197 known answers and a
library AES (OpenSSL through `cryptography`) on random keys and blocks."""
import numpy as np
import pytest

from conftest import golden_lines


def test_fips197_cipher_vectors(orc):
    rows = golden_lines("fips197_aes128.txt")
    assert len(rows) == 2
    for key, pt, ct in rows:
        assert orc.aes128_encrypt(bytes.fromhex(key), bytes.fromhex(pt)).hex() == ct


def test_fips197_key_expansion(orc):
    rows = golden_lines("fips197_key_expansion.txt")
    key = bytes.fromhex(rows[0][1])
    rk = orc.aes128_round_keys(key)
    assert rk[:16] == key
    for idx, word in rows[1:]:
        i = int(idx)
        assert rk[4 * i:4 * i + 4].hex() == word


def test_fips197_sbox_entries(orc):
    for x, y in golden_lines("fips197_sbox.txt"):
        assert orc.sbox(int(x, 16)) == int(y, 16)
    assert sorted(orc.sbox(x) for x in range(256)) == list(range(256))  # a permutation


def test_aes_matches_library_on_random_inputs(orc):
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.default_rng(197)
    for _ in range(10000):
        key = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        pt = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        enc = ciphers.Cipher(ciphers.algorithms.AES(key), ciphers.modes.ECB()).encryptor()
        assert orc.aes128_encrypt(key, pt) == enc.update(pt) + enc.finalize()


def test_prf_definitions_match_library(orc):
    """PRF_s(x) = AES with key s over enc(x) (byte 0 = x); MMO: AES_{K_x}(s) ^ s."""
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")

    def aes(k, b):
        e = ciphers.Cipher(ciphers.algorithms.AES(k), ciphers.modes.ECB()).encryptor()
        return e.update(b) + e.finalize()

    mmo_keys = [b"IM-PIR MMO key 0", b"IM-PIR MMO key 1"]
    rng = np.random.default_rng(7)
    for _ in range(300):
        s = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        for x in (0, 1):
            assert orc.prf(orc.PRF_KEYED, s, x) == aes(s, bytes([x]) + bytes(15))
            want = bytes(a ^ b for a, b in zip(aes(mmo_keys[x], s), s))
            assert orc.prf(orc.PRF_MMO, s, x) == want
