"""Planted-mistake check of the oracle's pins: each mutant is a copy of oracle/impir_oracle.c
with one plausible error (a wrong constant, a transposed index, a dropped term, an inverted
test), compiled on the CPU into its own library. The pin battery below (FIPS-197 vectors,
a library AES, the two tree evaluation orders, brute-force DPF correctness, the Fig. 2
example, reconstruction, the threaded split) must reject every mutant, and accept the
unmodified source."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from conftest import golden_lines

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "impir_oracle.c")

MUTANTS = {
    "xtime_polynomial": ("return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00));",
                         "return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1d : 0x00));"),
    "shiftrows_direction": ("for (int c = 0; c < 4; c++) tmp[c] = st[r][(c + r) % 4];",
                            "for (int c = 0; c < 4; c++) tmp[c] = st[r][(c - r + 4) % 4];"),
    "mixcolumns_coefficient": ("st[0][c] = (uint8_t)(xtime(a0) ^ (xtime(a1) ^ a1) ^ a2 ^ a3);",
                               "st[0][c] = (uint8_t)((xtime(a0) ^ a0) ^ xtime(a1) ^ a2 ^ a3);"),
    "rotword_dropped": ("            temp[0] = temp[1];\n            temp[1] = temp[2];\n            temp[2] = temp[3];\n            temp[3] = t0;\n",
                        "            (void)t0;\n"),
    "rcon_value": ("0x80, 0x1b, 0x36};", "0x80, 0x36, 0x1b};"),
    "affine_constant": ("((0x63 >> i) & 1)", "((0x62 >> i) & 1)"),
    "prf_plaintext_byte": ("blk[0] = (uint8_t)x;", "blk[15] = (uint8_t)x;"),
    "mmo_feed_forward_dropped": ("for (int i = 0; i < 16; i++) out[i] = e[i] ^ s[i];",
                                 "for (int i = 0; i < 16; i++) out[i] = e[i];"),
    "control_bit_byte": ("int t = p[0] & 1; /* \"R(d-1, j/2) mod 2\" */", "int t = p[15] & 1;"),
    "codeword_index_transposed": ("const uint8_t* c = cw(k, t, x, d);", "const uint8_t* c = cw(k, x, t, d);"),
    "codeword_wrong_depth": ("const uint8_t* c = cw(k, t, x, d);", "const uint8_t* c = cw(k, t, x, d - 1);"),
    "root_from_wrong_codeword": ("        memcpy(out, cw(k, 0, 0, 0), 16);\n        return;",
                                 "        memcpy(out, cw(k, 1, 0, 0), 16);\n        return;"),
    "correction_term_dropped": ("for (int i = 0; i < 16; i++) out[i] = f[i] ^ c[i];",
                                "for (int i = 0; i < 16; i++) out[i] = f[i];"),
    "selection_inverted": ("        if (bits[j] & 1) {\n            const uint8_t* rec = db + j * (uint64_t)record_bytes;",
                           "        if (!(bits[j] & 1)) {\n            const uint8_t* rec = db + j * (uint64_t)record_bytes;"),
    "leaf_bit_from_wrong_byte": ("for (uint64_t j = 0; j < n; j++) bits[j] = leaves[16 * j] & 1;",
                                 "for (uint64_t j = 0; j < n; j++) bits[j] = leaves[16 * j + 15] & 1;"),
    "gen_leaf_offset": ("delta[0] = 1; /* b = 1: the leaves differ by the integer 1 */", "delta[0] = 3;"),
    "gen_path_bit_order": ("int ad = (int)((alpha >> (m - d)) & 1);", "int ad = (int)((alpha >> (d - 1)) & 1);"),
    "threaded_subtree_base": ("uint64_t base = s << h;", "uint64_t base = s << (h - 1);"),
    "additive_sign_dropped": ("if (k.party) v = 0u - v;", "(void)k.party;"),
    "additive_share_high_bytes": ("uint32_t v = (uint32_t)leaf[0] | ((uint32_t)leaf[1] << 8)",
                                  "uint32_t v = (uint32_t)leaf[12] | ((uint32_t)leaf[1] << 8)"),
    "dpxor_range_off_by_one": ("for (uint64_t j = 0; j < n; j++) {\n        if (bits[j] & 1) {",
                               "for (uint64_t j = 1; j < n; j++) {\n        if (bits[j] & 1) {"),
}


def build_variant(tmp_path, name, old_new):
    src = open(SRC).read()
    if old_new is not None:
        old, new = old_new
        assert src.count(old) >= 1, f"mutation site for {name} not found"
        src = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-w", "-o", str(so), str(c)])
    lib = ctypes.CDLL(str(so))
    vp = ctypes.c_void_p
    lib.orc_aes128_encrypt.argtypes = [vp, vp, vp]
    lib.orc_prf.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp]
    lib.orc_eval_point.argtypes = [vp, ctypes.c_uint64, vp]
    lib.orc_eval_all.argtypes = [vp, vp]
    lib.orc_dpxor.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32, vp, vp]
    lib.orc_dpxor.restype = None
    lib.orc_answer.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp]
    lib.orc_answer_threads.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp, ctypes.c_int]
    lib.orc_gen.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, vp, vp, vp]
    lib.orc_answer_add32.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp]
    lib.orc_reconstruct_add32.argtypes = [vp, vp, ctypes.c_uint32, vp]
    lib.orc_reconstruct_add32.restype = None
    return lib


def P(a):
    return ctypes.c_void_p(a.ctypes.data)


def pins(lib):
    """Names of the pins the library fails (empty when it passes them all)."""
    failed = []
    # FIPS-197 known answers
    for key, pt, ct in golden_lines("fips197_aes128.txt"):
        k, b, o = (np.frombuffer(bytes.fromhex(key), np.uint8).copy(),
                   np.frombuffer(bytes.fromhex(pt), np.uint8).copy(), np.zeros(16, np.uint8))
        lib.orc_aes128_encrypt(P(k), P(b), P(o))
        if o.tobytes().hex() != ct:
            failed.append("fips197")
            break
    # PRF definitions against a library AES
    try:
        from cryptography.hazmat.primitives.ciphers import Cipher, algorithms, modes

        def aes(k, b):
            e = Cipher(algorithms.AES(k), modes.ECB()).encryptor()
            return e.update(b) + e.finalize()
        rng = np.random.default_rng(1)
        for _ in range(20):
            s = rng.integers(0, 256, 16, dtype=np.uint8)
            for prf, x in ((0, 0), (0, 1), (1, 0), (1, 1)):
                o = np.zeros(16, np.uint8)
                lib.orc_prf(prf, P(s), x, P(o))
                want = aes(s.tobytes(), bytes([x]) + bytes(15)) if prf == 0 else bytes(
                    a ^ b for a, b in zip(aes(b"IM-PIR MMO key %d" % x, s.tobytes()), s.tobytes()))
                if o.tobytes() != want:
                    failed.append("prf_library")
                    raise StopIteration
    except StopIteration:
        pass
    except ImportError:
        pass
    # DPF brute force over tiny domains, both PRFs
    rng = np.random.default_rng(2)
    one = np.zeros(16, np.uint8)
    one[0] = 1
    try:
        for prf in (0, 1):
            for m in range(1, 7):
                for a in (range(1 << m) if m <= 3 else rng.integers(0, 1 << m, 3)):
                    kb = 8 + 64 * (m + 1)
                    k0, k1 = np.zeros(kb, np.uint8), np.zeros(kb, np.uint8)
                    seed = rng.integers(0, 256, 32, dtype=np.uint8)
                    assert lib.orc_gen(int(a), m, prf, P(seed), P(k0), P(k1)) == 0
                    l0, l1 = np.zeros((1 << m, 16), np.uint8), np.zeros((1 << m, 16), np.uint8)
                    lib.orc_eval_all(P(k0), P(l0))
                    lib.orc_eval_all(P(k1), P(l1))
                    want = np.zeros_like(l0)
                    want[int(a)] = one
                    if not np.array_equal(l0 ^ l1, want):
                        raise StopIteration
    except StopIteration:
        failed.append("dpf_brute_force")
    # the two evaluation orders agree on a key with random codewords
    m = 6
    kb = 8 + 64 * (m + 1)
    key = rng.integers(0, 256, kb, dtype=np.uint8)
    key[:8] = [1, 0, m, 0, 0, 0, 0, 0]
    for t, x in ((0, 1), (1, 0), (1, 1)):
        o = 8 + t * 32 * (m + 1) + x * (m + 1) * 16
        key[o:o + 16] = 0
    leaves = np.zeros((1 << m, 16), np.uint8)
    lib.orc_eval_all(P(key), P(leaves))
    for j in range(1 << m):
        o = np.zeros(16, np.uint8)
        lib.orc_eval_point(P(key), j, P(o))
        if not np.array_equal(o, leaves[j]):
            failed.append("two_orders")
            break
    # Fig. 2 worked example
    g = {r[0]: r[1:] for r in golden_lines("fig2_dpxor.txt")}
    db = np.array([int(s, 2) for s in g["db"]], np.uint8)
    for v, r in (("v1", "r1"), ("v2", "r2")):
        bits = np.array([int(b) for b in g[v]], np.uint8)
        o = np.zeros(1, np.uint8)
        lib.orc_dpxor(P(db), 4, 1, P(bits), P(o))
        if o[0] != int(g[r][0], 2):
            failed.append("fig2")
            break
    # dpXOR special cases: a unit selection returns exactly that record, none returns zero
    dbs = rng.integers(0, 256, (9, 5), dtype=np.uint8)
    for sel, want in ((np.eye(9, dtype=np.uint8)[4], dbs[4]), (np.zeros(9, np.uint8), np.zeros(5, np.uint8))):
        o = np.zeros(5, np.uint8)
        lib.orc_dpxor(P(dbs), 9, 5, P(np.ascontiguousarray(sel)), P(o))
        if not np.array_equal(o, want):
            failed.append("dpxor_special")
            break
    # additive answer: r_0 + r_1 = D[alpha] (mod 2^32 per word)
    Na, Ba, ma = 200, 12, 8
    dba = rng.integers(0, 256, (Na, Ba), dtype=np.uint8)
    for a in (3, 199):
        kb = 8 + 64 * (ma + 1)
        k0, k1 = np.zeros(kb, np.uint8), np.zeros(kb, np.uint8)
        seed = rng.integers(0, 256, 32, dtype=np.uint8)
        lib.orc_gen(a, ma, 0, P(seed), P(k0), P(k1))
        r0, r1, rr = np.zeros(Ba, np.uint8), np.zeros(Ba, np.uint8), np.zeros(Ba, np.uint8)
        lib.orc_answer_add32(P(k0), P(dba), Na, Ba, P(r0))
        lib.orc_answer_add32(P(k1), P(dba), Na, Ba, P(r1))
        lib.orc_reconstruct_add32(P(r0), P(r1), Ba, P(rr))
        if not np.array_equal(rr, dba[a]):
            failed.append("additive_reconstruction")
            break
    # reconstruction and the threaded split on a small DB
    N, B, m = 300, 7, 9
    dbr = rng.integers(0, 256, (N, B), dtype=np.uint8)
    for a in (0, 5, 299):
        kb = 8 + 64 * (m + 1)
        k0, k1 = np.zeros(kb, np.uint8), np.zeros(kb, np.uint8)
        seed = rng.integers(0, 256, 32, dtype=np.uint8)
        lib.orc_gen(a, m, 0, P(seed), P(k0), P(k1))
        r0, r1, rt = np.zeros(B, np.uint8), np.zeros(B, np.uint8), np.zeros(B, np.uint8)
        lib.orc_answer(P(k0), P(dbr), N, B, P(r0))
        lib.orc_answer(P(k1), P(dbr), N, B, P(r1))
        lib.orc_answer_threads(P(k0), P(dbr), N, B, P(rt), 3)
        if not np.array_equal(r0 ^ r1, dbr[a]):
            failed.append("reconstruction")
            break
        if not np.array_equal(rt, r0):
            failed.append("threaded_split")
            break
    return failed


def test_unmodified_oracle_passes_every_pin(tmp_path):
    assert pins(build_variant(tmp_path, "original", None)) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(tmp_path, name):
    failed = pins(build_variant(tmp_path, name, MUTANTS[name]))
    assert failed, f"mutant {name} survived every pin"
