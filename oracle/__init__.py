"""CPU oracle for IM-PIR's server side (DPF EvalAll + dpXOR), loaded through ctypes.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers. The product (``paper_2509_06514_gb300``) never imports
this package, and this package never imports the product.

The arithmetic lives in ``impir_oracle.c`` (plain C, byte-oriented AES from FIPS-197, the
GGM tree of Eqs. (1)-(3) of §3.2, dpXOR of §2.3/§3.3); this file only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "impir_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PRF_KEYED = 0
PRF_MMO = 1


def build(force: bool = False) -> str:
    """Compile impir_oracle.c into liboracle.so with gcc (plain -O2, no intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.c_void_p
            lib.orc_aes128_encrypt.argtypes = [u8p, u8p, u8p]
            lib.orc_aes128_round_keys.argtypes = [u8p, u8p]
            lib.orc_sbox.argtypes = [ctypes.c_uint8]
            lib.orc_sbox.restype = ctypes.c_uint8
            lib.orc_prf.argtypes = [ctypes.c_int, u8p, ctypes.c_int, u8p]
            lib.orc_key_bytes.argtypes = [ctypes.c_uint32]
            lib.orc_key_bytes.restype = ctypes.c_size_t
            lib.orc_key_check.argtypes = [u8p]
            lib.orc_eval_point.argtypes = [u8p, ctypes.c_uint64, u8p]
            lib.orc_eval_all.argtypes = [u8p, u8p]
            lib.orc_eval_bits.argtypes = [u8p, ctypes.c_uint64, u8p]
            lib.orc_dpxor.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, u8p, u8p]
            lib.orc_dpxor.restype = None
            lib.orc_answer.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32, u8p]
            lib.orc_answer_points.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32, u8p]
            lib.orc_answer_add32.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32, u8p]
            lib.orc_reconstruct_add32.argtypes = [u8p, u8p, ctypes.c_uint32, u8p]
            lib.orc_reconstruct_add32.restype = None
            lib.orc_answer_threads.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32, u8p, ctypes.c_int]
            lib.orc_gen.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, u8p, u8p, u8p]
            lib.orc_reconstruct.argtypes = [u8p, u8p, ctypes.c_uint32, u8p]
            lib.orc_reconstruct.restype = None
            lib.orc_aes_per_eval.argtypes = [ctypes.c_uint32]
            lib.orc_aes_per_eval.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def aes128_encrypt(key, block) -> bytes:
    k, b, out = _u8(key), _u8(block), np.zeros(16, np.uint8)
    _load().orc_aes128_encrypt(_ptr(k), _ptr(b), _ptr(out))
    return out.tobytes()


def aes128_round_keys(key) -> bytes:
    k, out = _u8(key), np.zeros(176, np.uint8)
    _load().orc_aes128_round_keys(_ptr(k), _ptr(out))
    return out.tobytes()


def sbox(x: int) -> int:
    return int(_load().orc_sbox(x))


def prf(kind: int, seed, x: int) -> bytes:
    s, out = _u8(seed), np.zeros(16, np.uint8)
    _load().orc_prf(kind, _ptr(s), x, _ptr(out))
    return out.tobytes()


def key_bytes(m: int) -> int:
    return int(_load().orc_key_bytes(m))


def key_check(key) -> int:
    return int(_load().orc_key_check(_ptr(_u8(key))))


def eval_point(key, j: int) -> bytes:
    k, out = _u8(key), np.zeros(16, np.uint8)
    _check(_load().orc_eval_point(_ptr(k), j, _ptr(out)), "eval_point")
    return out.tobytes()


def eval_all(key) -> np.ndarray:
    """All 2^m leaves, shape (2^m, 16) uint8, level by level."""
    k = _u8(key)
    m = int(k[2])
    out = np.zeros((1 << m, 16), np.uint8)
    _check(_load().orc_eval_all(_ptr(k), _ptr(out)), "eval_all")
    return out


def eval_bits(key, n: int | None = None) -> np.ndarray:
    k = _u8(key)
    m = int(k[2])
    n = (1 << m) if n is None else n
    out = np.zeros(n, np.uint8)
    _check(_load().orc_eval_bits(_ptr(k), n, _ptr(out)), "eval_bits")
    return out


def dpxor(db: np.ndarray, bits: np.ndarray, record_bytes: int) -> bytes:
    """XOR of the records whose bit is set (§2.3); db is (n, record_bytes) or flat."""
    d = np.ascontiguousarray(db, dtype=np.uint8).reshape(-1)
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    n = len(b)
    assert d.size >= n * record_bytes
    out = np.zeros(record_bytes, np.uint8)
    _load().orc_dpxor(_ptr(d), n, record_bytes, _ptr(b), _ptr(out))
    return out.tobytes()


def answer(key, db: np.ndarray, n_records: int, record_bytes: int, threads: int = 1) -> bytes:
    """One server's answer r = XOR_j v[j] D[j] over j < min(N, 2^m)."""
    k = _u8(key)
    d = np.ascontiguousarray(db, dtype=np.uint8).reshape(-1)
    assert d.size >= n_records * record_bytes
    out = np.zeros(record_bytes, np.uint8)
    if threads <= 1:
        _check(_load().orc_answer(_ptr(k), _ptr(d), n_records, record_bytes, _ptr(out)), "answer")
    else:
        _check(
            _load().orc_answer_threads(_ptr(k), _ptr(d), n_records, record_bytes, _ptr(out), threads),
            "answer_threads",
        )
    return out.tobytes()


def answer_points(key, db: np.ndarray, n_records: int, record_bytes: int) -> bytes:
    """Same answer, every record's leaf from its own root-to-leaf walk (any domain size)."""
    k = _u8(key)
    d = np.ascontiguousarray(db, dtype=np.uint8).reshape(-1)
    out = np.zeros(record_bytes, np.uint8)
    _check(_load().orc_answer_points(_ptr(k), _ptr(d), n_records, record_bytes, _ptr(out)), "answer_points")
    return out.tobytes()


def answer_add32(key, db: np.ndarray, n_records: int, record_bytes: int) -> bytes:
    """Additive answer over Z_{2^32}: sum_j (-1)^party low32(R(m,j)) * D[j], word by word."""
    k = _u8(key)
    d = np.ascontiguousarray(db, dtype=np.uint8).reshape(-1)
    out = np.zeros(record_bytes, np.uint8)
    _check(_load().orc_answer_add32(_ptr(k), _ptr(d), n_records, record_bytes, _ptr(out)), "answer_add32")
    return out.tobytes()


def reconstruct_add32(r0: bytes, r1: bytes) -> bytes:
    a, b = _u8(r0), _u8(r1)
    out = np.zeros(len(a), np.uint8)
    _load().orc_reconstruct_add32(_ptr(a), _ptr(b), len(a), _ptr(out))
    return out.tobytes()


def gen(alpha: int, m: int, prf_kind: int, seed: bytes) -> tuple[bytes, bytes]:
    assert len(seed) == 32
    kb = key_bytes(m)
    k0, k1, s = np.zeros(kb, np.uint8), np.zeros(kb, np.uint8), _u8(seed)
    _check(_load().orc_gen(alpha, m, prf_kind, _ptr(s), _ptr(k0), _ptr(k1)), "gen")
    return k0.tobytes(), k1.tobytes()


def reconstruct(r0: bytes, r1: bytes) -> bytes:
    a, b = _u8(r0), _u8(r1)
    out = np.zeros(len(a), np.uint8)
    _load().orc_reconstruct(_ptr(a), _ptr(b), len(a), _ptr(out))
    return out.tobytes()


def aes_per_eval(m: int) -> int:
    return int(_load().orc_aes_per_eval(m))
