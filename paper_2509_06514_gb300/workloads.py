"""Seeded synthetic inputs shaped like IM-PIR's workloads (§5: random fixed-size records).

This module holds none of the PIR method's arithmetic. It produces the database bytes, the
query targets, the domain sizes, the batch splits, the per-query key-generation seeds and the
arrival times that the CUDA path, the CPU oracle, the tests and the benchmark all consume.

Database bytes come from a counter-based SplitMix64 stream (``inputs_gen.c``), so any record
can be regenerated on its own; everything else comes from numpy's PCG64 with a fixed seed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "inputs_gen.c")
_LIB = os.path.join(_HERE, "libimpir_inputs.so")
_lock = threading.Lock()
_lib = None

GAMMA = 0x9E3779B97F4A7C15


def build_inputs(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_inputs())
            lib.impir_inputs_fill.argtypes = [
                ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            lib.impir_inputs_fill.restype = ctypes.c_int
            _lib = lib
    return _lib


def stream_bytes(n: int, seed: int, offset: int = 0, threads: int | None = None) -> np.ndarray:
    """Bytes [offset, offset+n) of SplitMix64 stream `seed`, as a uint8 array."""
    out = np.empty(n, np.uint8)
    if n:
        threads = threads or min(64, os.cpu_count() or 1)
        _load().impir_inputs_fill(ctypes.c_void_p(out.ctypes.data), n, seed & (2**64 - 1), offset, threads)
    return out


def stream_bytes_numpy(n: int, seed: int, offset: int = 0) -> np.ndarray:
    """Plain numpy restatement of the same stream, used to cross-check the C helper."""
    if n == 0:
        return np.zeros(0, np.uint8)
    w0, w1 = offset // 8, (offset + n + 7) // 8
    with np.errstate(over="ignore"):
        i = np.arange(w0, w1, dtype=np.uint64)
        z = np.uint64(seed & (2**64 - 1)) + (i + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    b = z.astype("<u8").view(np.uint8)
    s = offset - 8 * w0
    return b[s:s + n].copy()


def make_db(n_records: int, record_bytes: int, seed: int) -> np.ndarray:
    """Uniform random database, shape (N, B) uint8, row-major (§3.3 preloads it once)."""
    return stream_bytes(n_records * record_bytes, seed).reshape(n_records, record_bytes)


def record(n_records: int, record_bytes: int, seed: int, j: int) -> bytes:
    """Record j of make_db(N, B, seed), regenerated alone."""
    assert 0 <= j < n_records
    return stream_bytes(record_bytes, seed, offset=j * record_bytes, threads=1).tobytes()


def key_seed(base: int, q: int) -> bytes:
    """32-byte key-generation seed for query q of a workload."""
    rng = np.random.default_rng([base & 0xFFFFFFFF, q])
    return rng.integers(0, 256, 32, dtype=np.uint8).tobytes()


@dataclass
class Batch:
    ms: list[int]          # domain bits of each query
    alphas: list[int]      # target index of each query (alpha < 2^m)
    seeds: list[bytes]     # key-generation seed of each query


@dataclass
class Workload:
    name: str
    n_records: int
    record_bytes: int
    db_seed: int
    batches: list[Batch] = field(default_factory=list)

    @property
    def n_queries(self) -> int:
        return sum(len(b.ms) for b in self.batches)

    @property
    def db_bytes(self) -> int:
        return self.n_records * self.record_bytes


def _batch(rng, n: int, ms, n_records: int, base_seed: int, q0: int) -> Batch:
    ms = [int(x) for x in ms]
    alphas = [int(rng.integers(0, min(1 << m, n_records))) for m in ms]
    seeds = [key_seed(base_seed, q0 + i) for i in range(n)]
    return Batch(ms=ms, alphas=alphas, seeds=seeds)


def single_query(seed: int = 0) -> Workload:
    """Plain two-server DPF-PIR, one query: N=2^16 x 32 B (2 MiB), domain 16 bits."""
    rng = np.random.default_rng(seed)
    w = Workload("single: N=2^16 x 32 B, m=16, 1 query", 1 << 16, 32, seed)
    w.batches.append(_batch(rng, 1, [16], w.n_records, seed + 1000, 0))
    return w


def batched_256mib(seed: int = 1, n_queries: int = 64) -> Workload:
    """Batched: N=2^20 x 256 B (256 MiB), n_queries (64) queries, domain 20 bits, one launch."""
    rng = np.random.default_rng(seed)
    w = Workload(f"batched: N=2^20 x 256 B, m=20, Q={n_queries}", 1 << 20, 256, seed)
    w.batches.append(_batch(rng, n_queries, [20] * n_queries, w.n_records, seed + 1000, 0))
    return w


def batched_4gib(seed: int = 2, record_bytes: int = 1024, db_bytes: int = 4 << 30) -> Workload:
    """Batched GB-scale: 4 GiB (db_bytes) of records of record_bytes (a power of two; default
    1 KiB: N=2^22), 256 queries whose domain covers the DB (m = log2 N)."""
    assert record_bytes > 0 and record_bytes & (record_bytes - 1) == 0
    n = db_bytes // record_bytes
    m = log2_exact(n)
    rng = np.random.default_rng(seed)
    name = (f"batched: N=2^{m} x {record_bytes // 1024} KiB, m={m}, Q=256" if record_bytes >= 1024
            else f"batched: N=2^{m} x {record_bytes} B, m={m}, Q=256")
    w = Workload(name, n, record_bytes, seed)
    w.batches.append(_batch(rng, 256, [m] * 256, w.n_records, seed + 1000, 0))
    return w


def uneven_8gib(seed: int = 3, n_queries: int = 1024, max_batch: int = 512, log2n: int = 25) -> Workload:
    """Batched uneven: N=2^25 x 256 B (8 GiB); n_queries split into batches of uniform
    size 1..max_batch (the last one truncated), domains mixed over 2^23, 2^24, 2^25, each
    query against the DB prefix its domain covers. log2n < 25 gives the same batch sizes over a
    smaller database (N = 2^log2n, domains 2^(log2n-2) .. 2^log2n), for profiling captures."""
    rng = np.random.default_rng(seed)
    mset = [log2n - 2, log2n - 1, log2n]
    w = Workload(f"uneven: N=2^{log2n} x 256 B, m in {{{','.join(map(str, mset))}}}, {n_queries} queries in "
                 f"batches of 1..{max_batch}", 1 << log2n, 256, seed)
    q = 0
    while q < n_queries:
        n = min(int(rng.integers(1, max_batch + 1)), n_queries - q)
        ms = rng.choice(mset, size=n)
        w.batches.append(_batch(rng, n, ms, w.n_records, seed + 1000, q))
        q += n
    return w


SERVING_DBS = [(1 << 18, 64), (1 << 22, 256), (1 << 24, 512)]
SERVING_RATES = [5_000, 10_000, 20_000, 50_000, 100_000, 200_000]
# offered loads below the server's capacity (about 3k queries/s here), for latency context
SERVING_LOW_RATES = [500, 1_000, 2_000]


@dataclass
class Arrivals:
    t: np.ndarray        # arrival time of each request, seconds from start
    db: np.ndarray       # index into SERVING_DBS
    alpha: np.ndarray    # target record
    seeds: list[bytes]


def poisson_arrivals(rate: float, n: int, seed: int = 5, dbs=SERVING_DBS) -> Arrivals:
    """Poisson arrivals at `rate` req/s, uniform DB choice and uniform target."""
    rng = np.random.default_rng([seed, int(rate)])
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    db = rng.integers(0, len(dbs), size=n)
    alpha = np.array([int(rng.integers(0, dbs[d][0])) for d in db], dtype=np.int64)
    seeds = [key_seed(seed * 7919 + int(rate), i) for i in range(n)]
    return Arrivals(t=t, db=db, alpha=alpha, seeds=seeds)


def log2_exact(n: int) -> int:
    assert n > 0 and n & (n - 1) == 0
    return n.bit_length() - 1
