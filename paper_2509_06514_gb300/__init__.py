"""GB300 server side of two-server DPF-based PIR (IM-PIR, arXiv 2509.06514).

A thin ctypes binding over ``libimpir.so`` (C ABI in ``include/impir.h``). Every call has
the C name and only marshals arguments; every step of the answer path runs in the
library's CUDA kernels. There is no CPU fallback: if the library is missing or no CUDA
device is present, calls raise.

Host buffers are ``bytes`` / numpy uint8 arrays; device buffers are torch CUDA tensors
(torch supplies device memory and streams) or raw integer device pointers.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# IMPIR_BOUNDS=1 in the environment loads the debug build with index checks instead
# (libimpir_bounds.so, from `python -m paper_2509_06514_gb300.build --bounds`).
BOUNDS = os.environ.get("IMPIR_BOUNDS") == "1"
LIB_PATH = os.path.join(_HERE, "libimpir_bounds.so" if BOUNDS else "libimpir.so")

IMPIR_OK, IMPIR_EINVAL, IMPIR_ENOMEM, IMPIR_ECUDA, IMPIR_ETIMEOUT, IMPIR_EBUSY = range(6)
IMPIR_PRF_AES_KEYED = 0
IMPIR_PRF_AES_MMO = 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY"}

# Every symbol include/impir.h declares.
EXPORTS = [
    "impir_key_bytes", "impir_db_load", "impir_db_attach", "impir_db_free", "impir_db_info", "impir_answer",
    "impir_workspace_bytes", "impir_answer_async", "impir_workspace_status", "impir_get_config",
    "impir_set_config", "impir_autotune", "dpf_gen", "impir_reconstruct", "impir_last_error",
    "impir_device_sm_count", "impir_timing_enable", "impir_timing_read", "impir_answer_noalloc",
    "impir_server_create", "impir_server_submit", "impir_server_take", "impir_server_stats", "impir_server_destroy",
    "impir_aes_calibrate", "impir_db_update", "impir_db_update_async", "impir_db_version", "impir_server_update",
    "impir_answer_streamed", "impir_answer_add32", "impir_answer_add32_async", "impir_tune_cache_save",
    "impir_tune_cache_load", "impir_db_load_rows", "impir_db_rows", "impir_combine_partials",
    "impir_get_config_add32", "impir_bounds_status", "impir_aes_calibrate_bitsliced",
]


class ImpirError(RuntimeError):
    def __init__(self, status: int, what: str, message: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class impir_config(ctypes.Structure):
    _fields_ = [("lane_bits", ctypes.c_uint32), ("queries_per_warp", ctypes.c_uint32),
                ("warps_per_cta", ctypes.c_uint32), ("queries_per_launch", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class impir_server_config(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("streams", ctypes.c_uint32), ("max_record_bytes", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("accumulator_budget", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libimpir.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run "
                                  "__graft_entry__.build() or python -m paper_2509_06514_gb300.build"
                                  + (" --bounds" if BOUNDS else ""))
            L = ctypes.CDLL(LIB_PATH)
            vp, u8p = ctypes.c_void_p, ctypes.c_void_p
            sig = {
                "impir_key_bytes": (ctypes.c_size_t, [ctypes.c_uint32]),
                "impir_db_load": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]),
                "impir_db_attach": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                                   ctypes.POINTER(ctypes.c_int32)]),
                "impir_db_free": (ctypes.c_int, [ctypes.c_int32]),
                "impir_db_info": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                                                 ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                                 ctypes.POINTER(ctypes.c_void_p)]),
                "impir_answer": (ctypes.c_int, [ctypes.c_int32, u8p, ctypes.c_uint32, u8p]),
                "impir_workspace_bytes": (ctypes.c_size_t, [ctypes.c_uint32, ctypes.c_uint32]),
                "impir_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
                "impir_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint32)]),
                "impir_answer_add32": (ctypes.c_int, [ctypes.c_int32, u8p, ctypes.c_uint32, u8p]),
                "impir_answer_add32_async": (ctypes.c_int, [ctypes.c_int32, vp, vp, ctypes.c_uint32, vp, vp,
                                                            ctypes.c_size_t, vp]),
                "impir_answer_async": (ctypes.c_int, [ctypes.c_int32, vp, vp, ctypes.c_uint32, vp, vp,
                                                      ctypes.c_size_t, vp]),
                "impir_workspace_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_uint32),
                                                          ctypes.POINTER(ctypes.c_uint32)]),
                "impir_get_config": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(impir_config)]),
                "impir_get_config_add32": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(impir_config)]),
                "impir_set_config": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(impir_config)]),
                "impir_autotune": (ctypes.c_int, [ctypes.c_int32, vp, vp, ctypes.c_uint32, vp, vp, ctypes.c_size_t,
                                                  vp, ctypes.POINTER(impir_config)]),
                "dpf_gen": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, u8p, u8p, u8p]),
                "impir_reconstruct": (ctypes.c_int, [u8p, u8p, ctypes.c_uint32, u8p]),
                "impir_last_error": (ctypes.c_char_p, []),
                "impir_device_sm_count": (ctypes.c_int32, []),
                "impir_timing_enable": (ctypes.c_int, [ctypes.c_int]),
                "impir_aes_calibrate": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                       u8p, u8p, ctypes.POINTER(ctypes.c_double)]),
                "impir_server_create": (ctypes.c_int, [ctypes.POINTER(impir_server_config), ctypes.POINTER(ctypes.c_void_p)]),
                "impir_server_submit": (ctypes.c_int, [vp, ctypes.c_int32, u8p, ctypes.c_uint64]),
                "impir_server_take": (ctypes.c_int, [vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                                     ctypes.POINTER(ctypes.c_int32), u8p, ctypes.c_uint32,
                                                     ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64),
                                                     ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)]),
                "impir_server_update": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, vp]),
                "impir_db_update": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, vp]),
                "impir_db_update_async": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, vp, vp,
                                                         ctypes.POINTER(ctypes.c_uint64)]),
                "impir_db_version": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]),
                "impir_answer_streamed": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, u8p, ctypes.c_uint32, u8p,
                                                         ctypes.c_uint64, ctypes.POINTER(impir_config)]),
                "impir_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                                      ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
                "impir_server_destroy": (ctypes.c_int, [vp]),
                "impir_answer_noalloc": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vp, vp,
                                                        ctypes.c_uint32, vp, vp]),
                "impir_timing_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                                                     ctypes.POINTER(ctypes.c_uint64)]),
                "impir_db_load_rows": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                                      ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]),
                "impir_db_rows": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                                                 ctypes.POINTER(ctypes.c_uint64)]),
                "impir_combine_partials": (ctypes.c_int, [ctypes.c_int, vp, ctypes.c_uint32, ctypes.c_uint64, vp, vp]),
                "impir_bounds_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                                       ctypes.POINTER(ctypes.c_uint64)]),
                "impir_aes_calibrate_bitsliced": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                                 u8p, u8p, ctypes.POINTER(ctypes.c_double)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
    return _lib


def _check(st: int, what: str) -> None:
    if st != IMPIR_OK:
        raise ImpirError(st, what, lib().impir_last_error().decode(errors="replace"))


def _host(buf) -> tuple[np.ndarray, ctypes.c_void_p]:
    a = np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray, memoryview)) else \
        np.ascontiguousarray(buf, dtype=np.uint8)
    return a, ctypes.c_void_p(a.ctypes.data)


def _dev(x) -> ctypes.c_void_p:
    """Device pointer of a torch CUDA tensor, or an integer pointer."""
    if x is None:
        return ctypes.c_void_p(0)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"not a device buffer: {type(x)}")


def _stream(s) -> ctypes.c_void_p:
    if s is None:
        return ctypes.c_void_p(0)
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)


# ---- C ABI, same names ----

def impir_key_bytes(m: int) -> int:
    return int(lib().impir_key_bytes(m))


def impir_db_load(records, n_records: int, record_bytes: int) -> int:
    arr, p = _host(records)
    assert arr.size >= n_records * record_bytes
    h = ctypes.c_int32(0)
    _check(lib().impir_db_load(p, n_records, record_bytes, ctypes.byref(h)), "impir_db_load")
    return h.value


def impir_db_attach(d_records, n_records: int, record_bytes: int, stride_bytes: int) -> int:
    h = ctypes.c_int32(0)
    _check(lib().impir_db_attach(_dev(d_records), n_records, record_bytes, stride_bytes, ctypes.byref(h)),
           "impir_db_attach")
    return h.value


def impir_db_free(db: int) -> None:
    _check(lib().impir_db_free(db), "impir_db_free")


def impir_db_load_rows(records, n_rows: int, record_bytes: int, row_lo: int, n_total: int) -> int:
    """Row shard [row_lo, row_lo + n_rows) of an n_total-record database; `records` holds those rows."""
    arr, p = _host(records)
    assert arr.size >= n_rows * record_bytes
    h = ctypes.c_int32(0)
    _check(lib().impir_db_load_rows(p, n_rows, record_bytes, row_lo, n_total, ctypes.byref(h)), "impir_db_load_rows")
    return h.value


def impir_db_rows(db: int) -> tuple[int, int]:
    """(row_lo, n_total) of a handle."""
    lo, n = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().impir_db_rows(db, ctypes.byref(lo), ctypes.byref(n)), "impir_db_rows")
    return lo.value, n.value


def impir_combine_partials(mode: int, d_parts, n_parts: int, part_bytes: int, d_out, stream=None) -> None:
    """d_out = XOR (mode 0) or sum mod 2^32 (mode 1) of n_parts back-to-back device parts."""
    _check(lib().impir_combine_partials(mode, _dev(d_parts), n_parts, part_bytes, _dev(d_out), _stream(stream)),
           "impir_combine_partials")


def impir_db_info(db: int) -> dict:
    n, b, s, d = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_void_p()
    _check(lib().impir_db_info(db, ctypes.byref(n), ctypes.byref(b), ctypes.byref(s), ctypes.byref(d)),
           "impir_db_info")
    return {"n_records": n.value, "record_bytes": b.value, "stride_bytes": s.value, "d_records": d.value}


def impir_answer(db: int, keys, n_queries: int, record_bytes: int) -> np.ndarray:
    """Synchronous answer of n_queries host keys; returns (n_queries, record_bytes) uint8."""
    _, kp = _host(keys)
    out = np.zeros((n_queries, record_bytes), np.uint8)
    _check(lib().impir_answer(db, kp, n_queries, ctypes.c_void_p(out.ctypes.data)), "impir_answer")
    return out


def impir_answer_streamed(records, n_records: int, record_bytes: int, keys, n_queries: int, chunk_bytes: int):
    """Answer against a host-resident database streamed through the device in chunks.
    `records` is a numpy array or an integer host pointer; returns (answers, launch shape)."""
    if isinstance(records, int):
        rp = ctypes.c_void_p(records)
    else:
        arr, rp = _host(records)
        assert arr.size >= n_records * record_bytes
    _, kp = _host(keys)
    out = np.zeros((n_queries, record_bytes), np.uint8)
    cfg = impir_config()
    _check(lib().impir_answer_streamed(rp, n_records, record_bytes, kp, n_queries, ctypes.c_void_p(out.ctypes.data),
                                       chunk_bytes, ctypes.byref(cfg)), "impir_answer_streamed")
    return out, cfg.as_dict()


def impir_answer_add32(db: int, keys, n_queries: int, record_bytes: int) -> np.ndarray:
    """Additive answer over Z_2^32 (party from each key's header); (n_queries, record_bytes) uint8."""
    _, kp = _host(keys)
    out = np.zeros((n_queries, record_bytes), np.uint8)
    _check(lib().impir_answer_add32(db, kp, n_queries, ctypes.c_void_p(out.ctypes.data)), "impir_answer_add32")
    return out


def impir_answer_add32_async(db: int, d_keys, d_key_offsets, n_queries: int, d_out, d_workspace,
                             workspace_bytes: int, stream=None) -> None:
    _check(lib().impir_answer_add32_async(db, _dev(d_keys), _dev(d_key_offsets), n_queries, _dev(d_out),
                                          _dev(d_workspace), workspace_bytes, _stream(stream)),
           "impir_answer_add32_async")


def impir_tune_cache_save(path: str) -> None:
    _check(lib().impir_tune_cache_save(path.encode()), "impir_tune_cache_save")


def impir_tune_cache_load(path: str) -> int:
    n = ctypes.c_uint32()
    _check(lib().impir_tune_cache_load(path.encode(), ctypes.byref(n)), "impir_tune_cache_load")
    return n.value


def impir_workspace_bytes(n_queries: int, stride_bytes: int) -> int:
    return int(lib().impir_workspace_bytes(n_queries, stride_bytes))


def impir_answer_async(db: int, d_keys, d_key_offsets, n_queries: int, d_out, d_workspace, workspace_bytes: int,
                       stream=None) -> None:
    _check(lib().impir_answer_async(db, _dev(d_keys), _dev(d_key_offsets), n_queries, _dev(d_out),
                                    _dev(d_workspace), workspace_bytes, _stream(stream)), "impir_answer_async")


def impir_workspace_status(d_workspace) -> tuple[int, int]:
    nb, fb = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().impir_workspace_status(_dev(d_workspace), ctypes.byref(nb), ctypes.byref(fb)),
           "impir_workspace_status")
    return nb.value, fb.value


def impir_get_config(db: int, n_queries: int = 1) -> impir_config:
    c = impir_config()
    _check(lib().impir_get_config(db, n_queries, ctypes.byref(c)), "impir_get_config")
    return c


def impir_get_config_add32(db: int, n_queries: int = 1) -> impir_config:
    """The launch shape of the additive answer for a batch of n_queries on this database."""
    c = impir_config()
    _check(lib().impir_get_config_add32(db, n_queries, ctypes.byref(c)), "impir_get_config_add32")
    return c


def impir_set_config(db: int, lane_bits: int, queries_per_warp: int, warps_per_cta: int = 16,
                     queries_per_launch: int = 0) -> None:
    c = impir_config(lane_bits, queries_per_warp, warps_per_cta, queries_per_launch)
    _check(lib().impir_set_config(db, ctypes.byref(c)), "impir_set_config")


def impir_autotune(db: int, d_keys, d_key_offsets, n_queries: int, d_out, d_workspace, workspace_bytes: int,
                   stream=None) -> impir_config:
    c = impir_config()
    _check(lib().impir_autotune(db, _dev(d_keys), _dev(d_key_offsets), n_queries, _dev(d_out), _dev(d_workspace),
                                workspace_bytes, _stream(stream), ctypes.byref(c)), "impir_autotune")
    return c


def dpf_gen(alpha: int, m: int, prf: int, rng_seed: bytes) -> tuple[bytes, bytes]:
    assert len(rng_seed) == 32
    kb = impir_key_bytes(m)
    k0, k1 = np.zeros(kb, np.uint8), np.zeros(kb, np.uint8)
    _, sp = _host(rng_seed)
    _check(lib().dpf_gen(alpha, m, prf, sp, ctypes.c_void_p(k0.ctypes.data), ctypes.c_void_p(k1.ctypes.data)),
           "dpf_gen")
    return k0.tobytes(), k1.tobytes()


def impir_reconstruct(r0, r1) -> bytes:
    a, pa = _host(r0)
    _, pb = _host(r1)
    out = np.zeros(a.size, np.uint8)
    _check(lib().impir_reconstruct(pa, pb, a.size, ctypes.c_void_p(out.ctypes.data)), "impir_reconstruct")
    return out.tobytes()


def impir_last_error() -> str:
    return lib().impir_last_error().decode(errors="replace")


def impir_bounds_status() -> dict:
    """Failed index checks of the debug build since the last call (waits for the device)."""
    n, site, idx = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
    _check(lib().impir_bounds_status(ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx)), "impir_bounds_status")
    return {"n_failed": n.value, "first_site": site.value, "first_index": idx.value}


def impir_device_sm_count() -> int:
    return int(lib().impir_device_sm_count())


IMPIR_NOALLOC_SCRATCH_BYTES = 8 << 20
IMPIR_SHARD_ALIGN = 32768


def impir_server_create(max_batch: int, streams: int, max_record_bytes: int, accumulator_budget: int) -> int:
    cfg = impir_server_config(max_batch, streams, max_record_bytes, 0, accumulator_budget)
    h = ctypes.c_void_p()
    _check(lib().impir_server_create(ctypes.byref(cfg), ctypes.byref(h)), "impir_server_create")
    return h.value


def impir_server_submit(server: int, db: int, key: bytes, tag: int) -> None:
    _, kp = _host(key)
    _check(lib().impir_server_submit(ctypes.c_void_p(server), db, kp, tag), "impir_server_submit")


def impir_server_take(server: int, timeout_us: int, answer_capacity: int = 1 << 16):
    """Next finished request: dict(tag, db, answer, latency_ns, batch) or None on timeout."""
    tag, db, nb, lat, bs = ctypes.c_uint64(), ctypes.c_int32(), ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32()
    ver = ctypes.c_uint64()
    buf = np.zeros(answer_capacity, np.uint8)
    st = lib().impir_server_take(ctypes.c_void_p(server), timeout_us, ctypes.byref(tag), ctypes.byref(db),
                                 ctypes.c_void_p(buf.ctypes.data), answer_capacity, ctypes.byref(nb),
                                 ctypes.byref(lat), ctypes.byref(bs), ctypes.byref(ver))
    if st == IMPIR_ETIMEOUT:
        return None
    _check(st, "impir_server_take")
    return {"tag": tag.value, "db": db.value, "answer": buf[: nb.value].tobytes(), "latency_ns": lat.value,
            "batch": bs.value, "version": ver.value}


def impir_server_update(server: int, db: int, first_record: int, records: np.ndarray) -> None:
    """Queue a bulk update of len(records) records starting at first_record."""
    r = np.ascontiguousarray(records, dtype=np.uint8)
    n = r.shape[0] if r.ndim == 2 else 0
    _check(lib().impir_server_update(ctypes.c_void_p(server), db, first_record, n, ctypes.c_void_p(r.ctypes.data)),
           "impir_server_update")


def impir_db_update(db: int, first_record: int, records: np.ndarray) -> None:
    r = np.ascontiguousarray(records, dtype=np.uint8)
    _check(lib().impir_db_update(db, first_record, r.shape[0], ctypes.c_void_p(r.ctypes.data)), "impir_db_update")


def impir_db_version(db: int) -> int:
    v = ctypes.c_uint64()
    _check(lib().impir_db_version(db, ctypes.byref(v)), "impir_db_version")
    return v.value


def impir_server_stats(server: int) -> dict:
    b, q, mi, p = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().impir_server_stats(ctypes.c_void_p(server), ctypes.byref(b), ctypes.byref(q), ctypes.byref(mi),
                                    ctypes.byref(p)), "impir_server_stats")
    return {"batches": b.value, "queries": q.value, "max_inflight_batches": mi.value, "pending": p.value}


def impir_server_destroy(server: int) -> None:
    _check(lib().impir_server_destroy(ctypes.c_void_p(server)), "impir_server_destroy")


def impir_answer_noalloc(d_records, n_records: int, record_bytes: int, stride_bytes: int, d_keys, d_key_offsets,
                         n_queries: int, d_out, stream=None) -> None:
    """Answer without allocating: scratch lives in a fixed device array inside the library."""
    _check(lib().impir_answer_noalloc(_dev(d_records), n_records, record_bytes, stride_bytes, _dev(d_keys),
                                      _dev(d_key_offsets), n_queries, _dev(d_out), _stream(stream)),
           "impir_answer_noalloc")


def impir_aes_calibrate(prf: int, iters: int, seeds: np.ndarray, threads_per_cta: int = 512):
    """AES-only engine run: returns (final states (n, 16) uint8, device ms)."""
    sd = np.ascontiguousarray(seeds, dtype=np.uint8).reshape(-1, 16)
    out = np.zeros_like(sd)
    ms = ctypes.c_double()
    _check(lib().impir_aes_calibrate(prf, iters, sd.shape[0], threads_per_cta, ctypes.c_void_p(sd.ctypes.data),
                                     ctypes.c_void_p(out.ctypes.data), ctypes.byref(ms)), "impir_aes_calibrate")
    return out, ms.value


def impir_aes_calibrate_bitsliced(iters: int, seeds: np.ndarray, threads_per_cta: int = 256):
    """Bitsliced engine run (fixed-key PRF): seeds (16 n, 16) uint8, 16 per thread; returns
    (final states (16 n, 16) uint8, device ms)."""
    sd = np.ascontiguousarray(seeds, dtype=np.uint8).reshape(-1, 16)
    if sd.shape[0] % 16:
        raise ValueError("the bitsliced engine takes 16 seeds per thread")
    out = np.zeros_like(sd)
    ms = ctypes.c_double()
    _check(lib().impir_aes_calibrate_bitsliced(iters, sd.shape[0] // 16, threads_per_cta,
                                               ctypes.c_void_p(sd.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                                               ctypes.byref(ms)), "impir_aes_calibrate_bitsliced")
    return out, ms.value


def impir_timing_enable(enable: bool = True) -> None:
    _check(lib().impir_timing_enable(1 if enable else 0), "impir_timing_enable")


def impir_timing_read() -> tuple[float, int, int]:
    """(summed fused-kernel ms, fused launches, all library launches) since the last enable."""
    ms, nf, na = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().impir_timing_read(ctypes.byref(ms), ctypes.byref(nf), ctypes.byref(na)), "impir_timing_read")
    return ms.value, nf.value, na.value


# ---- small conveniences over the ABI (argument packing only) ----

def pack_keys(keys: list[bytes]) -> tuple[bytes, np.ndarray]:
    """Concatenates wire keys; returns (blob, uint32 byte offsets)."""
    offs = np.zeros(len(keys), np.uint32)
    o = 0
    for i, k in enumerate(keys):
        offs[i] = o
        o += len(k)
    return b"".join(keys), offs
