"""The C-ABI library loads without a GPU, exports every symbol include/impir.h declares,
and its host-side pieces (key sizes, client key generation, reconstruction, argument
checks) behave; no compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2509_06514_gb300 as impir

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2509_06514_gb300 import build
    build.build()
    return impir.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "impir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)
    return sorted({n for n in names if n.startswith(("impir_", "dpf_"))})


def test_header_declarations_are_exported(L):
    decl = declared_functions()
    assert "impir_answer" in decl and "dpf_gen" in decl and "impir_db_load" in decl
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(impir.EXPORTS) == decl


def test_key_bytes(L):
    for m in (1, 16, 20, 22, 25, 40):
        assert impir.impir_key_bytes(m) == 8 + 64 * (m + 1)


@pytest.mark.parametrize("prf", [0, 1])
def test_dpf_gen_matches_oracle_gen_bytes(L, orc, prf):
    """Both key generators follow the same published construction and draw order."""
    rng = np.random.default_rng(prf)
    for m in (1, 2, 5, 13, 20, 25, 40):
        for _ in range(3):
            a = int(rng.integers(0, 1 << min(m, 62)))
            seed = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
            assert impir.dpf_gen(a, m, prf, seed) == orc.gen(a, m, prf, seed)


@pytest.mark.parametrize("prf", [0, 1])
def test_dpf_gen_keys_evaluate_to_point_function(L, orc, prf):
    one = np.zeros(16, np.uint8)
    one[0] = 1
    for m, a in ((1, 1), (4, 9), (8, 200), (11, 2047)):
        k0, k1 = impir.dpf_gen(a, m, prf, bytes(range(32)))
        x = orc.eval_all(k0) ^ orc.eval_all(k1)
        want = np.zeros_like(x)
        want[a] = one
        assert np.array_equal(x, want)


def test_dpf_gen_rejects_bad_arguments(L):
    with pytest.raises(impir.ImpirError) as e:
        impir.dpf_gen(16, 4, 0, bytes(32))
    assert e.value.status == impir.IMPIR_EINVAL
    with pytest.raises(impir.ImpirError):
        impir.dpf_gen(0, 41, 0, bytes(32))
    with pytest.raises(impir.ImpirError):
        impir.dpf_gen(0, 3, 7, bytes(32))


def test_reconstruct(L):
    a = bytes(range(40))
    b = bytes((7 * i) & 0xFF for i in range(40))
    assert impir.impir_reconstruct(a, b) == bytes(x ^ y for x, y in zip(a, b))


def test_unknown_handle_is_rejected(L):
    with pytest.raises(impir.ImpirError) as e:
        impir.impir_db_free(12345)
    assert e.value.status == impir.IMPIR_EINVAL
    with pytest.raises(impir.ImpirError):
        impir.impir_db_info(-1)


def test_workspace_bytes_grows_with_batch(L):
    a = impir.impir_workspace_bytes(1, 256)
    b = impir.impir_workspace_bytes(1024, 256)
    assert a % 256 == 0 and b % 256 == 0
    assert b - a >= 1023 * 256


def test_tune_cache_round_trip(L, tmp_path):
    src = tmp_path / "tune.txt"
    src.write_text("# comment\n152 33554432 256 416 8 4 16 0\n152 1048576 256 64 5 8 16 0\n"
                   "152 1048576 256 65 11 8 16 0\nnot a line\n")
    assert impir.impir_tune_cache_load(str(src)) == 2          # lane_bits 11 is rejected
    out = tmp_path / "out.txt"
    impir.impir_tune_cache_save(str(out))
    lines = [ln for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert "152 33554432 256 416 8 4 16 0" in lines and "152 1048576 256 64 5 8 16 0" in lines
    with pytest.raises(impir.ImpirError):
        impir.impir_tune_cache_load(str(tmp_path / "missing.txt"))


def test_oversized_inputs_are_rejected_before_any_device_call(L):
    """Record counts times strides (and batch sizes times strides) that would exceed 1 PiB are
    rejected with EINVAL before any allocation, copy or launch, so no size product can wrap."""
    buf = np.zeros(64, np.uint8)
    p = ctypes.c_void_p(buf.ctypes.data)
    aligned = ctypes.c_void_p(256)     # never dereferenced: the call fails first
    h = ctypes.c_int32(0)
    calls = [
        lambda: L.impir_db_load(p, 1 << 40, 0xFFFFFF00, ctypes.byref(h)),
        lambda: L.impir_db_load(p, 1 << 30, 0xFFFFFFFF, ctypes.byref(h)),
        lambda: L.impir_db_attach(aligned, 1 << 40, 1 << 20, 1 << 20, ctypes.byref(h)),
        lambda: L.impir_db_load_rows(p, 1, 0xFFFFFF00, 0, 1 << 40, ctypes.byref(h)),
        lambda: L.impir_answer_streamed(p, 1 << 40, 1 << 20, p, 1, p, 0, None),
        lambda: L.impir_answer_streamed(p, 16, 0xFFFFFFF8, p, 1, p, 0, None),
        lambda: L.impir_answer_noalloc(aligned, 1 << 40, 1 << 20, 1 << 20, p, p, 1, p, None),
    ]
    for i, call in enumerate(calls):
        assert call() == impir.IMPIR_EINVAL, i
        assert b"too large" in L.impir_last_error(), (i, L.impir_last_error())
