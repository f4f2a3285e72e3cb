"""Failure paths on a GPU, all host-detected: an impossible device allocation, an undersized
workspace, invalid launch shapes, and malformed batches return a status; nothing faults."""
import ctypes

import numpy as np
import pytest

import paper_2509_06514_gb300 as impir
from paper_2509_06514_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()


def test_impossible_database_allocation_is_enomem(built):
    # 2^38 records of 16 bytes (4 TiB) cannot be allocated; the host buffer is never read
    tiny = np.zeros(16, np.uint8)
    h = ctypes.c_int32(0)
    st = impir.lib().impir_db_load(ctypes.c_void_p(tiny.ctypes.data), 1 << 38, 16, ctypes.byref(h))
    assert st == impir.IMPIR_ENOMEM
    assert "allocation" in impir.impir_last_error()


def test_undersized_workspace_and_bad_shapes(built):
    import torch
    N, B = 4096, 64
    db = workloads.make_db(N, B, seed=3)
    h = impir.impir_db_load(db, N, B)
    try:
        keys = [impir.dpf_gen(i, 12, 0, bytes([i]) * 32)[0] for i in range(3)]
        blob, offs = impir.pack_keys(keys)
        d_keys = torch.from_numpy(np.frombuffer(blob, np.uint8).copy()).cuda()
        d_off = torch.from_numpy(offs.view(np.int32).copy()).cuda()
        d_out = torch.zeros((3, B), dtype=torch.uint8, device="cuda")
        small = torch.empty(256, dtype=torch.uint8, device="cuda")
        with pytest.raises(impir.ImpirError) as e:
            impir.impir_answer_async(h, d_keys, d_off, 3, d_out, small, 256, None)
        assert e.value.status == impir.IMPIR_ENOMEM
        for bad in (dict(lane_bits=11, queries_per_warp=1), dict(lane_bits=3, queries_per_warp=3),
                    dict(lane_bits=9, queries_per_warp=16), dict(lane_bits=3, queries_per_warp=2, warps_per_cta=2),
                    dict(lane_bits=3, queries_per_warp=2, queries_per_launch=2),
                    dict(lane_bits=3, queries_per_warp=2, warps_per_cta=21),
                    dict(lane_bits=3, queries_per_warp=16, warps_per_cta=20)):
            with pytest.raises(impir.ImpirError) as e:
                impir.impir_set_config(h, **bad)
            assert e.value.status == impir.IMPIR_EINVAL
        # the database still answers after the rejected calls
        r = impir.impir_answer(h, blob, 3, B)
        k1 = [impir.dpf_gen(i, 12, 0, bytes([i]) * 32)[1] for i in range(3)]
        r1 = impir.impir_answer(h, b"".join(k1), 3, B)
        for i in range(3):
            assert np.array_equal(r[i] ^ r1[i], db[i])
        # a truncated batch (declared count larger than the keys present) is caught by the
        # header check of the first missing key
        with pytest.raises(impir.ImpirError):
            impir.impir_answer(h, blob + bytes(8), 4, B)
    finally:
        impir.impir_db_free(h)
    with pytest.raises(impir.ImpirError):
        impir.impir_db_free(h)       # double free: unknown handle
