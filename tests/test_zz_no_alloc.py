"""The allocation-free answer entry point, for callers that may not allocate device memory
at the moment they answer (code inside an allocator or memory-pool callback, a process whose
device memory a framework reserved up front, a path that must not synchronize through
cudaMalloc/cudaFree). Through the C ABI it gives the same bits as the workspace-based
asynchronous entry point and as the CPU oracle, on two calls in a row and for records wide
enough to need column passes; after its first call on the device, later calls (even of new
launch shapes) take no device memory; and it rejects a batch too large for its fixed scratch.
This file is collected last on purpose."""
import numpy as np
import pytest

import paper_2509_06514_gb300 as impir
from paper_2509_06514_gb300 import workloads

pytestmark = pytest.mark.gpu


def _device_keys(torch, keys):
    blob, offs = impir.pack_keys(keys)
    return (torch.from_numpy(np.frombuffer(blob, np.uint8).copy()).cuda(),
            torch.from_numpy(offs.view(np.int32).copy()).cuda())


def _keys(rng, n, ms, n_records):
    keys = []
    for i in range(n):
        m = ms[i % len(ms)]
        a = int(rng.integers(0, min(n_records, 1 << m)))
        keys.append(impir.dpf_gen(a, m, i % 2, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())[0])
    return keys


def _device_db(torch, db, stride):
    n, b = db.shape
    d_db = torch.zeros((n, stride), dtype=torch.uint8, device="cuda")
    d_db[:, :b] = torch.from_numpy(db).cuda()
    return d_db


def test_noalloc_matches_async_and_oracle_twice(orc):
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()
    N, B, stride = 70000, 40, 48
    db = workloads.make_db(N, B, seed=77)
    d_db = _device_db(torch, db, stride)
    dbh = impir.impir_db_attach(d_db, N, B, stride)
    rng = np.random.default_rng(99)
    try:
        s = torch.cuda.Stream()
        for call, (n, ms) in enumerate(((13, [17, 16, 12]), (40, [17, 9, 14, 17]))):
            keys = _keys(rng, n, ms, N)
            d_keys, d_off = _device_keys(torch, keys)
            want = torch.zeros((n, B), dtype=torch.uint8, device="cuda")
            wsb = impir.impir_workspace_bytes(n, stride)
            d_ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
            impir.impir_answer_async(dbh, d_keys, d_off, n, want, d_ws, wsb, s)
            got = torch.full((n, B), 0xA5, dtype=torch.uint8, device="cuda")
            impir.impir_answer_noalloc(d_db, N, B, stride, d_keys, d_off, n, got, s)
            s.synchronize()
            assert torch.equal(got, want), f"call {call}"
            g = got.cpu().numpy()
            for i, k in enumerate(keys):
                assert g[i].tobytes() == orc.answer(k, db, N, B), (call, i)
    finally:
        impir.impir_db_free(dbh)


def test_noalloc_wide_records_take_no_device_memory(orc):
    """Records of 1040 and 4100 bytes (two and five column passes of the scan at the default
    launch shape), against the asynchronous path and the oracle; the device's free memory is
    the same before and after each call once the entry point has been called on the device."""
    import torch
    assert torch.cuda.is_available()
    rng = np.random.default_rng(5)
    s = torch.cuda.Stream()
    # the first call on this device (if no earlier test made it) does the one-time set-up
    warm_db = torch.zeros((64, 16), dtype=torch.uint8, device="cuda")
    wk, wo = _device_keys(torch, [impir.dpf_gen(3, 6, 0, bytes(32))[0]])
    wout = torch.zeros((1, 16), dtype=torch.uint8, device="cuda")
    impir.impir_answer_noalloc(warm_db, 64, 16, 16, wk, wo, 1, wout, s)
    s.synchronize()
    for B, N, n in ((1040, 5000, 24), (4100, 3000, 9)):
        stride = (B + 15) // 16 * 16
        db = workloads.make_db(N, B, seed=B)
        d_db = _device_db(torch, db, stride)
        dbh = impir.impir_db_attach(d_db, N, B, stride)
        try:
            keys = _keys(rng, n, [12, 11, 7], N)
            d_keys, d_off = _device_keys(torch, keys)
            want = torch.zeros((n, B), dtype=torch.uint8, device="cuda")
            wsb = impir.impir_workspace_bytes(n, stride)
            d_ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
            impir.impir_answer_async(dbh, d_keys, d_off, n, want, d_ws, wsb, s)
            got = torch.full((n, B), 0x5A, dtype=torch.uint8, device="cuda")
            s.synchronize()
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            impir.impir_answer_noalloc(d_db, N, B, stride, d_keys, d_off, n, got, s)
            s.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            assert free1 == free0, (B, free0, free1)
            assert torch.equal(got, want), B
            g = got.cpu().numpy()
            for i, k in enumerate(keys):
                assert g[i].tobytes() == orc.answer(k, db, N, B), (B, i)
        finally:
            impir.impir_db_free(dbh)


def test_noalloc_rejects_batch_beyond_scratch():
    import torch
    d_db = torch.zeros((64, 4096), dtype=torch.uint8, device="cuda")
    n = impir.IMPIR_NOALLOC_SCRATCH_BYTES // 4096 + 1
    keys = [impir.dpf_gen(0, 6, 0, bytes(32))[0]] * n
    d_keys, d_off = _device_keys(torch, keys)
    out = torch.zeros((n, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(impir.ImpirError) as e:
        impir.impir_answer_noalloc(d_db, 64, 4096, 4096, d_keys, d_off, n, out, None)
    assert e.value.status == impir.IMPIR_EINVAL
    assert "scratch" in impir.impir_last_error()
