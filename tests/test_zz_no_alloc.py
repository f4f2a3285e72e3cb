"""The allocation-free answer entry point (for callers that may not allocate device memory
when they answer) gives the same bits as the workspace-based asynchronous entry point, on
two calls in a row through the C ABI, and rejects a batch too large for its fixed scratch.
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


def test_noalloc_matches_async_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()
    N, B, stride = 70000, 40, 48
    db = workloads.make_db(N, B, seed=77)
    d_db = torch.zeros((N, stride), dtype=torch.uint8, device="cuda")
    d_db[:, :B] = torch.from_numpy(db).cuda()
    dbh = impir.impir_db_attach(d_db, N, B, stride)
    rng = np.random.default_rng(99)
    try:
        s = torch.cuda.Stream()
        for call, (n, ms) in enumerate(((13, [17, 16, 12]), (40, [17, 9, 14, 17]))):
            keys = []
            for i in range(n):
                m = ms[i % len(ms)]
                a = int(rng.integers(0, min(N, 1 << m)))
                keys.append(impir.dpf_gen(a, m, i % 2, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())[0])
            d_keys, d_off = _device_keys(torch, keys)
            want = torch.zeros((n, B), dtype=torch.uint8, device="cuda")
            wsb = impir.impir_workspace_bytes(n, stride)
            d_ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
            impir.impir_answer_async(dbh, d_keys, d_off, n, want, d_ws, wsb, s)
            got = torch.full((n, B), 0xA5, dtype=torch.uint8, device="cuda")
            impir.impir_answer_noalloc(d_db, N, B, stride, d_keys, d_off, n, got, s)
            s.synchronize()
            assert torch.equal(got, want), f"call {call}"
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
