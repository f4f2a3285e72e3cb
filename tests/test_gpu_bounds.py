"""The debug build with index checks (the sanitizer plan for this pool, where
compute-sanitizer is closed): the same kernels compiled with IMPIR_BOUNDS compare every
shared-memory, database record, key, query, schedule and accumulator index with the extent of
its buffer before the access, skip a failing access and record it.

* The small parity cases (the XOR answer on every launch shape, wide records, every domain
  size, large batches; the additive answer on every lane-subtree size) run against the debug
  library and must pass with no failed check (checked after every test by the autouse fixture
  in conftest.py).
* A check is seen to fire: with the last records of the database withheld from the checked
  extent (the memory itself stays valid, so no access can leave it), the synchronous call
  reports the failure as an error and the asynchronous one records it (site 3, a database word
  at or past the withheld records) in the device record and in the workspace header."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bounds_lib():
    from paper_2509_06514_gb300 import build
    build.build()
    return build.build(bounds=True)


def _run(args, **env):
    e = dict(os.environ, IMPIR_BOUNDS="1", **env)
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=e, capture_output=True, text=True, timeout=1500)


def test_parity_cases_pass_every_index_check(bounds_lib):
    r = _run(["-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
              "tests/test_gpu_parity.py", "tests/test_gpu_additive.py"])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert " passed" in r.stdout and "error" not in r.stdout.splitlines()[-1]


CHILD = r'''
import numpy as np
import torch
import paper_2509_06514_gb300 as impir
from paper_2509_06514_gb300 import workloads

assert impir.BOUNDS and impir.LIB_PATH.endswith("libimpir_bounds.so")
N, B, W = 4096, 64, 4                   # W: 16-byte words per record
db = workloads.make_db(N, B, seed=3)
h = impir.impir_db_load(db, N, B)
k0, _ = impir.dpf_gen(7, 12, 0, bytes(range(32)))
try:
    impir.impir_answer(h, k0, 1, B)
    raise SystemExit("the synchronous call reported no failed check")
except impir.ImpirError as e:
    assert e.status == impir.IMPIR_ECUDA and "index checks failed" in str(e) and "site 3" in str(e), e
assert impir.impir_bounds_status()["n_failed"] == 0    # that call read and cleared the record
blob, offs = impir.pack_keys([k0])
d_keys = torch.from_numpy(np.frombuffer(blob, np.uint8).copy()).cuda()
d_off = torch.from_numpy(offs.view(np.int32).copy()).cuda()
d_out = torch.zeros((1, B), dtype=torch.uint8, device="cuda")
wsb = impir.impir_workspace_bytes(1, B)
d_ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
impir.impir_answer_async(h, d_keys, d_off, 1, d_out, d_ws, wsb, None)
st = impir.impir_bounds_status()
assert st["n_failed"] > 0 and st["first_site"] == 3 and st["first_index"] >= (N - 5) * W, st
# the workspace header's failure counter: the 32-bit word after the four 64/32-bit fields
# counter, n_units, n_bad, first_bad, n_groups, n_segs (byte offset 32)
hdr_failed = int(d_ws[32:36].cpu().numpy().view("<u4")[0])
assert hdr_failed == st["n_failed"], (hdr_failed, st)
impir.impir_db_free(h)
print("BOUNDS_FIRED_OK", st)
'''


def test_withheld_records_fire_the_record_check(bounds_lib):
    r = _run(["-c", CHILD], IMPIR_BOUNDS_TEST_WITHHOLD_RECORDS="5")
    assert r.returncode == 0 and "BOUNDS_FIRED_OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
