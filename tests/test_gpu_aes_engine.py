"""The AES engines on their own: chained node expansions p <- PRF_p(0) ^ PRF_p(1) (Eq. (3) with
zero codewords) agree with the oracle's FIPS-197 AES, for the fused kernel's T-table engine
(both PRFs) and for the bitsliced engine (fixed-key PRF), which also equals the T-table engine
on every seed."""
import numpy as np
import pytest

import paper_2509_06514_gb300 as impir

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prf", [0, 1])
def test_engine_matches_oracle(orc, prf):
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()
    rng = np.random.default_rng(prf)
    seeds = rng.integers(0, 256, (1000, 16), dtype=np.uint8)   # not a multiple of the CTA size
    out, ms = impir.impir_aes_calibrate(prf, 3, seeds, threads_per_cta=256)
    assert ms > 0
    for i in (0, 1, 255, 256, 511, 999):
        p = seeds[i].tobytes()
        for _ in range(3):
            p = bytes(a ^ b for a, b in zip(orc.prf(prf, p, 0), orc.prf(prf, p, 1)))
        assert out[i].tobytes() == p, i


def test_bitsliced_engine_matches_table_engine_and_oracle(orc):
    import torch
    assert torch.cuda.is_available()
    from paper_2509_06514_gb300 import build
    build.build()
    rng = np.random.default_rng(11)
    seeds = rng.integers(0, 256, (16 * 300, 16), dtype=np.uint8)   # 300 threads: a ragged last CTA
    out, ms = impir.impir_aes_calibrate_bitsliced(3, seeds, threads_per_cta=128)
    assert ms > 0
    ref, _ = impir.impir_aes_calibrate(impir.IMPIR_PRF_AES_MMO, 3, seeds, threads_per_cta=256)
    assert np.array_equal(out, ref)
    for i in (0, 1, 15, 16, 17, 2047, 16 * 300 - 1):
        p = seeds[i].tobytes()
        for _ in range(3):
            p = bytes(a ^ b for a, b in zip(orc.prf(1, p, 0), orc.prf(1, p, 1)))
        assert out[i].tobytes() == p, i
