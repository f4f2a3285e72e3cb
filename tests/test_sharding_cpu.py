"""Row sharding on CPU: the shard split covers the database in aligned blocks, and two gloo
ranks that each answer over their own block (here with the oracle, rows outside the block
zeroed) and exchange their partial answers through the package's all-gather reconstruct the
full answer, for the XOR and the additive answers."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2509_06514_gb300 import IMPIR_SHARD_ALIGN  # noqa: E402
from paper_2509_06514_gb300.sharding import shard_rows  # noqa: E402


@pytest.mark.parametrize("n_total", [1, 5, IMPIR_SHARD_ALIGN - 1, IMPIR_SHARD_ALIGN, IMPIR_SHARD_ALIGN + 1,
                                     70000, 1 << 25, 3 * IMPIR_SHARD_ALIGN + 17])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shard_rows_cover_the_database_in_aligned_blocks(n_total, world):
    blocks = shard_rows(n_total, world)
    assert len(blocks) == world
    pos = 0
    for lo, n in blocks:
        assert lo == pos and n >= 0
        assert lo % IMPIR_SHARD_ALIGN == 0 or n == 0
        end = lo + n
        assert end == n_total or end % IMPIR_SHARD_ALIGN == 0
        pos = end
    assert pos == n_total
    sizes = [n for _, n in blocks if n]
    units = -(-n_total // IMPIR_SHARD_ALIGN)
    assert len(sizes) == min(world, units)
    if len(sizes) > 1:      # balanced to within one aligned block (plus the ragged end)
        assert max(sizes) - min(sizes) <= 2 * IMPIR_SHARD_ALIGN


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("world", [2, 3, 5])
def test_weighted_shard_rows_balance_the_work(seed, world):
    from paper_2509_06514_gb300.sharding import domain_weights
    rng = np.random.default_rng(seed)
    n_total = int(rng.integers(1, 40)) * IMPIR_SHARD_ALIGN + int(rng.integers(0, IMPIR_SHARD_ALIGN))
    units = -(-n_total // IMPIR_SHARD_ALIGN)
    weights = rng.integers(0, 10, units).tolist() if seed % 2 else \
        domain_weights(n_total, rng.integers(15, 27, 50).tolist())
    blocks = shard_rows(n_total, world, weights=weights)
    pos, work = 0, []
    for lo, n in blocks:
        assert lo == pos and (lo % IMPIR_SHARD_ALIGN == 0 or n == 0)
        assert lo + n == n_total or (lo + n) % IMPIR_SHARD_ALIGN == 0
        work.append(sum(weights[lo // IMPIR_SHARD_ALIGN:-(-(lo + n) // IMPIR_SHARD_ALIGN)]) if n else 0)
        pos = lo + n
    assert pos == n_total
    # every shard's work is at most its share plus one block's
    assert max(work) <= sum(weights) / world + max(weights) + 1e-9
    with pytest.raises(ValueError):
        shard_rows(n_total, world, weights=weights[:-1] if len(weights) > 1 else [-1])


def test_domain_weights_count_covering_queries():
    from paper_2509_06514_gb300.sharding import domain_weights
    a = IMPIR_SHARD_ALIGN
    assert domain_weights(4 * a, [15, 16, 17, 40]) == [4, 3, 2, 2]   # 2^15 = a, 2^16 = 2a, 2^17 = 4a


def test_shard_rows_rejects_empty():
    with pytest.raises(ValueError):
        shard_rows(0, 2)
    with pytest.raises(ValueError):
        shard_rows(10, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


N, B = 70000, 16
MS = [17, 16, 15, 12]


def _keys():
    import oracle
    rng = np.random.default_rng(8080)
    return [oracle.gen(int(rng.integers(0, min(N, 1 << m))), m, i % 2, rng.integers(0, 256, 32, dtype=np.uint8).tobytes())
            for i, m in enumerate(MS)]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2509_06514_gb300 import workloads
    from paper_2509_06514_gb300.sharding import exchange, shard_rows
    dist.init_process_group("gloo", rank=rank, world_size=world)
    db = workloads.make_db(N, B, seed=77)
    lo, n = shard_rows(N, world)[rank]
    mine = np.zeros_like(db)
    mine[lo:lo + n] = db[lo:lo + n]           # this rank's block; other rows contribute nothing
    pairs = _keys()
    xor_part = np.stack([np.frombuffer(oracle.answer(p[0], mine, N, B), np.uint8) for p in pairs])
    add_part = np.stack([np.frombuffer(oracle.answer_add32(p[0], mine, N, B), np.uint8) for p in pairs])
    gx = exchange(torch.from_numpy(xor_part)).numpy()
    ga = exchange(torch.from_numpy(add_part)).numpy()
    dist.destroy_process_group()
    q.put((rank, (lo, n), gx, ga))


def test_two_gloo_ranks_exchange_partial_answers():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = sorted((q.get(timeout=10) for _ in range(2)), key=lambda g: g[0])
    assert got[0][1] == (0, IMPIR_SHARD_ALIGN) and got[1][1] == (IMPIR_SHARD_ALIGN, N - IMPIR_SHARD_ALIGN)
    from paper_2509_06514_gb300 import workloads
    db = workloads.make_db(N, B, seed=77)
    pairs = _keys()
    for rank, _, gx, ga in got:
        assert gx.shape == (2, len(MS), B)
        xor = gx[0] ^ gx[1]
        add = ((ga[0].view("<u4").astype(np.uint64) + ga[1].view("<u4").astype(np.uint64)) % (1 << 32)).astype("<u4")
        for i, p in enumerate(pairs):
            assert xor[i].tobytes() == oracle.answer(p[0], db, N, B), (rank, i)
            assert add[i].view(np.uint8).tobytes() == oracle.answer_add32(p[0], db, N, B), (rank, i)
        # m = 15 and 12 lie inside the first block: rank 1's partial answer is zero there
        assert not gx[1][2].any() and not gx[1][3].any()
