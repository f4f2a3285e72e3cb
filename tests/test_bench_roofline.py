"""The benchmark's roofline arithmetic, checked on the CPU against independent counts: the AES
blocks of a full-domain evaluation (one per tree edge), the table lookups the kernel's code
executes per domain (345 per internal node pair, 288 per leaf-level pair, counted here by
enumerating the tree's nodes), and the scaling of a small-case DRAM capture to a workload."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def tree_pairs(m):
    """(internal pairs, leaf-level pairs) of a depth-m GGM tree, by walking its nodes: every
    node above the leaves is expanded once into its two children."""
    internal = leaf = 0
    frontier = [0]
    for d in range(m):
        nxt = []
        for j in frontier:
            if d == m - 1:
                leaf += 1
            else:
                internal += 1
            nxt += [2 * j, 2 * j + 1]
        frontier = nxt
    return internal, leaf


@pytest.mark.parametrize("m", [1, 2, 3, 7, 12])
def test_blocks_and_lookups_match_an_enumerated_tree(m):
    internal, leaf = tree_pairs(m)
    assert bench.aes_blocks(m) == 2 * (internal + leaf)
    assert bench.lookups_per_query(m) == 345 * internal + 288 * leaf
    assert bench.lookups_per_query(m, bench.LOOKUPS_LEAF_PAIR_ADD) == 345 * internal + 321 * leaf


def test_lookups_per_block_and_port_peak():
    per = bench.lookups_per_query(25) / bench.aes_blocks(25)
    assert abs(per - 158.25) < 1e-3
    # 152 SMs x 2070 MHz x 32 lookups per clock / 158.25 lookups per block
    assert abs(bench.smem_peak_gaes(152, 2070.0, 158.25) - 63.6239) < 1e-3


def test_small_case_traffic_scales_per_batch(tmp_path, monkeypatch):
    # a capture of two batches on a 1 GiB prefix: 2x and 3x the prefix in DRAM bytes
    import json
    prof = tmp_path / "profiles"
    prof.mkdir()
    launch = {"lane_bits": 7, "queries_per_warp": 8, "warps_per_cta": 20, "queries_per_launch": 0}
    (prof / "fused_kernel_traffic.json").write_text(json.dumps({
        "kernel_source_sha256": bench.kernel_source_hash(), "launch": launch,
        "per_batch": [{"queries": 5, "dram_read_bytes": 2 << 30, "dram_write_bytes": 0, "db_prefix_bytes": 1 << 30},
                      {"queries": 9, "dram_read_bytes": 3 << 30, "dram_write_bytes": 0, "db_prefix_bytes": 1 << 30}]}))
    src_hash = bench.kernel_source_hash()      # of the repository's kernel sources
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: src_hash)
    batches = [{"n": 5, "prefix_bytes": 8 << 30}, {"n": 9, "prefix_bytes": 4 << 30}]
    got = bench.captured_traffic(launch, batches)
    assert got == (2 * (8 << 30) + 3 * (4 << 30)) / 2
    # another launch shape, or other batches: no figure
    assert bench.captured_traffic(dict(launch, lane_bits=6), batches) is None
    assert bench.captured_traffic(launch, batches[:1]) is None
