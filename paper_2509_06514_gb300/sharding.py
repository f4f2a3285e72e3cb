"""Row sharding of one database across ranks (one GPU each), the 1-D block layout of §3.3.

Each rank holds a block of rows (``impir_db_load_rows``) and answers every query over its rows
only; the ranks then exchange their partial answers (one all-gather, the only collective of
the path) and combine them on the device (``impir_combine_partials``): XOR for the XOR answer,
sum mod 2^32 for the additive one, as Algorithm 1 aggregates its partial results.
"""
from __future__ import annotations

from . import IMPIR_SHARD_ALIGN, impir_combine_partials


def shard_rows(n_total: int, world: int, align: int = IMPIR_SHARD_ALIGN, weights=None) -> list[tuple[int, int]]:
    """Split records [0, n_total) into `world` blocks (row_lo, n_rows) whose bounds are
    multiples of `align` (the last ends at n_total). Without `weights` the blocks hold as even a
    number of rows as that allows; with `weights` (one non-negative work estimate per aligned
    block of `align` rows, e.g. ``domain_weights``) they hold as even a share of the work. Ranks
    beyond the number of aligned blocks get an empty block (n_rows == 0) and hold no rows."""
    if n_total <= 0 or world <= 0:
        raise ValueError("need n_total > 0 and world > 0")
    units = -(-n_total // align)                     # aligned blocks of `align` rows (last partial)
    if weights is None:
        cuts = [units * r // world for r in range(world + 1)]
    else:
        w = [float(x) for x in weights]
        if len(w) != units or min(w) < 0:
            raise ValueError(f"need {units} non-negative block weights")
        total, acc, cuts, r = sum(w), 0.0, [0], 1
        for u, x in enumerate(w):                    # cut after the block where the running work
            acc += x                                  # first reaches r / world of the total
            while r < world and acc >= total * r / world:
                cuts.append(u + 1)
                r += 1
        cuts += [units] * (world + 1 - len(cuts))
    out = []
    for r in range(world):
        lo, hi = min(cuts[r] * align, n_total), min(cuts[r + 1] * align, n_total)
        out.append((lo, hi - lo))
    return out


def domain_weights(n_total: int, ms, align: int = IMPIR_SHARD_ALIGN) -> list[int]:
    """Work per aligned block of rows for queries of domain bits `ms`: a query with domain 2^m
    covers records [0, min(2^m, n_total)), so block b counts the queries whose domain reaches it
    (each covered record costs the same scan and, per leaf, the same tree work)."""
    units = -(-n_total // align)
    return [sum(1 for m in ms if (1 << m) > b * align) for b in range(units)]


def exchange(partial, group=None):
    """All-gather every rank's partial answers (a tensor of the same shape on every rank) into
    one tensor of shape (world, *partial.shape), on the device the tensors live on."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(partial) for _ in range(world)]
    dist.all_gather(parts, partial.contiguous(), group=group)
    return torch.stack(parts)


def combine(parts, mode: int = 0, stream=None):
    """Combine gathered partial answers (world, n_queries, record_bytes) uint8 on the GPU:
    XOR (mode 0) or sum mod 2^32 (mode 1). Returns (n_queries, record_bytes)."""
    import torch
    parts = parts.contiguous()
    out = torch.empty(parts.shape[1:], dtype=torch.uint8, device=parts.device)
    impir_combine_partials(mode, parts, parts.shape[0], parts[0].numel(), out, stream)
    return out
