"""Host side of the multi-device partition of one system (one process per
device, torch.distributed).

SINR: every (UE, subcarrier) unit is independent (eq. 2, 9; the precoders
of eq. 7 are per subcarrier), so a system's K subcarriers are split into
contiguous ranges, one per rank, with G, C and the coefficients replicated;
each rank evaluates its range with ts_sinr_svd_range / ts_sinr_mmse_range
and no data crosses devices on the way.  `gather_sinr` assembles the whole
result where it is wanted (not part of the evaluation).

Fit: the block updates of Algorithm 2 (eq. 20-22) take the leading
eigenvectors of mode Grams summed over channels -- over the UEs k of a
transmit factor B_k, over the BSs of a receive factor A_i -- so with the
channels sharded across ranks each rank sums its own channels' Grams and
one all-reduce per block update completes the sums (`allreduce_grams`)."""
from __future__ import annotations


def subcarrier_ranges(K: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [k0, k1) ranges of K subcarriers over `world` ranks, sizes
    differing by at most one (the first K % world ranks get one more)."""
    if K < 1 or world < 1:
        raise ValueError("K and world must be positive")
    base, extra = divmod(K, world)
    out, k0 = [], 0
    for r in range(world):
        k1 = k0 + base + (1 if r < extra else 0)
        out.append((k0, k1))
        k0 = k1
    return out


def channel_shard(J: int, rank: int, world: int) -> list[tuple[int, int]]:
    """The links (i, k) of a J-cell system held by `rank`: round robin over
    the J^2 links, so that every rank holds links of every UE and BS."""
    return [(ch // J, ch % J) for ch in range(J * J) if ch % world == rank]


def gather_sinr(local, K: int, group=None):
    """All ranks' SINR ranges (J, count_r, L) -> the whole (J, K, L) on every
    rank (torch.distributed all_gather on the ranges, padded to the longest)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    ranges = subcarrier_ranges(K, world)
    longest = max(k1 - k0 for k0, k1 in ranges)
    J, cnt, L = local.shape
    pad = torch.zeros(J, longest, L, dtype=local.dtype, device=local.device)
    pad[:, :cnt] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:, :k1 - k0] for p, (k0, k1) in zip(parts, ranges)], dim=1)


def allreduce_grams(grams, group=None):
    """Sum each rank's partial mode Grams (a tensor, or a list of tensors)
    over the ranks, in place (one all-reduce per tensor)."""
    import torch.distributed as dist
    items = grams if isinstance(grams, (list, tuple)) else [grams]
    for g in items:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return grams
