"""Packet-id sharding across ranks.

Packets are independent (each draws its own Philox stream keyed by packet
id), so N ranks run disjoint id ranges of the same workload and their tallies
add up to the single-rank result.  Rank r of `world` takes ids
[r * n, (r + 1) * n) at every wavelength, and every rank normalises packet
weights by the total count world * n.  No collective is needed on the data
path; summing the tallies (if wanted) is one reduction at the end.
"""


def shard(rank: int, world: int, n_per_rank: int):
    """(first packet id, packets per wavelength, weight normalisation) for `rank`."""
    if not (0 <= rank < world) or n_per_rank < 0:
        raise ValueError("bad rank, world size or packet count")
    return rank * n_per_rank, n_per_rank, world * n_per_rank
