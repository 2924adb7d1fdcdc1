"""TX-sharded runs of one workload over several processes (one GPU each).

The paper launches rays for each TX separately (Section 2.2), and every later step
is per TX: the propagation tree grows from one TX, the kappa limit and both
duplicate removals (Section 2.3) act within one TX/RX pair.  So a workload with
several TXs splits by TX with no exchange on the data path: rank r traces and
refines its own TXs against every RX on a full replica of the scene, and the exact
path lists are gathered to rank 0 afterwards (a host gather of variable-size
lists).  The union of the ranks' lists equals the list one process computes for
all TXs, with TX indices mapped back to the workload's numbering.
"""
from __future__ import annotations

import numpy as np

__all__ = ["tx_shard", "merge_shards", "gather_paths", "run_sharded"]

PATH_KEYS = ("tx", "rx", "n", "type", "label", "material", "ie", "pts", "length", "delay", "grad", "iters",
             "status")


def tx_shard(n_tx: int, rank: int, world: int) -> np.ndarray:
    """Indices of the TXs rank `rank` of `world` traces: a contiguous block, sizes
    differing by at most one, every TX in exactly one block (empty when world >
    n_tx for the ranks past the end)."""
    if world < 1 or not 0 <= rank < world or n_tx < 0:
        raise ValueError("tx_shard: need 0 <= rank < world and n_tx >= 0")
    base, extra = divmod(n_tx, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return np.arange(lo, hi, dtype=np.int64)


def merge_shards(parts: list[tuple[np.ndarray, dict]]) -> dict:
    """One path dict from (tx indices of the shard, the shard's path dict) pairs.

    A shard's paths number their TXs 0..len(shard)-1; they are mapped back to the
    workload's indices and the lists concatenated in rank order."""
    out = {}
    for k in PATH_KEYS:
        arrs = []
        for txi, P in parts:
            if k not in P:
                continue
            a = np.asarray(P[k])
            if k == "tx":
                a = np.asarray(txi, dtype=np.int64)[a.astype(np.int64)] if len(a) else a.astype(np.int64)
            arrs.append(a)
        if arrs:
            out[k] = np.concatenate(arrs)
    return out


def gather_paths(txi: np.ndarray, paths: dict, rank: int, world: int):
    """Gather every rank's (tx indices, exact paths) to rank 0 over the default
    process group (torch.distributed, any backend); rank 0 gets the merged dict,
    the others None.  With world == 1 no process group is needed."""
    mine = (np.asarray(txi), {k: np.asarray(paths[k]) for k in PATH_KEYS if k in paths})
    if world == 1:
        return merge_shards([mine])
    import torch.distributed as dist
    got = [None] * world if rank == 0 else None
    dist.gather_object(mine, got, dst=0)
    return merge_shards(got) if rank == 0 else None


def run_sharded(run_pairs, tx: np.ndarray, rx: np.ndarray, rank: int, world: int):
    """Run one workload's TX shard: run_pairs(tx_subset, rx) -> exact path dict for
    those TXs (numbered within the subset).  Returns (tx indices, paths)."""
    txi = tx_shard(int(np.asarray(tx).shape[0]), rank, world)
    if len(txi) == 0:
        return txi, {k: np.zeros(0) for k in PATH_KEYS}
    return txi, run_pairs(np.asarray(tx)[txi], rx)
