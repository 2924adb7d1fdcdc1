"""TX sharding of one workload (paper_2402_13747_b300.shard), on CPU.

The paper traces each TX separately and every later step is per TX/RX pair, so a
workload splits by TX.  These tests check the partition, and, with two gloo ranks
and a stand-in for the per-rank GPU run, that the exact paths gathered to rank 0
equal the single-process result and that no TX is traced twice.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2402_13747_b300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_tx", [0, 1, 2, 5, 16, 17])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_tx_shard_is_a_partition(n_tx, world):
    parts = [shard.tx_shard(n_tx, r, world) for r in range(world)]
    allidx = np.concatenate(parts)
    assert sorted(allidx.tolist()) == list(range(n_tx))
    sizes = [len(q) for q in parts]
    assert max(sizes) - min(sizes) <= 1
    for q in parts:   # contiguous blocks
        assert len(q) == 0 or list(q) == list(range(q[0], q[0] + len(q)))


def test_tx_shard_rejects_bad_ranks():
    with pytest.raises(ValueError):
        shard.tx_shard(4, 2, 2)
    with pytest.raises(ValueError):
        shard.tx_shard(4, 0, 0)


def fake_run_pairs(tx, rx, log=None):
    """A stand-in for trace + refine on one GPU: for TX t (numbered within `tx`) and
    RX j, a deterministic number of 'paths' whose fields depend on the TX's and the
    RX's coordinates only (so a TX's paths do not depend on its shard)."""
    out = {k: [] for k in shard.PATH_KEYS}
    for t in range(tx.shape[0]):
        if log is not None:
            log.append(tuple(np.round(tx[t], 9)))
        for j in range(rx.shape[0]):
            seed = int(abs(np.sum(tx[t] * 1e3 + rx[j] * 7e2))) % 5
            for q in range(seed):
                n = q % 3
                out["tx"].append(t)
                out["rx"].append(j)
                out["n"].append(n)
                out["type"].append(np.zeros(8, np.int32))
                out["label"].append(np.full(8, q, np.uint32))
                out["material"].append(np.zeros(8, np.uint8))
                out["ie"].append(np.arange(8) + q)
                out["pts"].append(np.tile(tx[t] + rx[j] * (q + 1), (8, 1)))
                out["length"].append(float(np.linalg.norm(tx[t] - rx[j]) + q))
                out["delay"].append(out["length"][-1] / 299792458.0)
                out["grad"].append(0.0)
                out["iters"].append(q)
                out["status"].append(0)
    return {k: np.array(v) for k, v in out.items()}


def _workload():
    rng = np.random.default_rng(5)
    return rng.uniform(0, 10, (5, 3)), rng.uniform(0, 10, (7, 3))


def _key_set(P):
    return sorted((int(P["tx"][i]), int(P["rx"][i]), int(P["n"][i]), round(float(P["length"][i]), 9),
                   tuple(np.round(P["pts"][i].ravel(), 9))) for i in range(len(P["n"])))


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tx, rx = _workload()
        log = []
        txi, paths = shard.run_sharded(lambda t, r: fake_run_pairs(t, r, log), tx, rx, rank, world)
        got = shard.gather_paths(txi, paths, rank, world)
        traced = [None] * world
        dist.all_gather_object(traced, log)
        out[rank] = (None if got is None else _key_set(got), traced)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_equals_one_process():
    world = 2
    tx, rx = _workload()
    single = _key_set(shard.gather_paths(np.arange(tx.shape[0]), fake_run_pairs(tx, rx), 0, 1))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        got0, traced = out[0]
        got1, _ = out[1]
    assert got1 is None
    assert got0 == single and len(single) > 0
    flat = [t for per_rank in traced for t in per_rank]
    assert len(flat) == tx.shape[0] == len(set(flat))   # every TX traced once, on one rank
