"""The N > 1 path of bench.py on CPU: two gloo ranks, no GPU.

One workload of N TXs is split by TX: each rank takes its own TX against every RX
on a replica of the same scene (weak scaling, no collective on the data path);
after the timed region the slowest rank's time and the units of all ranks are
reduced.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2402_13747_b300 import scenes
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.room_noisy(n_tx=1, n_rx=16)
        tx_all, txi = bench.rank_pairs(sc, rank, world)
        # per-rank figures as the timed loop would produce them
        t_total, cones, paths, vis = 1.0 + rank, 1000.0 * (rank + 1), 10.0 * (rank + 1), 5e4 * (rank + 1)
        res = bench.reduce_over_ranks(t_total, cones, paths, torch.device("cpu"), vis)
        dist.barrier()
        out[rank] = (res, tx_all.copy(), txi.copy(), sc.rx.copy())
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_and_split_the_tx_list():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res0, tx0, txi0, rx0 = out[0]
        res1, tx1, txi1, rx1 = out[1]
    # max over ranks for the time, sums for the units, identical on every rank
    assert res0 == res1 == (2.0, 3000.0, 30.0, 150000.0)
    # one workload: the same TX list and RXs on every rank, the scene's own TX first,
    # each rank one TX of it (fixed work per rank)
    np.testing.assert_array_equal(tx0, tx1)
    np.testing.assert_array_equal(rx0, rx1)
    assert tx0.shape == (2, 3) and not np.allclose(tx0[0], tx0[1])
    assert list(txi0) == [0] and list(txi1) == [1]


def test_traffic_gate_hashes_device_code_only():
    """The stored refine traffic is tied to a hash of the kernel's device code: the
    hash finds the end of that code, and a change to the host launcher after it leaves
    the hash unchanged."""
    h = bench.kernel_sources_sha256()
    assert len(h) == 64 and int(h, 16) >= 0
    path, end = bench.KERNEL_SOURCES[0]
    text = open(os.path.join(bench.ROOT, path), "rb").read()
    assert text.count(end) == 1
    assert b"__global__" not in text[text.index(end):]


def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference launched as two ranks: rank 0 alone times the oracle
    and prints the one JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
                        os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
