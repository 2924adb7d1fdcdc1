"""Write the oracle's exact paths for the noisy room, 1 TX x 16 RX, <= 3 reflections +
1 diffraction (the depth of the benchmark's workloads) to room_noisy_1x16.npz.

    python tests/golden/make_room_noisy_1x16.py

Calls only the FP64 oracle (about 15 minutes on one core: 86,633 coarse paths
refined); the inputs come from the seeded scene generator.  The GPU parity test
tests/test_gpu_depth.py compares the CUDA path's exact paths with this file.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2402_13747_b300 import config, scenes  # noqa: E402

OUT = os.path.join(HERE, "room_noisy_1x16.npz")
MAX_INT = 4


def workload():
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:16])
    return sc, config.params_for(sc)


def main():
    sc, p = workload()
    assert p.max_interactions == MAX_INT
    t0 = time.time()
    s = oracle.Scene.from_scene(sc, p)
    c = s.trace(sc.tx, sc.rx)
    e = s.refine(c)
    P = e.paths()
    np.savez_compressed(
        OUT, tx=P["tx"].astype(np.int16), rx=P["rx"].astype(np.int16), n=P["n"].astype(np.int8),
        type=P["type"][:, :MAX_INT].astype(np.int8), label=P["label"][:, :MAX_INT].astype(np.uint32),
        pts=P["pts"][:, :MAX_INT], length=P["length"], n_coarse=np.int64(c.stats["n_paths"]),
        n_coarse_raw=np.int64(c.stats["n_before_kappa"]))
    print(f"{len(P['n'])} exact paths from {c.stats['n_paths']} coarse paths in {time.time() - t0:.0f} s -> {OUT}")


if __name__ == "__main__":
    main()
