"""Whole-set parity at the benchmark's depth: the noisy room, 1 TX x 16 RX, <= 3
reflections + 1 diffraction -- the depth of the benchmark's workloads -- traced and
refined on the CUDA path and compared element by element with the oracle's exact
paths, stored by tests/golden/make_room_noisy_1x16.py (the oracle needs about 15
minutes for it).  The GPU test needs a B300; the checks of the stored file run on
the CPU."""
import math
import os

import numpy as np
import pytest

from tests.golden.make_room_noisy_1x16 import MAX_INT, OUT, workload
from tests.pathsets import compare, confirm_alternates, oracle_confirms

# On the noisy cloud the gradient descent of one coarse path can settle on one of
# several stationary points a few centimetres to decimetres apart, or cycle around
# one until rho (Section 2.3 fixes neither the start nor the step).  Which candidate
# of a label sequence wins the shortest-path dedup can then depend on rounding: in
# the oracle, 64 of the 100 coarse paths of one (ceiling, wall, wall) sequence of
# this workload cycle between two points 1.8 cm apart that straddle a stationary
# point the CUDA path converges to from another candidate.  Such an alternate winner
# is accepted when the oracle confirms it is an exact path (on its surfaces,
# stationary, visible) and its length is within 1e-4 relative, for at most one path
# in 500 of the set.
ALT_PER = 500


def _golden():
    g = np.load(OUT)
    m = len(g["n"])
    pad = lambda a, fill: np.concatenate([a, np.full((m, 8 - MAX_INT) + a.shape[2:], fill, a.dtype)], 1)  # noqa: E731
    return dict(tx=g["tx"].astype(np.int32), rx=g["rx"].astype(np.int32), n=g["n"].astype(np.int32),
                type=pad(g["type"].astype(np.int32), 0), label=pad(g["label"], 0xFFFFFFFF),
                pts=pad(g["pts"], 0.0), length=g["length"]), int(g["n_coarse"])


def test_stored_oracle_paths_are_consistent():
    """The stored file against closed forms: every LOS path has length |TX - RX|, no
    path is shorter than its pair's straight line, every path's length is the sum of
    its segments through its stored points, and the depth limits hold."""
    ref, n_coarse = _golden()
    sc, p = workload()
    assert len(ref["n"]) > 2000 and n_coarse > 80_000
    for i in range(len(ref["n"])):
        n = ref["n"][i]
        tx, rx = sc.tx[ref["tx"][i]], sc.rx[ref["rx"][i]]
        nodes = [tx] + list(ref["pts"][i][:n]) + [rx]
        L = sum(float(np.linalg.norm(b - a)) for a, b in zip(nodes[:-1], nodes[1:]))
        assert L == pytest.approx(ref["length"][i], rel=1e-12)
        assert ref["length"][i] >= np.linalg.norm(rx - tx) * (1 - 1e-12)
        t = ref["type"][i][:n]
        assert (t == 0).sum() <= p.max_refl and (t == 1).sum() <= p.max_diff and n <= p.max_interactions
    los = ref["n"] == 0
    assert los.any()
    for i in np.where(los)[0]:
        assert ref["length"][i] == pytest.approx(math.dist(sc.tx[ref["tx"][i]], sc.rx[ref["rx"][i]]), rel=1e-12)


def test_exact_path_check_on_the_stored_paths():
    """The exact-path check that admits alternate winners, on the oracle's own stored
    reflection paths (the file keeps no entity indices, which the check needs for an
    edge): each passes; a reflection point moved 1 cm along its surface fails the
    stationarity bound, one lifted 1 mm off it fails the surface bound."""
    import oracle
    ref, _ = _golden()
    sc, p = workload()
    osc = oracle.Scene.from_scene(sc, p)
    rng = np.random.default_rng(7)
    refl_only = (ref["n"] >= 1) & ~((ref["type"] == 1) & (np.arange(8)[None, :] < ref["n"][:, None])).any(1)
    picks = rng.choice(np.nonzero(refl_only)[0], size=40, replace=False)
    moved = lifted = 0
    for i in picks:
        f_max, grad, vis = oracle_confirms(osc, sc, ref, i, p)
        assert f_max < 1e-4 and grad < p.delta and vis, (i, f_max, grad, vis)
        refl = [k for k in range(int(ref["n"][i])) if ref["type"][i][k] == 0]
        if not refl:
            continue
        k = refl[0]
        x = ref["pts"][i][k]
        _, nn = osc.sdf_label(int(ref["label"][i][k]), x)
        t = np.cross(nn, [1.0, 0.0, 0.0] if abs(nn[0]) < 0.9 else [0.0, 1.0, 0.0])
        t /= np.linalg.norm(t)
        for shift, which in ((0.01 * t, "moved"), (1e-3 * nn, "lifted")):
            Q = {kk: np.array(v[i:i + 1]) for kk, v in ref.items()}
            Q["pts"] = Q["pts"].copy()
            Q["pts"][0][k] = x + shift
            f2, g2, _ = oracle_confirms(osc, sc, Q, 0, p)
            if which == "moved":
                assert g2 > p.delta, (i, g2)
                moved += 1
            else:
                assert f2 > 5e-4, (i, f2)
                lifted += 1
    assert moved >= 20 and lifted >= 20


@pytest.mark.gpu
def test_noisy_room_1x16_full_depth_matches_oracle():
    """The CUDA path's exact paths equal the oracle's: the same (TX, RX, type sequence,
    label sequence) set, every point within 1e-3 m and every length within 1e-6
    relative, up to the oracle-confirmed alternate winners above.  The coarse sets may differ by a few paths whose FP32 cone or
    visibility decisions sit at a margin (2 of 86,633 when this was written); none
    of them reaches the exact set."""
    from paper_2402_13747_b300 import _abi
    ref, n_coarse = _golden()
    sc, p = workload()
    ctx = _abi.Context(0)
    s = ctx.voxelize_scene(sc, p)
    c = ctx.trace(s, sc.tx, sc.rx, p)
    C = ctx.coarse_counts(c)
    P = ctx.refine(s, c, p)
    G = ctx.query(P, 0)
    ctx.close()
    assert abs(C["n_coarse"] - n_coarse) <= 1e-3 * n_coarse, (C["n_coarse"], n_coarse)
    cmp = compare(G, ref, atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [], cmp
    assert cmp["n_common"] == len(ref["n"])
    confirm_alternates(G, cmp["bad"], sc, p, len(ref["n"]) // ALT_PER)
