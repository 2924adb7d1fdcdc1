"""The benchmark workload at full size, in the configuration bench.py times, checked
on sampled outputs the oracle computes one by one (needs a B300)."""
import numpy as np
import pytest

import oracle
from paper_2402_13747_b300 import config, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_run():
    from paper_2402_13747_b300 import _abi
    sc = scenes.room_noisy()                   # 4 TX x 16 RX, <= 3 reflections + 1 diffraction
    p = config.params_for(sc)
    ctx = _abi.Context(0)
    s = ctx.voxelize_scene(sc, p)
    c = ctx.trace(s, sc.tx, sc.rx, p)
    C = ctx.query_coarse(c)
    P = ctx.refine(s, c, p)
    A = ctx.query(P, 1)                        # one refined result per coarse path, same order
    F = ctx.query(P, 0)
    ctx.close()
    osc = oracle.Scene.from_scene(sc, p)
    return sc, p, C, A, F, osc


def test_full_size_counts_and_invariants(full_run):
    sc, p, C, A, F, osc = full_run
    assert C["counts"]["overflow"] == 0
    assert len(C["n"]) == len(A["n"]) > 100_000
    # kappa: at most kappa coarse paths per (TX, RX, type + label sequence)
    keys = {}
    for i in range(len(C["n"])):
        n = int(C["n"][i])
        k = (int(C["tx"][i]), int(C["rx"][i]), tuple(C["type"][i][:n]), tuple(C["label"][i][:n]))
        keys[k] = keys.get(k, 0) + 1
    assert max(keys.values()) <= p.kappa
    # exact paths: unique per label sequence, within the interaction limits
    seen = set()
    for i in range(len(F["n"])):
        n = int(F["n"][i])
        k = (int(F["tx"][i]), int(F["rx"][i]), tuple(F["type"][i][:n]), tuple(F["label"][i][:n]))
        assert k not in seen
        seen.add(k)
        assert sum(1 for t in F["type"][i][:n] if t == 0) <= 3 and sum(1 for t in F["type"][i][:n] if t == 1) <= 1
    assert len(F["n"]) > 1000


def test_sampled_refinement_matches_oracle(full_run):
    """200 sampled coarse paths of the full workload refined by the oracle one by one."""
    sc, p, C, A, F, osc = full_run
    rng = np.random.default_rng(21)
    idx = np.sort(rng.choice(len(C["n"]), size=200, replace=False))
    sub = {k: C[k][idx] for k in ("tx", "rx", "n", "ie", "type", "label")}
    R = osc.refine_given(sc.tx, sc.rx, sub)
    g_status = A["status"][idx]
    agree = g_status == R["status"]
    assert agree.mean() >= 0.95, (g_status, R["status"])
    both = (g_status == 0) & (R["status"] == 0)
    assert both.sum() >= 40
    for j in np.where(both)[0]:
        n = int(sub["n"][j])
        np.testing.assert_allclose(A["pts"][idx[j]][:n], R["pts"][j][:n], atol=1e-3)
        assert abs(A["length"][idx[j]] - R["length"][j]) <= 1e-6 * R["length"][j]


def test_sampled_coarse_segments_are_visible(full_run):
    """Each segment of a sampled coarse path passes the oracle's visibility test."""
    sc, p, C, A, F, osc = full_run
    ies = osc.ies()
    rng = np.random.default_rng(22)
    idx = rng.choice(len(C["n"]), size=150, replace=False)
    ok = total = 0
    for i in idx:
        n = int(C["n"][i])
        nodes = [(sc.tx[C["tx"][i]], 0, oracle.NONE_LABEL)]
        for q in range(n):
            ie = int(C["ie"][i][q])
            nodes.append((ies["rp"][ie], 2 if ies["kind"][ie] == 1 else 1, int(ies["label"][ie])))
        nodes.append((sc.rx[C["rx"][i]], 0, oracle.NONE_LABEL))
        for (a, ma, la), (b, mb, lb) in zip(nodes[:-1], nodes[1:]):
            total += 1
            ok += osc.visible(a, b, ma, la, mb, lb)
    assert ok >= 0.97 * total
