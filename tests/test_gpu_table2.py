"""The shape of the paper's Table 2 runs (Section 3): one TX and one RX, at most five
interactions, without (Sim A) and with (Sim B) one diffraction, on the noisy room.
Five-interaction trees are far beyond what the oracle traces in a test, so the runs
are checked on sampled outputs the oracle computes one by one (needs a B300)."""
import json

import pytest

import oracle
from paper_2402_13747_b300 import config, scenes
from tests.sampled import coarse_invariants, exact_invariants, sampled_refinement, sampled_visibility

pytestmark = pytest.mark.gpu


def _run(ctx, s, sc, p):
    """Trace with bounds sized by a first overflowing trace when needed, then refine."""
    c = ctx.trace(s, sc.tx, sc.rx, p, allow_overflow=True)
    cc = ctx.coarse_counts(c)
    if cc["overflow"]:
        ctx.release(c)
        c = ctx.trace(s, sc.tx, sc.rx, p, max_nodes=max(1 << 23, int(1.2 * cc["needed_nodes"])),
                      max_coarse=max(1 << 23, int(1.2 * cc["needed_coarse"])))
    C = ctx.query_coarse(c)
    P = ctx.refine(s, c, p)
    A = ctx.query(P, 1)
    F = ctx.query(P, 0)
    pc = ctx.counts(P)
    ctx.release(P)
    ctx.release(c)
    return C, A, F, pc


@pytest.fixture(scope="module")
def table2_runs():
    from paper_2402_13747_b300 import _abi
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:1])
    ctx = _abi.Context(0)
    out = {}
    s = None
    for sim, n_diff in (("A", 0), ("B", 1)):
        p = config.params_for(sc, max_refl=5, max_diff=n_diff, max_int=5)
        if s is None:
            s = ctx.voxelize_scene(sc, p)
        out[sim] = (p,) + _run(ctx, s, sc, p)
    ctx.close()
    osc = oracle.Scene.from_scene(sc, out["B"][0])
    return sc, osc, out


@pytest.mark.parametrize("sim", ["A", "B"])
def test_table2_shape_invariants_and_samples(table2_runs, sim):
    sc, osc, out = table2_runs
    p, C, A, F, pc = out[sim]
    coarse_invariants(C, p)
    exact_invariants(F, p)
    assert len(C["n"]) > 10_000 and len(F["n"]) > 50
    assert C["n"].max() == 5                      # the depth limit is reached
    if sim == "B":
        assert (F["type"] == 1).any()             # diffracted exact paths exist
    sampled_refinement(sc, C, A, osc, 120, seed=31, min_both=20)
    sampled_visibility(sc, C, osc, 80, seed=32)
    cc = C["counts"]
    print(json.dumps({"sim": sim, "cones": cc["n_cones"], "vis_rays": cc["n_vis"], "nodes": cc["n_nodes"],
                      "coarse_raw": cc["n_coarse_raw"], "coarse": cc["n_coarse"], "exact": len(F["n"]),
                      "ms_levels": round(cc["ms_levels"], 1), "ms_refine": round(pc["ms_refine"], 1)}))


def test_table2_shape_fans_dominate(table2_runs):
    """One diffraction multiplies the cones: every diffracting node spawns a Keller fan."""
    _, _, out = table2_runs
    a, b = out["A"][1]["counts"], out["B"][1]["counts"]
    assert b["n_cones"] > 1.5 * a["n_cones"]
    assert b["n_nodes"] > a["n_nodes"]
