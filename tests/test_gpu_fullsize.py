"""The benchmark workload at full size, in the configuration bench.py times, checked
on sampled outputs the oracle computes one by one (needs a B300)."""
import pytest

import oracle
from paper_2402_13747_b300 import config, scenes
from tests.sampled import coarse_invariants, exact_invariants, sampled_refinement, sampled_visibility

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
    assert len(C["n"]) == len(A["n"]) > 100_000
    coarse_invariants(C, p)
    exact_invariants(F, p)
    assert len(F["n"]) > 1000


def test_sampled_refinement_matches_oracle(full_run):
    """200 sampled coarse paths of the full workload refined by the oracle one by one."""
    sc, p, C, A, F, osc = full_run
    sampled_refinement(sc, C, A, osc, 200, seed=21, min_both=40)


def test_sampled_coarse_segments_are_visible(full_run):
    """Each segment of a sampled coarse path passes the oracle's visibility test."""
    sc, p, C, A, F, osc = full_run
    sampled_visibility(sc, C, osc, 150, seed=22)
