"""The larger synthetic configurations on the GPU (needs a B300): the indoor scan
(2M points, 1 TX x 256 RX, <= 3 reflections + 1 diffraction) at its full size, and
the street canyon (20M points) at its full 16 TX x 1024 RX pair set with <= 1
reflection + 1 diffraction and on 2 TX x 16 RX with <= 2 reflections + 1
diffraction.  Voxel tables are compared bit for bit; paths on sampled outputs the
oracle computes one by one."""
import pytest

import oracle
from paper_2402_13747_b300 import config, scenes
from tests.sampled import coarse_invariants, exact_invariants, sampled_refinement, sampled_visibility
from tests.test_gpu_parity import _tables_match

pytestmark = pytest.mark.gpu


def _run(sc, p):
    from paper_2402_13747_b300 import _abi
    ctx = _abi.Context(0)
    s = ctx.voxelize_scene(sc, p)
    c = ctx.trace(s, sc.tx, sc.rx, p, allow_overflow=True)
    C = ctx.query_coarse(c)
    if C["counts"]["overflow"]:
        # grow the level and coarse buffers to what the first pass reported
        need_n, need_c = C["counts"]["needed_nodes"], C["counts"]["needed_coarse"]
        ctx.release(c)
        c = ctx.trace(s, sc.tx, sc.rx, p, max_nodes=max(8 << 20, int(need_n * 1.1)),
                      max_coarse=max(8 << 20, int(need_c * 1.1)))
        C = ctx.query_coarse(c)
    P = ctx.refine(s, c, p)
    A = ctx.query(P, 1)
    F = ctx.query(P, 0)
    ctx.close()
    return C, A, F


@pytest.fixture(scope="module")
def indoor():
    sc = scenes.indoor()
    p = config.params_for(sc)
    C, A, F = _run(sc, p)
    return sc, p, C, A, F, oracle.Scene.from_scene(sc, p)


@pytest.fixture(scope="module")
def street():
    return scenes.street()


def test_indoor_tables_match_oracle(indoor):
    from paper_2402_13747_b300 import _abi
    sc, p = indoor[0], indoor[1]
    ctx = _abi.Context(0)
    _tables_match(ctx, sc, p)
    ctx.close()


def test_indoor_full_config(indoor):
    sc, p, C, A, F, osc = indoor
    assert sc.xyz.shape[0] > 1_800_000 and sc.rx.shape[0] == 256
    assert len(C["n"]) > 100_000
    coarse_invariants(C, p)
    exact_invariants(F, p)
    sampled_refinement(sc, C, A, osc, 120, seed=31)
    sampled_visibility(sc, C, osc, 100, seed=32)


def test_street_tables_match_oracle(street):
    from paper_2402_13747_b300 import _abi
    ctx = _abi.Context(0)
    _tables_match(ctx, street, config.params_for(street))
    ctx.close()


def test_street_all_pairs_one_bounce(street):
    sc = street
    p = config.params_for(sc, max_refl=1, max_diff=1)
    assert sc.xyz.shape[0] > 19_000_000 and sc.tx.shape[0] * sc.rx.shape[0] == 16 * 1024
    C, A, F = _run(sc, p)
    assert len(C["n"]) > 1_000_000
    coarse_invariants(C, p)
    exact_invariants(F, p)
    osc = oracle.Scene.from_scene(sc, p)
    sampled_refinement(sc, C, A, osc, 120, seed=41)
    sampled_visibility(sc, C, osc, 100, seed=42)


def test_street_two_bounces_subset(street):
    sc = street.with_pairs(street.tx[:2], street.rx[:16])
    p = config.params_for(sc, max_refl=2, max_diff=1)
    C, A, F = _run(sc, p)
    coarse_invariants(C, p)
    exact_invariants(F, p)
    osc = oracle.Scene.from_scene(sc, p)
    sampled_refinement(sc, C, A, osc, 100, seed=43)
    sampled_visibility(sc, C, osc, 60, seed=44)
