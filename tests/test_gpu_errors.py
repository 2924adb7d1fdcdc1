"""Error statuses of the boundary that a caller relies on: a device-memory budget too
small for the call (NIMBUS_ERR_OOM), and a bounded device wait that gives up
(NIMBUS_ERR_TIMEOUT).  Both failures are made on the host: a small budget, and a
wait limit of one cycle (nimbus_set_wait_limit).  Neither faults nor hangs the GPU:
every wait of the propagation levels ends at its limit and the kernel returns.
After each error the call must have freed what it allocated, and the context must
give the same results as before."""
import numpy as np
import pytest

from paper_2402_13747_b300 import _abi, config, scenes

pytestmark = pytest.mark.gpu


def _rows(cq):
    miss = np.asarray(cq["miss"], np.float32).view(np.uint32)
    return sorted(zip(cq["tx"].tolist(), cq["rx"].tolist(), cq["n"].tolist(), map(tuple, cq["ie"].tolist()),
                      map(tuple, cq["type"].tolist()), map(tuple, cq["label"].tolist()), miss.tolist()))


def test_budget_too_small_returns_oom():
    """A 64 KB budget cannot hold the tiny room's tables: voxelise returns
    NIMBUS_ERR_OOM, creates no scene and leaves nothing allocated; a context with room
    enough runs the same scene to its 25 paths."""
    sc = scenes.room_tiny()
    p = config.params_for(sc)
    ctx = _abi.Context(0, mem_budget=1 << 16)
    try:
        with pytest.raises(_abi.NimbusError) as e:
            ctx.voxelize_scene(sc, p)
        assert e.value.code == _abi.ERR_OOM
        assert "budget" in str(e.value)
        assert ctx.memory_used() == 0
    finally:
        ctx.close()
    ctx = _abi.Context(0, mem_budget=1 << 30)
    try:
        G = ctx.run(sc, p)
        assert len(G["n"]) == 25
    finally:
        ctx.close()


@pytest.mark.parametrize("layout", ["single_launch", "help_board"])
def test_wait_limit_gives_timeout_and_context_recovers(layout):
    """With every level wait limited to one cycle, the waits give up at once: in the
    single launch a warp that finds no task ready, in the per-depth launch with the
    help board a warp whose block still runs cones.  trace returns NIMBUS_ERR_TIMEOUT
    with the wait named, frees its buffers, and after the limit is lifted the same
    context traces the same coarse set with the same counters."""
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:3])
    p = config.params_for(sc, max_refl=2, max_diff=1)
    ctx = _abi.Context(0)
    try:
        ctx.set_tuning(level_queue=1 if layout == "single_launch" else 0, level_help=1, level_block=512)
        s = ctx.voxelize_scene(sc, p)
        c0 = ctx.trace(s, sc.tx, sc.rx, p)
        base, base_cc = _rows(ctx.query_coarse(c0)), ctx.coarse_counts(c0)
        ctx.release(c0)
        assert base_cc["n_coarse"] > 0
        used = ctx.memory_used()
        ctx.set_wait_limit(1)
        with pytest.raises(_abi.NimbusError) as e:
            ctx.trace(s, sc.tx, sc.rx, p)
        assert e.value.code == _abi.ERR_TIMEOUT
        assert "gave up" in str(e.value)
        assert ctx.memory_used() == used
        ctx.set_wait_limit(0)
        c1 = ctx.trace(s, sc.tx, sc.rx, p)
        assert _rows(ctx.query_coarse(c1)) == base
        cc = ctx.coarse_counts(c1)
        for k in ("n_cones", "n_vis", "n_nodes", "n_coarse", "n_coarse_raw", "bytes_levels"):
            assert cc[k] == base_cc[k], k
        ctx.release(c1)
        with pytest.raises(_abi.NimbusError) as e:
            ctx.set_wait_limit(-1)
        assert e.value.code == _abi.ERR_ARG
        ctx.release(s)
    finally:
        ctx.close()
