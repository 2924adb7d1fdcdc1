"""The help board's counting rule, on the host.

At the last propagation level a cone's point IEs only decide where it stops: walked in
order, the point IEs after the first visible one are skipped.  With the board, the
candidates of one evaluation are walked by several warps in any order; a warp skips a
point-IE entry only when a visible point IE with a smaller index is already known, and
the owner then counts (rays and bytes) exactly the entries the in-order walk tests:
every RX entry, and the point-IE entries up to and including the first visible one.
This model of that protocol, run under random interleavings, checks the two facts the
CUDA board relies on: every entry the in-order walk tests is walked whatever the
order, and the counted set equals the in-order walk's tested set.  Entries are split
into batches as the board's slot capacity splits them; the first visible index carries
over from batch to batch within the evaluation.
"""
import numpy as np

POINT, RX = 0, 2


def in_order(kinds, visible):
    """Indices the in-order walk tests (the last level: no children)."""
    tested, stop = [], False
    for q, (k, v) in enumerate(zip(kinds, visible)):
        if k == POINT and stop:
            continue
        tested.append(q)
        if k == POINT and v:
            stop = True
    return tested


def board(kinds, visible, cap, warps, rng):
    """The board: batches of at most cap entries, each walked by `warps` warps that
    take entries in ticket order but finish them in a random order; returns (walked,
    counted) index lists."""
    n = len(kinds)
    first_vis = np.iinfo(np.int64).max
    walked, counted = [], []
    for base in range(0, n, cap):
        batch = list(range(base, min(n, base + cap)))
        # each entry is taken in ticket order; its skip decision reads first_vis when
        # its warp takes it, and its visibility lands in first_vis when its walk ends:
        # simulate with a random number of walks still in flight at each decision
        pending = []          # (q, visible) walks taken but not finished
        done = []
        for q in batch:
            # finish a random subset of the walks in flight
            keep = []
            for item in pending:
                if rng.random() < 0.5:
                    done.append(item)
                else:
                    keep.append(item)
            pending = keep[-(warps - 1):] if warps > 1 else []
            done += keep[:max(0, len(keep) - (warps - 1))]
            for dq, dv in done:
                if kinds[dq] == POINT and dv:
                    first_vis = min(first_vis, dq)
            done = []
            skip = kinds[q] == POINT and first_vis < q
            if not skip:
                walked.append(q)
                pending.append((q, visible[q]))
        for dq, dv in pending:
            if kinds[dq] == POINT and dv:
                first_vis = min(first_vis, dq)
        # the owner counts after the batch: every walked RX, walked point IEs <= first_vis
        for q in batch:
            if q in walked and (kinds[q] == RX or q <= first_vis):
                counted.append(q)
    return walked, counted


def test_counted_set_is_the_in_order_walk():
    rng = np.random.default_rng(3)
    extra = 0   # cases where the board walked entries the in-order walk skips
    for _ in range(3000):
        n = int(rng.integers(1, 150))
        kinds = np.where(rng.random(n) < 0.2, RX, POINT)
        visible = rng.random(n) < rng.choice([0.02, 0.1, 0.5])
        ref = in_order(kinds, visible)
        for cap, warps in ((64, 1), (64, 16), (7, 4), (1, 3)):
            walked, counted = board(kinds, visible, cap, warps, rng)
            assert set(ref) <= set(walked), (kinds, visible, cap, warps)
            assert counted == ref, (kinds, visible, cap, warps)
            extra += len(walked) > len(ref)
    assert extra > 100, extra


def test_a_plain_point_sequence():
    """Five point IEs, the third visible: the in-order walk tests the first three; on
    the board the fourth and fifth may be walked too, but are not counted."""
    kinds = np.array([POINT] * 5)
    visible = np.array([False, False, True, False, True])
    assert in_order(kinds, visible) == [0, 1, 2]
    rng = np.random.default_rng(0)
    walked, counted = board(kinds, visible, 64, 16, rng)
    assert counted == [0, 1, 2] and set(walked) >= {0, 1, 2}
