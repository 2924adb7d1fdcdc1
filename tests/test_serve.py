"""Continuous-batching scheduler (host logic, CPU) and the served results (GPU)."""
import threading
import time

import numpy as np
import pytest

from paper_2402_13747_b300 import config, scenes
from paper_2402_13747_b300.serve import Scheduler, Server, request_bytes, run_stream
from tests.pathsets import keyed


class FakeExecutor:
    """Stands in for the GPU: sleeps, records batches, returns one fake path per RX."""

    shared = {"busy": 0, "max_busy": 0}
    lock = threading.Lock()

    def __init__(self, delay=0.05, log=None):
        self.delay = delay
        self.log = log if log is not None else []
        self.updates = {}

    def apply_updates(self, sid, ups):
        self.updates[sid] = len(ups)

    def run(self, batch):
        with self.lock:   # concurrency over all executors
            self.shared["busy"] += 1
            self.shared["max_busy"] = max(self.shared["max_busy"], self.shared["busy"])
        self.log.append([(r.id, r.scene) for r in batch])
        time.sleep(self.delay)
        with self.lock:
            self.shared["busy"] -= 1
        res = [{"n": np.zeros(r.pairs, np.int32), "rx": np.arange(r.pairs), "tx": np.zeros(r.pairs, np.int32),
                "id": r.id} for r in batch]
        return res, {"n_cones": 7 * len(batch)}


def _server(n_workers=1, delay=0.05, mem=1 << 40, max_pairs=256):
    log = []
    srv = Server({"a": None, "b": None}, config.Params(), n_workers=n_workers, mem_budget=mem, max_pairs=max_pairs,
                 executor_factory=lambda: FakeExecutor(delay, log))
    return srv, log


class FailingExecutor(FakeExecutor):
    """A device call that fails for requests on scene "bad" (an error from the library)."""

    def run(self, batch):
        if batch[0].scene == "bad":
            raise RuntimeError("NIMBUS_ERR_OOM: device memory budget exhausted")
        return super().run(batch)


def test_a_failed_batch_reports_its_error_and_the_worker_keeps_serving():
    """A batch whose device call fails: each of its requests gets the error, the memory
    it held is returned to the scheduler, and the same worker serves the next batches."""
    srv = Server({"a": None, "bad": None}, config.Params(), n_workers=1, mem_budget=1 << 40,
                 executor_factory=lambda: FailingExecutor(0.01))
    bad = [srv.submit("bad", [0, 0, 0], np.zeros((1, 3)), 2) for _ in range(3)]
    good = [srv.submit("a", [0, 0, 0], np.zeros((2, 3)), 2) for _ in range(3)]
    for r in bad:
        with pytest.raises(RuntimeError, match="NIMBUS_ERR_OOM"):
            r.future.result(timeout=30)
    for r in good:
        assert r.future.result(timeout=30)["id"] == r.id
    later = srv.submit("a", [0, 0, 0], np.zeros((1, 3)), 2)
    assert later.future.result(timeout=30)["id"] == later.id
    end = time.perf_counter() + 5.0          # a batch returns its memory just after its results
    while srv.sched.in_flight and time.perf_counter() < end:
        time.sleep(0.01)
    assert srv.sched.in_flight == 0
    srv.close()


def test_batches_hold_one_scene_and_route_results():
    srv, log = _server(delay=0.1)
    reqs = [srv.submit("a" if i % 2 else "b", [1, 1, 1], np.zeros((2, 3)), 2) for i in range(9)]
    for r in reqs:
        assert r.future.result(timeout=30)["id"] == r.id
    srv.close()
    for batch in log:
        assert len({s for _, s in batch}) == 1
    assert sorted(i for b in log for i, _ in b) == list(range(9))


def test_requests_arriving_during_a_batch_join_the_next_one():
    srv, log = _server(delay=0.3)
    first = srv.submit("a", [0, 0, 0], np.zeros((1, 3)), 2)
    time.sleep(0.1)                                   # first batch is on the "GPU"
    later = [srv.submit("a", [0, 0, 0], np.zeros((1, 3)), 3) for _ in range(5)]
    for r in [first] + later:
        r.future.result(timeout=30)
    srv.close()
    assert [i for i, _ in log[0]] == [first.id]
    assert sorted(i for i, _ in log[1]) == sorted(r.id for r in later)   # admitted together


def test_memory_budget_limits_batches_in_flight():
    one = request_bytes(1, 2)
    for mem, allowed in ((int(1.5 * one), 1), (int(3.5 * one), 3)):
        FakeExecutor.shared.update(busy=0, max_busy=0)
        srv, log = _server(n_workers=3, delay=0.15, mem=mem, max_pairs=1)
        reqs = [srv.submit("a", [0, 0, 0], np.zeros((1, 3)), 2) for _ in range(6)]
        for r in reqs:
            r.future.result(timeout=30)
        srv.close()
        assert FakeExecutor.shared["max_busy"] <= allowed   # batches in flight fit the budget
        assert srv.sched.in_flight == 0
    assert FakeExecutor.shared["max_busy"] >= 2            # with room, workers do overlap


def test_pair_limit_splits_batches():
    s = Scheduler(1 << 40, max_pairs=10)
    from paper_2402_13747_b300.serve import Request
    for i in range(5):
        s.submit(Request(i, "a", np.zeros((1, 3)), np.zeros((4, 3)), 2))
    b1, _ = s.next_batch()
    b2, _ = s.next_batch()
    b3, _ = s.next_batch()
    assert [len(b1), len(b2), len(b3)] == [2, 2, 1]


def test_uneven_depths_share_a_batch():
    """Requests of one scene with different depth limits and pair counts join one
    batch; another scene's request waits for its own."""
    s = Scheduler(1 << 40, max_pairs=64)
    from paper_2402_13747_b300.serve import Request
    for i, (sid, k, d) in enumerate([("a", 3, 2), ("a", 7, 5), ("b", 1, 3), ("a", 1, 4)]):
        s.submit(Request(i, sid, np.zeros((1, 3)), np.zeros((k, 3)), d))
    b1, _ = s.next_batch()
    b2, _ = s.next_batch()
    assert [r.id for r in b1] == [0, 1, 3] and sorted(r.depth for r in b1) == [2, 4, 5]
    assert [r.id for r in b2] == [2]


def test_stream_reports_latency_percentiles():
    srv, log = _server(n_workers=2, delay=0.02)
    reqs = scenes.serving_requests(30, 200.0, ["a", "b"], seed=1, max_pairs=8)
    st = run_stream(srv, reqs)
    srv.close()
    assert st["requests"] == 30 and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["rays_per_s"] > 0 and st["batches"] <= 30
    assert sum(c["n"] for c in st["by_class"].values()) == 30


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    """A request served alone and the same request batched with others: same paths."""
    room = scenes.room_noisy(n_tx=1, n_rx=1)
    rng = np.random.default_rng(12)
    lo, hi = np.array([0.4, 0.4, 0.4]), np.array([9.6, 9.6, 2.6])
    qs = []
    for k in range(6):
        tx = lo + (hi - lo) * rng.random(3)
        while 4.2 <= tx[0] <= 5.8 and 6.2 <= tx[1] <= 7.8:
            tx = lo + (hi - lo) * rng.random(3)
        rx = lo + (hi - lo) * rng.random((1 + k % 4, 3))
        rx = rx[~((rx[:, 0] >= 4.2) & (rx[:, 0] <= 5.8) & (rx[:, 1] >= 6.2) & (rx[:, 1] <= 7.8))]
        qs.append((tx, rx, 2 + k % 2))
    alone = []
    srv = Server({"room": room}, config.Params(), n_workers=1)
    for tx, rx, d in qs:
        alone.append(srv.submit("room", tx, rx, d).future.result(timeout=600))
    srv.close()
    srv = Server({"room": room}, config.Params(), n_workers=2)
    reqs = [srv.submit("room", tx, rx, d) for tx, rx, d in qs]
    mixed = [r.future.result(timeout=600) for r in reqs]
    batches = srv.batches
    srv.close()
    assert batches < len(qs)            # the mix really was batched
    for a, m in zip(alone, mixed):
        ka, km = keyed(a), keyed(m)
        assert ka.keys() == km.keys()
        for k in ka:
            np.testing.assert_allclose(ka[k][0], km[k][0], atol=1e-6)
            assert abs(ka[k][1] - km[k][1]) <= 1e-9 * ka[k][1]
