"""Continuous-batching request loop over resident voxelised scenes.

Requests name a resident scene, one TX, up to a few dozen RXs and a maximum
number of interactions.  Free workers (slots) pull the oldest waiting request
and batch with it the other waiting requests on the same scene, up to a pair
and a device-memory limit; one trace + refine call serves the whole batch
(each RX is tied to its request's TX and depth, so every request gets exactly
the paths it would get alone).  Requests that arrive while batches run are
admitted as soon as a slot and memory free up, and the workers' GPU work
overlaps on separate streams.  Dynamic scenes are updated by region: every
worker applies pending region updates to its resident copy before its next
batch on that scene.  Latency is measured from arrival to result.

The scheduler is plain host logic (unit-tested on CPU with a fake executor);
the executor drives the CUDA library through the C ABI.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from .config import Params


@dataclass
class Request:
    id: int
    scene: str
    tx: np.ndarray           # (1, 3)
    rx: np.ndarray           # (k, 3)
    depth: int               # maximum number of interactions
    t_arrival: float = 0.0
    future: Future = field(default_factory=Future)
    t_start: float = 0.0
    t_done: float = 0.0

    @property
    def pairs(self) -> int:
        return int(self.rx.shape[0])


def request_bytes(pairs: int, depth: int) -> int:
    """Device-memory estimate of one request: node buffers grow with depth."""
    per_level = {0: 1 << 16, 1: 1 << 17, 2: 1 << 18, 3: 1 << 20, 4: 1 << 21, 5: 1 << 22}.get(min(depth, 5), 1 << 22)
    return int(per_level * 40 * (depth + 1) + pairs * 100 * 320 + (64 << 20))


class Scheduler:
    """Waiting requests, the memory budget of in-flight batches, batch formation."""

    def __init__(self, mem_budget: int, max_pairs: int = 256, max_tx: int = 16):
        self.mem_budget = int(mem_budget)
        self.max_pairs = max_pairs
        self.max_tx = max_tx
        self.queue: deque[Request] = deque()
        self.in_flight = 0
        self.cv = threading.Condition()
        self.closed = False

    def submit(self, req: Request):
        with self.cv:
            self.queue.append(req)
            self.cv.notify_all()

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()

    def _form(self):
        """Oldest request plus followers on the same scene, of any depth (each RX keeps
        its request's depth limit and each TX's tree grows only as deep as its own
        RXs need, so a request's paths do not depend on its batch), within the pair,
        TX and memory limits."""
        if not self.queue:
            return None
        head = self.queue[0]
        free = self.mem_budget - self.in_flight
        batch, pairs, depth = [], 0, 0
        for r in list(self.queue):
            if r.scene != head.scene:
                continue
            d = max(depth, r.depth)
            est = request_bytes(pairs + r.pairs, d) * (len(batch) + 1)
            if batch and (pairs + r.pairs > self.max_pairs or len(batch) >= self.max_tx or est > free):
                continue
            if not batch and est > free and self.in_flight > 0:
                return None          # wait until memory frees up
            batch.append(r)
            pairs += r.pairs
            depth = d
        for r in batch:
            self.queue.remove(r)
        return batch, request_bytes(pairs, depth) * len(batch)

    def next_batch(self, timeout: float = 0.1):
        """Block until a batch can be admitted (or timeout / close); returns (batch, bytes)."""
        with self.cv:
            end = time.perf_counter() + timeout
            while True:
                got = self._form()
                if got is not None:
                    batch, est = got
                    self.in_flight += est
                    return batch, est
                if self.closed:
                    return None
                left = end - time.perf_counter()
                if left <= 0:
                    return None
                self.cv.wait(left)

    def done(self, est: int):
        with self.cv:
            self.in_flight -= est
            self.cv.notify_all()


class GpuExecutor:
    """One worker's context, stream and resident scene copies."""

    def __init__(self, scenes: dict, params: Params, device: int = 0):
        import torch
        from . import _abi
        self.torch = torch
        self.ctx = _abi.Context(device)
        self.stream = torch.cuda.Stream(device=device)
        self.params = params
        self.handles = {}
        self.applied = {}
        self.need = {}   # (scene, depth) -> largest node / coarse counts per TX seen so far
        self.resident = {}   # device bytes of each resident scene in this worker's context
        self.update_ms = []  # wall time of each region update applied
        for sid, sc in scenes.items():
            before = self.ctx.memory_used()
            self.handles[sid] = self.ctx.voxelize_scene(sc, params, stream=self.stream)
            self.resident[sid] = self.ctx.memory_used() - before
            self.applied[sid] = 0

    def apply_updates(self, sid: str, updates: list):
        for k in range(self.applied.get(sid, 0), len(updates)):
            lo, hi, cloud = updates[k]
            t0 = time.perf_counter()
            self.ctx.update_region(self.handles[sid], lo, hi, *cloud, stream=self.stream)
            self.stream.synchronize()
            self.update_ms.append(1e3 * (time.perf_counter() - t0))
        self.applied[sid] = len(updates)

    def run(self, batch: list[Request]) -> list[dict]:
        """One trace + refine for a batch; the exact paths split per request."""
        sid = batch[0].scene
        tx = np.concatenate([r.tx.reshape(1, 3) for r in batch])
        rx = np.concatenate([r.rx.reshape(-1, 3) for r in batch])
        owner = np.concatenate([np.full(r.pairs, i, np.int32) for i, r in enumerate(batch)])
        depth = np.concatenate([np.full(r.pairs, r.depth, np.int32) for r in batch])
        rx_off = np.cumsum([0] + [r.pairs for r in batch])
        dmax = int(max(r.depth for r in batch))
        p = self.params.replace(max_refl=dmax, max_diff=min(1, dmax), max_int=dmax)
        # node / coarse buffers: sized from what this scene and depth needed per TX in
        # earlier batches (the library's defaults at first); a batch that still
        # overflows is traced again with the sizes the first pass reported
        n_tx = len(batch)
        per_tx = self.need.get((sid, dmax))
        caps = (0, 0) if per_tx is None else (max(1 << 23, int(per_tx[0] * n_tx * 1.25)),
                                              max(1 << 23, int(per_tx[1] * n_tx * 1.25)))
        for attempt in range(2):
            c = self.ctx.trace(self.handles[sid], tx, rx, p, rx_owner=owner, rx_max_int=depth, max_nodes=caps[0],
                               max_coarse=caps[1], stream=self.stream, allow_overflow=True)
            cc = self.ctx.coarse_counts(c, stream=self.stream)
            ov = cc["overflow"]
            if ov:
                seen = (cc["needed_nodes"] / n_tx, cc["needed_coarse"] / n_tx)
                old = self.need.get((sid, dmax), (0, 0))
                self.need[(sid, dmax)] = (max(old[0], seen[0]), max(old[1], seen[1]))
            if not ov or attempt == 1:
                break
            self.ctx.release(c)
            caps = (max(1 << 23, int(cc["needed_nodes"] * 1.2)), max(1 << 23, int(cc["needed_coarse"] * 1.2)))
        P = self.ctx.refine(self.handles[sid], c, p, stream=self.stream)
        out = self.ctx.query(P, 0, stream=self.stream)
        self.ctx.release(P)
        self.ctx.release(c)
        res = []
        for i, r in enumerate(batch):
            m = out["tx"] == i
            sub = {k: v[m] for k, v in out.items() if k != "counts"}
            sub["tx"] = np.zeros(int(m.sum()), np.int32)
            sub["rx"] = sub["rx"] - rx_off[i]
            sub["overflow"] = int(ov)
            res.append(sub)
        res_counts = out["counts"]
        return res, res_counts

    def close(self):
        for h in self.handles.values():
            self.ctx.release(h)
        self.ctx.close()


class Server:
    """Worker threads pulling batches from a shared scheduler."""

    def __init__(self, scenes: dict, params: Params | None = None, n_workers: int = 2, mem_budget: int = 32 << 30,
                 max_pairs: int = 256, executor_factory=None, device: int = 0):
        self.params = params or Params()
        self.sched = Scheduler(mem_budget, max_pairs=max_pairs)
        self.updates: dict[str, list] = {sid: [] for sid in scenes}
        self.lock = threading.Lock()
        self.completed: list[Request] = []
        self.cones = 0
        self.batches = 0
        factory = executor_factory or (lambda: GpuExecutor(scenes, self.params, device))
        self.executors = [factory() for _ in range(n_workers)]
        self.threads = [threading.Thread(target=self._loop, args=(e,), daemon=True) for e in self.executors]
        self._next_id = 0
        for t in self.threads:
            t.start()

    def submit(self, scene: str, tx, rx, depth: int, t_arrival: float | None = None) -> Request:
        with self.lock:
            rid = self._next_id
            self._next_id += 1
        req = Request(rid, scene, np.asarray(tx, np.float64).reshape(1, 3), np.asarray(rx, np.float64).reshape(-1, 3),
                      int(depth), time.perf_counter() if t_arrival is None else t_arrival)
        self.sched.submit(req)
        return req

    def update_region(self, scene: str, lo, hi, cloud):
        """Replace the points inside [lo, hi] by `cloud` (xyz, nrm, label, material)."""
        with self.lock:
            self.updates[scene].append((np.asarray(lo, float), np.asarray(hi, float), cloud))

    def _loop(self, ex):
        while True:
            got = self.sched.next_batch(timeout=0.05)
            if got is None:
                if self.sched.closed and not self.sched.queue:
                    return
                continue
            batch, est = got
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                with self.lock:
                    ups = list(self.updates[batch[0].scene])
                ex.apply_updates(batch[0].scene, ups)
                results, counts = ex.run(batch)
                t1 = time.perf_counter()
                with self.lock:
                    self.cones += counts.get("n_cones", 0)
                    self.batches += 1
                for r, res in zip(batch, results):
                    r.t_done = t1
                    r.future.set_result(res)
                    with self.lock:
                        self.completed.append(r)
            except Exception as e:  # report the failure on every request of the batch not yet answered
                for r in batch:
                    if not r.future.done():
                        r.t_done = time.perf_counter()
                        r.future.set_exception(e)
            finally:
                self.sched.done(est)

    def close(self):
        self.sched.close()
        for t in self.threads:
            t.join(timeout=600)
        for e in self.executors:
            if hasattr(e, "close"):
                e.close()

    def stats(self, since: int = 0) -> dict:
        """Latency (arrival to result), service time (batch start to result) and
        counts over the requests completed after the first `since`; per class
        (scene, depth) the p50 / p99 latency and the count."""
        done = self.completed[since:]
        lat = np.array([r.t_done - r.t_arrival for r in done])
        svc = np.array([r.t_done - r.t_start for r in done])
        paths = sum(len(r.future.result()["n"]) for r in done if r.future.done() and r.future.exception() is None)
        pct = lambda a, q: float(np.percentile(a, q) * 1e3) if len(a) else None  # noqa: E731
        classes = {}
        for key in sorted({(r.scene, r.depth) for r in done}):
            a = np.array([r.t_done - r.t_arrival for r in done if (r.scene, r.depth) == key])
            classes[f"{key[0]}/d{key[1]}"] = {"n": int(len(a)), "p50_ms": pct(a, 50), "p99_ms": pct(a, 99)}
        return {"requests": len(done), "batches": self.batches,
                "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "service_p50_ms": pct(svc, 50),
                "service_p99_ms": pct(svc, 99), "exact_paths": paths, "cones": self.cones, "by_class": classes}


def run_stream(server: Server, requests: list[dict], scenes_update=None, update_every: int = 50,
               time_scale: float = 1.0) -> dict:
    """Submit a timed request stream (arrival times in seconds; all at once with
    time_scale 0) and wait for all results; figures over this stream alone.  Every
    update_every requests scenes_update(k) posts a region update."""
    since, b0, c0 = len(server.completed), server.batches, server.cones
    t0 = time.perf_counter()
    reqs, updates = [], 0
    for k, q in enumerate(requests):
        due = t0 + q["t"] * time_scale
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        if scenes_update is not None and k > 0 and k % update_every == 0:
            scenes_update(k // update_every)
            updates += 1
        reqs.append(server.submit(q["scene"], q["tx"], q["rx"], q["depth"], t_arrival=due))
    for r in reqs:
        r.future.exception()   # wait
    wall = time.perf_counter() - t0
    st = server.stats(since)
    st["batches"] = server.batches - b0
    st["cones"] = server.cones - c0
    st["region_updates"] = updates
    st["wall_s"] = wall
    st["requests_per_s"] = len(reqs) / wall
    st["exact_paths_per_s"] = st["exact_paths"] / wall
    st["rays_per_s"] = st["cones"] / wall
    return st


def bench_latency(ctx=None, device: int = 0, n_requests: int = 36, fractions=(0.5, 0.8, 1.0), n_workers: int = 2,
                  seed: int = 4, max_pairs: int = 64, depth_range=(2, 5), depth_caps=None, update_every: int = 12,
                  burst: int = 24) -> dict:
    """Serving measurement on the three resident scenes of the larger configurations.

    Resident: the noisy room with its box (133k points), the indoor scan (1.92M) and
    the street canyon (20.0M).  Each request picks a scene, 1 TX and 1..max_pairs RXs
    from free-space positions of that scene, and a maximum depth in depth_range,
    capped per scene where deeper trees leave the latency budget (street: 2, indoor
    and room: 4; node counts grow about 6x per level in the open street, and a
    64-pair depth-5 request in the room refines millions of coarse paths).  First a
    burst of `burst` requests, all arriving at once, measures the batched capacity
    (requests per second); then one seeded Poisson stream of n_requests at each
    fraction of that capacity.  A 2x2x2 m box moves in the noisy room and is
    re-voxelised by region every update_every requests of a stream.  Returns the
    capacity, and per rate p50/p99 latency, per-class latency, batches, region
    updates and throughput; the resident bytes of each scene (every worker holds
    its own copy).
    """
    from . import scenes
    caps = {"street": 2, "indoor": 4, "room_noisy": 4} if depth_caps is None else depth_caps
    room = scenes.room_noisy(n_tx=1, n_rx=1)
    indoor = scenes.indoor(n_rx=512)
    street = scenes.street(n_rx=512)
    sc = {"room_noisy": room, "indoor": indoor, "street": street}
    pools = {"room_noisy": scenes.room_noisy_pairs(900, 1, 512)[1], "indoor": indoor.rx, "street": street.rx}
    server = Server(sc, Params(), n_workers=n_workers, device=device, max_pairs=128)
    state = {"box": None, "step": 0}

    def move(_k):
        state["step"] += 1
        server.update_region("room_noisy", *moved_box_update(room, state, state["step"]))

    kw = dict(max_pairs=max_pairs, depth_range=depth_range, pools=pools, depth_caps=caps)
    out = {"scenes": {k: int(v.xyz.shape[0]) for k, v in sc.items()}, "workers": n_workers,
           "pairs_per_request": f"1-{max_pairs}", "depth": f"{depth_range[0]}-{depth_range[1]}", "depth_caps": caps,
           "moving_box": f"2x2x2 m in the noisy room, region update every {update_every} requests of a stream"}
    try:
        ex = server.executors[0]
        out["resident_bytes_per_worker"] = {k: int(v) for k, v in getattr(ex, "resident", {}).items()}
        reqs = scenes.serving_requests(burst, 1.0, list(sc), seed=seed, **kw)
        cap = run_stream(server, reqs, time_scale=0.0)
        capacity = cap["requests_per_s"]
        out["capacity"] = {"requests_per_s": capacity, "burst": burst, "p50_ms": cap["p50_ms"],
                           "p99_ms": cap["p99_ms"], "batches": cap["batches"], "wall_s": cap["wall_s"]}
        out["rates"] = []
        for i, fr in enumerate(fractions):
            reqs = scenes.serving_requests(n_requests, fr * capacity, list(sc), seed=seed + 1 + i, **kw)
            st = run_stream(server, reqs, scenes_update=move, update_every=update_every)
            st["fraction_of_capacity"] = fr
            st["rate_hz"] = fr * capacity
            out["rates"].append(st)
        ups = [u for e in server.executors for u in getattr(e, "update_ms", [])]
        out["region_update_ms_p50"] = float(np.median(ups)) if ups else None
    finally:
        server.close()
    return out


def moved_box_update(room, state: dict, step: int):
    """Region update for the moving box: the box of the walk's `step` replaces the
    region that held the previous box.  The region covers both boxes; it is refilled
    with the room's own points there (minus the floor under the new box) plus the box."""
    from . import scenes
    xyz, nrm, lab, mat, lo, hi = scenes.moving_box(room, step)
    old = state.get("box")
    r_lo = (np.minimum(lo, old[0]) if old is not None else lo) - 0.01
    r_hi = (np.maximum(hi, old[1]) if old is not None else hi) + 0.01
    r_lo32, r_hi32 = r_lo.astype(np.float32), r_hi.astype(np.float32)
    inside = np.all((room.xyz >= r_lo32) & (room.xyz <= r_hi32), axis=1)
    under = ((room.xyz[:, 0] >= lo[0]) & (room.xyz[:, 0] <= hi[0]) & (room.xyz[:, 1] >= lo[1]) &
             (room.xyz[:, 1] <= hi[1]) & (room.label == 4))
    keep = inside & ~under
    cloud = (np.concatenate([room.xyz[keep], xyz]), np.concatenate([room.nrm[keep], nrm]),
             np.concatenate([room.label[keep], lab]), np.concatenate([room.material[keep], mat]))
    state["box"] = (lo, hi)
    return r_lo, r_hi, cloud
