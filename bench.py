"""Benchmark: the point-cloud ray launcher's whole hot path on synthetic scenes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole path -- voxelisation of the cloud, coarse path
tracing for every TX/RX pair and refinement with duplicate removal -- over the
noisy box room: 10x10x3 m at 5 cm (~133k points, 5 mm position noise, 2 degree
normal tilt), a 1x1x2 m box with 8 exterior edges, 4 TX x 16 RX, up to 3
reflections and 1 diffraction.  Inputs are resident on the device when the timed
region starts; L2 is flushed between timed steps (the scene fits in L2).

Metric: rays/s = cones traced (uniform TX launch + every propagation level +
Keller fans) per second of step time, with exact paths/s beside it, the batched
form (all pairs in one trace + refine) against the plain form (one trace +
refine per TX/RX pair), and p50/p99 request latency of the serving loop.

N > 1 (torchrun): each rank runs the same workload with its own seeded TX/RX
draw (weak scaling, no collective on the data path; a barrier brackets timing).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (1 TX x 16 RX, <= 1 reflection + 1 diffraction) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "rays/s and exact paths/s on 1 B300, batched vs plain; p50/p99 request latency"
WORKLOAD = ("room_noisy: 10x10x3 m box room at 5 cm (~133k pts, sigma 5 mm / 2 deg noise), 1x1x2 m box "
            "with 8 exterior edges, 4 TX x 16 RX, <=3 reflections + <=1 diffraction, kappa 100, rho 2000")
CPU_SAMPLE = "room_noisy geometry, 1 TX x 16 RX, <=1 reflection + <=1 diffraction, full 0.5 deg launch"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# DRAM traffic of one full-size refine launch (dram__bytes_read.sum + dram__bytes_write.sum,
# one-pass ncu capture of a k_refine launch of this workload), valid only for the device
# code it was taken on: the hash below covers that code -- refine.cu up to its host
# launcher, and the two headers whole -- and a changed kernel reports null.
REFINE_TRAFFIC = {"bytes": 52.97e6 + 99.52e6, "sources_sha256": "2309aa0d002312697627dcaa165922f93141daba6e930a7497bd3c373c7e0daf"}
KERNEL_SOURCES = (("paper_2402_13747_b300/csrc/refine.cu", b"\nint refine_paths("),
                  ("paper_2402_13747_b300/csrc/warp_geom.cuh", None),
                  ("paper_2402_13747_b300/csrc/nimbus_internal.cuh", None))


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f, end in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            text = fh.read()
        if end is not None:
            cut = text.find(end)
            if cut < 0:
                raise RuntimeError(f"{f}: no {end!r} to end the hashed device code")
            text = text[:cut]
        h.update(text)
    return h.hexdigest()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"nimbus_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2402_13747_b300 import config, scenes
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:16])
    p = config.params_for(sc, max_refl=1, max_diff=1)
    times, cones, paths = [], 0, 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s, c, e = oracle.run(sc, p)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            cones += c.stats["n_cones"]
            paths += len(e.paths()["n"])
    T = sum(times)
    v = cones / T
    line = {"metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": CPU_SAMPLE}, "impl": "reference",
            "exact_paths_per_s": paths / T,
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": 1, "kind": "oracle", "sample": CPU_SAMPLE},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline():
    """The oracle as it stands, single-threaded, on a bounded sample of the workload."""
    import oracle
    from paper_2402_13747_b300 import config, scenes
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:16])
    p = config.params_for(sc, max_refl=1, max_diff=1)
    t0 = time.perf_counter()
    s, c, e = oracle.run(sc, p)
    T = time.perf_counter() - t0
    return {"value": c.stats["n_cones"] / T, "unit": "rays/s", "cores": 1, "kind": "oracle",
            "sample": CPU_SAMPLE + f" ({T:.1f} s, {c.stats['n_cones']} cones, {len(e.paths()['n'])} exact paths)",
            "exact_paths_per_s": len(e.paths()["n"]) / T}


def rank_scene(rank: int):
    """The workload of one rank: the same noisy room on every rank; rank 0 uses the
    scene's own 4 TX x 16 RX, rank r > 0 its own seeded draw (weak scaling)."""
    from paper_2402_13747_b300 import scenes
    sc = scenes.room_noisy()
    if rank:
        sc = sc.with_pairs(*scenes.room_noisy_pairs(1000 + rank, sc.tx.shape[0], sc.rx.shape[0]))
    return sc


def reduce_over_ranks(t_total: float, cones: float, paths: float, device, *more: float):
    """Whole-job figures after the timed region: the slowest rank's time and the
    units of all ranks -- cones, paths and any further counts -- (the only
    collectives; none on the data path)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_total, cones, paths, *more], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    units = t[1:].clone()
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    return (float(tmax[0]),) + tuple(float(u) for u in units)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-segment", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pairs", default="", help="TxR: only the first T TX and R RX (small profiling cases)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2402_13747_b300 import _abi, config, scenes
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sc = rank_scene(rank)
    workload = WORKLOAD
    if args.pairs:
        nt, nr = (int(v) for v in args.pairs.lower().split("x"))
        sc = sc.with_pairs(sc.tx[:nt], sc.rx[:nr])
        workload = WORKLOAD.replace("4 TX x 16 RX", f"{nt} TX x {nr} RX (subset)")
    p = config.params_for(sc)
    dev = torch.device("cuda", local)
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    d_xyz, d_nrm = T(sc.xyz, torch.float32), T(sc.nrm, torch.float32)
    d_lab = T(sc.label.astype(np.int64), torch.int64).to(torch.int32)
    d_mat = T(sc.material, torch.uint8)
    d_edges, d_elab = T(sc.edges, torch.float64), T(sc.edge_label.astype(np.int64), torch.int64).to(torch.int32)
    d_tx, d_rx = T(sc.tx, torch.float64), T(sc.rx, torch.float64)
    ctx = _abi.Context(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # larger than the 126 MB L2

    def step():
        s = ctx.voxelize(d_xyz, d_nrm, d_lab, d_mat, d_edges, d_elab, params=p)
        c = ctx.trace(s, d_tx, d_rx, p)
        P = ctx.refine(s, c, p)
        cnt = ctx.counts(P)
        for h in (P, c, s):
            ctx.release(h)
        return cnt

    # launch layouts (result-neutral) tuned on a small sample of the workload, untimed
    s0 = ctx.voxelize(d_xyz, d_nrm, d_lab, d_mat, d_edges, d_elab, params=p)
    tuning = ctx.autotune(s0, sc.tx, sc.rx[:4], p)   # every TX: the level work grows with the TX trees
    ctx.release(s0)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    ms, counts = [], []
    l0 = _abi.kernel_launches()
    wall0 = time.perf_counter()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            counts.append(step())
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    wall = time.perf_counter() - wall0
    launches = _abi.kernel_launches() - l0
    barrier()
    t_total = sum(ms) / 1e3
    cones = sum(c["n_cones"] for c in counts)
    paths = sum(c["n_paths"] for c in counts)
    vis = sum(c["n_vis"] for c in counts)
    if world > 1:
        t_total, cones, paths, vis = reduce_over_ranks(t_total, cones, paths, dev, vis)
    c0 = counts[-1]
    value = cones / t_total
    exact_ps = paths / t_total

    # end to end through the public API from pinned host buffers, results read back;
    # every rank runs it on its own draw (whole-job figure like the value)
    h = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
         dict(xyz=sc.xyz, nrm=sc.nrm, lab=sc.label, mat=sc.material, edges=sc.edges, elab=sc.edge_label,
              tx=sc.tx, rx=sc.rx).items()}
    h2d = sum(int(t.numel() * t.element_size()) for t in h.values())
    e2e_t, e2e_cones, e2e_paths, d2h = [], 0, 0, 0
    barrier()
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = ctx.voxelize(h["xyz"], h["nrm"], h["lab"], h["mat"], h["edges"], h["elab"], params=p)
        c = ctx.trace(s, h["tx"], h["rx"], p)
        P = ctx.refine(s, c, p)
        res = ctx.query(P)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for hh in (P, c, s):
            ctx.release(hh)
        if i >= args.warmup:
            e2e_t.append(dt)
            e2e_cones += res["counts"]["n_cones"]
            e2e_paths += res["counts"]["n_paths"]
            d2h = int(len(res["n"]) * 320 + 8 * 24)
    e2e = None
    if not args.no_e2e:
        t_e2e = sum(e2e_t)
        if world > 1:
            t_e2e, e2e_cones, e2e_paths = reduce_over_ranks(t_e2e, e2e_cones, e2e_paths, dev)
        e2e = {"value": e2e_cones / t_e2e, "unit": "rays/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "exact_paths_per_s": e2e_paths / t_e2e}

    out = None
    if rank == 0:
        # dominant kernel and its roofline (algorithmic bytes / CUDA-event time)
        stages = {"trace_levels": (c0["ms_levels"], c0["bytes_levels"]),
                  "trace_primary": (c0["ms_primary"], c0["bytes_primary"]),
                  "refine": (c0["ms_refine"], c0["bytes_refine"])}
        dom = max(stages, key=lambda k: stages[k][0])
        dms, dbytes = stages[dom]
        pk = peaks()
        peak = pk["hbm_gbs"] if pk else 6400.0
        achieved = dbytes / (dms * 1e-3) / 1e9 if dms > 0 else 0.0
        traffic = None
        if dom == "refine" and REFINE_TRAFFIC["sources_sha256"] == kernel_sources_sha256():
            traffic = REFINE_TRAFFIC["bytes"]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "kernel_ms": dms, "algorithmic_bytes": dbytes,
                "peak_source": "measured" if pk else "fallback",
                "stage_ms": {k: v[0] for k, v in stages.items()} | {"vis_tables": c0["ms_vis"],
                                                                     "kappa": c0["ms_kappa"],
                                                                     "dedup": c0["ms_dedup"]}}

        # plain form: one trace + refine per TX/RX pair on the resident scene
        plain = None
        if args.plain_steps > 0:
            pl_ms, pl_cones, pl_paths, lat = [], 0, 0, []
            for _ in range(args.plain_steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s = ctx.voxelize(d_xyz, d_nrm, d_lab, d_mat, d_edges, d_elab, params=p)
                for ti in range(sc.tx.shape[0]):
                    for ri in range(sc.rx.shape[0]):
                        q0 = time.perf_counter()
                        c = ctx.trace(s, d_tx[ti:ti + 1], d_rx[ri:ri + 1], p)
                        P = ctx.refine(s, c, p)
                        cc = ctx.counts(P)
                        lat.append(time.perf_counter() - q0)
                        pl_cones += cc["n_cones"]
                        pl_paths += cc["n_paths"]
                        ctx.release(P)
                        ctx.release(c)
                ctx.release(s)
                torch.cuda.synchronize()
                pl_ms.append(1e3 * (time.perf_counter() - t0))
            tpl = sum(pl_ms) / 1e3
            # rays_per_s counts the cones the plain form traced (each pair re-traces its TX's
            # launch); workload_rays_per_s is the batched workload's cones over the plain time
            plain = {"rays_per_s": pl_cones / tpl, "workload_rays_per_s": cones / len(counts) / world * args.plain_steps / tpl,
                     "exact_paths_per_s": pl_paths / tpl,
                     "ms_per_step": statistics.mean(pl_ms), "calls_per_step": int(sc.tx.shape[0] * sc.rx.shape[0]),
                     "pair_latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                     "pair_latency_ms_p99": 1e3 * float(np.percentile(lat, 99))}

        latency = None
        if not args.no_serving:
            try:
                from paper_2402_13747_b300 import serve
                latency = serve.bench_latency(ctx, device=local)
            except Exception as ex:  # the serving measurement must not hide the main line
                latency = {"error": repr(ex)}

        # automatic labels and edges of the workload's cloud (nimbus_segment), outside the
        # timed region: median device time of three calls after one warm-up call
        segment = None
        if not args.no_segment:
            try:
                seg_ms = []
                for _ in range(4):
                    G = ctx.segment(sc.xyz, sc.nrm)
                    seg_ms.append(G["counts"]["ms_total"])
                sm = float(np.median(seg_ms[1:]))
                segment = {"cloud": f"the workload's {sc.xyz.shape[0]} points without labels or edges",
                           "ms": sm, "points_per_s": sc.xyz.shape[0] / (sm / 1e3),
                           "surfaces": int(G["counts"]["n_surfaces"]), "edges": int(G["counts"]["n_edges"])}
            except Exception as ex:  # must not hide the main line
                segment = {"error": repr(ex)}

        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline()

        clocks = clk.summary()
        out = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": float(statistics.mean(ms)), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32 traversal / f64 refinement",
               "data": "synthetic",
               "config": {"workload": workload, "l2": "flushed between timed steps (512 MB write)",
                          "points": int(sc.xyz.shape[0]), "pairs": int(sc.tx.shape[0] * sc.rx.shape[0]),
                          "form": "batched: all pairs in one trace_coarse + refine",
                          "tuning": {k: v for k, v in tuning.items() if not k.endswith("_ms")},
                          "tuning_sample": "all TX x 4 RX of the workload"},
               "exact_paths_per_s": exact_ps, "exact_paths_per_step": paths / args.steps / world,
               "visibility_rays_per_s": vis / t_total,
               "cones_per_step": cones / args.steps / world, "wall_s_timed_region": wall,
               "plain": plain, "latency": latency, "segment": segment, "roofline": roof, "cpu_baseline": cpu,
               "e2e": e2e,
               "gpu_launches": launches, "clocks": clocks,
               "counts_last_step": {k: c0[k] for k in ("n_paths", "n_coarse", "n_coarse_raw", "n_nodes", "n_vis",
                                                       "n_cones", "launches")}}
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
