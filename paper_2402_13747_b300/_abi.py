"""ctypes binding of ``libnimbus.so`` (include/nimbus.h): argument marshalling only.

Every step of voxelisation, coarse tracing and refinement runs in the library's
CUDA kernels.  Inputs may be numpy arrays (host) or torch CUDA tensors (device);
the library copies them.  Loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from .config import Params

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnimbus.so")
MAXI = 8
NONE_LABEL = 0xFFFFFFFF

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_OVERFLOW, ERR_TIMEOUT, ERR_STATE, ERR_IO = range(8)
ERR_NAMES = {1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_OVERFLOW", 5: "ERR_TIMEOUT", 6: "ERR_STATE",
             7: "ERR_IO"}

EXPORTS = ("nimbus_create", "nimbus_destroy", "nimbus_last_error", "nimbus_voxelize", "nimbus_update_region",
           "nimbus_trace_coarse", "nimbus_refine", "nimbus_query", "nimbus_query_coarse", "nimbus_scene_info",
           "nimbus_scene_tables", "nimbus_release", "nimbus_memory_used", "nimbus_kernel_launches",
           "nimbus_device_allocations", "nimbus_voxelize_static", "nimbus_get_tuning", "nimbus_set_tuning", "nimbus_autotune",
           "nimbus_scene_save", "nimbus_scene_load", "nimbus_segment", "nimbus_set_wait_limit")

_vp = C.c_void_p


class Cloud(C.Structure):
    _fields_ = [("xyz", _vp), ("nrm", _vp), ("label", _vp), ("material", _vp), ("n", C.c_int64)]


class Edges(C.Structure):
    _fields_ = [("edges", _vp), ("label", _vp), ("n", C.c_int64)]


class VoxParams(C.Structure):
    _fields_ = [("voxel_size", C.c_double), ("sdf_sigma", C.c_double), ("sdf_eps", C.c_double),
                ("vis_ignore", C.c_double), ("region_min", C.c_double * 3), ("region_max", C.c_double * 3),
                ("has_region", C.c_int32), ("dv", C.c_int32), ("sdf_max_steps", C.c_int32), ("pad_", C.c_int32)]


class TraceParams(C.Structure):
    _fields_ = [("cone_half_angle", C.c_double), ("launch_spacing", C.c_double), ("sep_eps", C.c_double),
                ("n_launch", C.c_int32), ("max_refl", C.c_int32), ("max_diff", C.c_int32),
                ("max_int", C.c_int32), ("kappa", C.c_int32), ("launch_mode", C.c_int32),
                ("max_nodes", C.c_int64), ("max_coarse", C.c_int64), ("rx_owner", _vp), ("rx_max_int", _vp)]


class RefineParams(C.Structure):
    _fields_ = [("delta", C.c_double), ("gamma", C.c_double), ("grad_stop", C.c_double),
                ("freq_hz", C.c_double), ("rho", C.c_int32), ("pad_", C.c_int32)]


class Counts(C.Structure):
    _fields_ = ([(n, C.c_int64) for n in ("n_paths", "n_refined", "n_refined_valid", "n_coarse", "n_coarse_raw",
                                          "n_cones", "n_vis", "n_nodes", "needed_nodes", "needed_coarse",
                                          "bytes_read")] +
                [("overflow", C.c_int32), ("n_levels", C.c_int32)] +
                [(n, C.c_double) for n in ("ms_vis", "ms_primary", "ms_levels", "ms_kappa", "ms_refine",
                                           "ms_dedup")] +
                [(n, C.c_int64) for n in ("bytes_primary", "bytes_levels", "bytes_refine", "launches",
                                          "n_cones_no_rx")])

    def as_dict(self):
        return {f[0]: (float if f[1] is C.c_double else int)(getattr(self, f[0])) for f in self._fields_}


class PathView(C.Structure):
    _fields_ = [(n, _vp) for n in ("tx", "rx", "n_int", "types", "labels", "materials", "ies", "points",
                                   "length", "delay", "grad", "iters", "status")]


class CoarseView(C.Structure):
    _fields_ = [(n, _vp) for n in ("tx", "rx", "n_int", "ies", "types", "labels", "miss")]


class SceneView(C.Structure):
    _fields_ = [(n, _vp) for n in ("kind", "label", "cell", "gs", "prange", "rp", "normal", "bbc", "material",
                                   "cell_begin", "cell_count", "march", "slab")]


class StaticTables(C.Structure):
    _fields_ = [("kind", _vp), ("label", _vp), ("gs", _vp), ("pcount", _vp), ("rp", _vp), ("normal", _vp),
                ("bbc", _vp), ("material", _vp), ("ie_capacity", C.c_int64), ("cell_begin", _vp),
                ("cell_count", _vp), ("march", _vp), ("cell_capacity", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("level_block", C.c_int32), ("refine_blocks", C.c_int32), ("refine_order", C.c_int32),
                ("graph", C.c_int32), ("level_ms", C.c_double), ("refine_ms", C.c_double),
                ("level_queue", C.c_int32), ("refine_split", C.c_int32), ("refine_split_key", C.c_int32),
                ("level_help", C.c_int32), ("level_rx_first", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class StaticInfo(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("dims", C.c_int32 * 3), ("pad_", C.c_int32), ("n_ie", C.c_int64),
                ("n_cells", C.c_int64)]


class SegmentParamsC(C.Structure):
    _fields_ = [("voxel_size", C.c_double), ("flat_max", C.c_double), ("spread_min", C.c_double),
                ("join_angle", C.c_double), ("join_dist", C.c_double), ("edge_angle", C.c_double),
                ("dv", C.c_int32), ("min_points", C.c_int32), ("edge_min_groups", C.c_int32), ("pad_", C.c_int32)]


class SegmentCounts(C.Structure):
    _fields_ = [("n_groups", C.c_int64), ("n_planar", C.c_int64), ("n_surfaces", C.c_int64), ("n_edges", C.c_int64),
                ("ms", C.c_double), ("ms_total", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def segment_params(sp) -> SegmentParamsC:
    """config.SegmentParams -> the C parameter block (angles in radians)."""
    import math
    return SegmentParamsC(float(sp.voxel_size), float(sp.flat_max), float(sp.spread_min),
                          math.radians(sp.join_angle_deg), float(sp.join_dist), math.radians(sp.edge_angle_deg),
                          int(sp.dv), int(sp.min_points), int(sp.edge_min_groups), 0)


STATIC_MAX_POINTS = 1 << 17
STATIC_MAX_CELLS = 1 << 20


class NimbusError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    v = C.c_int64(0)
    load().nimbus_kernel_launches(C.byref(v))
    return int(v.value)


def device_allocations() -> int:
    """Device allocations the library has made in this process so far."""
    v = C.c_int64(0)
    load().nimbus_device_allocations(C.byref(v))
    return int(v.value)


def load():
    """Load libnimbus.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2402_13747_b300.build`")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    ctxp = _vp
    L.nimbus_create.argtypes = [P(ctxp), C.c_int, C.c_size_t]
    L.nimbus_destroy.argtypes = [ctxp]
    L.nimbus_last_error.restype = C.c_char_p
    L.nimbus_last_error.argtypes = [ctxp]
    L.nimbus_voxelize.argtypes = [ctxp, P(Cloud), P(Edges), P(VoxParams), P(C.c_uint64), _vp]
    L.nimbus_update_region.argtypes = [ctxp, C.c_uint64, P(C.c_double), P(C.c_double), P(Cloud), _vp]
    L.nimbus_trace_coarse.argtypes = [ctxp, C.c_uint64, _vp, C.c_int32, _vp, C.c_int32, P(TraceParams),
                                      P(C.c_uint64), _vp]
    L.nimbus_refine.argtypes = [ctxp, C.c_uint64, C.c_uint64, P(RefineParams), P(C.c_uint64), _vp]
    L.nimbus_query.argtypes = [ctxp, C.c_uint64, C.c_int32, P(Counts), P(PathView), _vp]
    L.nimbus_query_coarse.argtypes = [ctxp, C.c_uint64, P(Counts), P(CoarseView), _vp]
    L.nimbus_scene_info.argtypes = [ctxp, C.c_uint64, P(C.c_double), P(C.c_int32), P(C.c_int64), P(C.c_int64)]
    L.nimbus_scene_tables.argtypes = [ctxp, C.c_uint64, P(SceneView), _vp]
    L.nimbus_release.argtypes = [ctxp, C.c_uint64]
    L.nimbus_memory_used.argtypes = [ctxp, P(C.c_size_t)]
    L.nimbus_kernel_launches.argtypes = [P(C.c_int64)]
    L.nimbus_device_allocations.argtypes = [P(C.c_int64)]
    L.nimbus_voxelize_static.argtypes = [ctxp, P(Cloud), P(VoxParams), P(StaticTables), P(StaticInfo), _vp]
    L.nimbus_scene_save.argtypes = [ctxp, C.c_uint64, C.c_char_p, _vp]
    L.nimbus_scene_load.argtypes = [ctxp, C.c_char_p, P(C.c_uint64), _vp]
    L.nimbus_segment.argtypes = [ctxp, P(Cloud), P(SegmentParamsC), _vp, _vp, _vp, C.c_int64, P(SegmentCounts), _vp]
    L.nimbus_get_tuning.argtypes = [ctxp, P(Tuning)]
    L.nimbus_set_wait_limit.argtypes = [ctxp, C.c_int64]
    L.nimbus_set_tuning.argtypes = [ctxp, P(Tuning)]
    L.nimbus_autotune.argtypes = [ctxp, C.c_uint64, _vp, C.c_int32, _vp, C.c_int32, P(TraceParams), P(RefineParams),
                                  P(Tuning), _vp]
    for name in EXPORTS:
        L[name].restype = C.c_char_p if name == "nimbus_last_error" else C.c_int
    _lib = L
    return L


# ----------------------------------------------------------------------------- params
def vox_params(p: Params, region=None) -> VoxParams:
    v = VoxParams()
    v.voxel_size = p.voxel_size
    v.sdf_sigma = p.sdf_sigma
    v.sdf_eps = p.sdf_eps
    v.vis_ignore = p.ignore_dist
    v.dv = p.dv
    v.sdf_max_steps = p.sdf_max_steps
    if region is not None:
        r = np.asarray(region, np.float64).reshape(2, 3)
        v.has_region = 1
        for a in range(3):
            v.region_min[a] = r[0, a]
            v.region_max[a] = r[1, a]
    return v


def trace_params(p: Params, max_nodes=0, max_coarse=0) -> TraceParams:
    t = TraceParams()
    t.cone_half_angle = math.radians(p.cone_half_angle_deg)
    t.launch_spacing = math.radians(p.launch_spacing_deg)
    t.sep_eps = p.sep_eps
    t.n_launch = p.launch_count
    t.max_refl = p.max_refl
    t.max_diff = p.max_diff
    t.max_int = p.max_interactions
    t.kappa = p.kappa
    t.launch_mode = p.launch_mode
    t.max_nodes = max_nodes
    t.max_coarse = max_coarse
    return t


def refine_params(p: Params) -> RefineParams:
    r = RefineParams()
    r.delta = p.delta
    r.gamma = p.gamma
    r.grad_stop = p.grad_stop
    r.freq_hz = p.freq_hz
    r.rho = p.rho
    return r


# ----------------------------------------------------------------------------- helpers
def _ptr(a):
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    return a.ctypes.data


def _host(a, dt, shape=None):
    if hasattr(a, "data_ptr"):
        return a
    a = np.ascontiguousarray(a, dtype=dt)
    return a.reshape(shape) if shape is not None else a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Context:
    """One library context on one CUDA device with a device-memory budget."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        self.L = load()
        self.h = _vp()
        self._check(self.L.nimbus_create(C.byref(self.h), device, mem_budget), "create")

    def close(self):
        if self.h:
            self.L.nimbus_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != OK:
            msg = self.L.nimbus_last_error(self.h).decode() if self.h else what
            raise NimbusError(rc, f"{what}: {msg}")

    def last_error(self) -> str:
        return self.L.nimbus_last_error(self.h).decode()

    # -- Section 2.1
    def voxelize(self, xyz, nrm, label, material=None, edges=None, edge_label=None, params: Params = None,
                 region=None, stream=None) -> int:
        params = params or Params()
        keep = [_host(xyz, np.float32), _host(nrm, np.float32), _host(label, np.uint32),
                None if material is None else _host(material, np.uint8)]
        n = keep[0].shape[0] if hasattr(keep[0], "shape") else 0
        cl = Cloud(_ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), _ptr(keep[3]), int(n))
        ed = None
        if edges is not None and len(edges) > 0:
            e = _host(edges, np.float64, (-1, 12))
            el = _host(edge_label, np.uint32)
            keep += [e, el]
            ed = Edges(_ptr(e), _ptr(el), int(e.shape[0]))
        vp = vox_params(params, region)
        out = C.c_uint64(0)
        self._check(self.L.nimbus_voxelize(self.h, C.byref(cl), C.byref(ed) if ed else None, C.byref(vp),
                                           C.byref(out), _stream(stream)), "voxelize")
        return out.value

    def segment(self, xyz, nrm, sp=None, edges_cap: int = 1024, stream=None) -> dict:
        """Automatic labels and exterior edges of an unlabelled cloud (nimbus_segment).

        Returns labels [n] (uint32), edges [m, 12], edge_labels [m] and counts; a larger
        edge buffer is taken once when more than edges_cap edges exist."""
        from .config import SegmentParams
        sp = sp or SegmentParams()
        x, nr = _host(xyz, np.float32), _host(nrm, np.float32)
        n = int(x.shape[0])
        cl = Cloud(_ptr(x), _ptr(nr), None, None, n)
        prm = segment_params(sp)
        for _ in range(2):
            labels = np.zeros(n, np.uint32)
            edges = np.zeros((max(edges_cap, 1), 12))
            elab = np.zeros(max(edges_cap, 1), np.uint32)
            cnt = SegmentCounts()
            rc = self.L.nimbus_segment(self.h, C.byref(cl), C.byref(prm), _ptr(labels), _ptr(edges), _ptr(elab),
                                       int(edges_cap), C.byref(cnt), _stream(stream))
            if rc == ERR_OVERFLOW and cnt.n_edges > edges_cap:
                edges_cap = int(cnt.n_edges)
                continue
            self._check(rc, "segment")
            m = int(cnt.n_edges)
            return dict(labels=labels, edges=edges[:m].copy(), edge_labels=elab[:m].copy(), counts=cnt.as_dict())
        self._check(rc, "segment")

    def voxelize_scene(self, sc, params: Params = None, stream=None) -> int:
        return self.voxelize(sc.xyz, sc.nrm, sc.label, sc.material, sc.edges, sc.edge_label, params,
                             region=getattr(sc, "region", None), stream=stream)

    def update_region(self, scene: int, lo, hi, xyz=None, nrm=None, label=None, material=None, stream=None):
        lo = (C.c_double * 3)(*[float(v) for v in lo])
        hi = (C.c_double * 3)(*[float(v) for v in hi])
        cl = None
        keep = []
        if xyz is not None:
            keep = [_host(xyz, np.float32), _host(nrm, np.float32), _host(label, np.uint32),
                    None if material is None else _host(material, np.uint8)]
            cl = Cloud(_ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), _ptr(keep[3]), int(keep[0].shape[0]))
        self._check(self.L.nimbus_update_region(self.h, scene, lo, hi, C.byref(cl) if cl else None,
                                                _stream(stream)), "update_region")

    # -- Section 2.2
    def trace(self, scene: int, tx, rx, params: Params = None, max_nodes=0, max_coarse=0, stream=None,
              allow_overflow=False, rx_owner=None, rx_max_int=None) -> int:
        params = params or Params()
        t = _host(tx, np.float64, (-1, 3))
        r = _host(rx, np.float64, (-1, 3))
        tp = trace_params(params, max_nodes, max_coarse)
        own = None if rx_owner is None else _host(rx_owner, np.int32)
        mx = None if rx_max_int is None else _host(rx_max_int, np.int32)
        tp.rx_owner = _ptr(own)
        tp.rx_max_int = _ptr(mx)
        out = C.c_uint64(0)
        rc = self.L.nimbus_trace_coarse(self.h, scene, _ptr(t), int(t.shape[0]), _ptr(r), int(r.shape[0]),
                                        C.byref(tp), C.byref(out), _stream(stream))
        if rc == ERR_OVERFLOW and allow_overflow:
            return out.value
        self._check(rc, "trace_coarse")
        return out.value

    # -- Section 2.3
    def refine(self, scene: int, coarse: int, params: Params = None, stream=None) -> int:
        params = params or Params()
        rp = refine_params(params)
        out = C.c_uint64(0)
        self._check(self.L.nimbus_refine(self.h, scene, coarse, C.byref(rp), C.byref(out), _stream(stream)),
                    "refine")
        return out.value

    def counts(self, paths: int, which=0, stream=None) -> dict:
        c = Counts()
        self._check(self.L.nimbus_query(self.h, paths, which, C.byref(c), None, _stream(stream)), "query")
        return c.as_dict()

    def query(self, paths: int, which: int = 0, stream=None) -> dict:
        c = Counts()
        self._check(self.L.nimbus_query(self.h, paths, which, C.byref(c), None, _stream(stream)), "query")
        n = c.n_refined if which else c.n_paths
        out = dict(tx=np.zeros(n, np.int32), rx=np.zeros(n, np.int32), n=np.zeros(n, np.int32),
                   type=np.zeros((n, MAXI), np.int32), label=np.zeros((n, MAXI), np.uint32),
                   material=np.zeros((n, MAXI), np.uint8), ie=np.zeros((n, MAXI), np.int64),
                   pts=np.zeros((n, MAXI, 3)), length=np.zeros(n), delay=np.zeros(n), grad=np.zeros(n),
                   iters=np.zeros(n, np.int32), status=np.zeros(n, np.int32))
        v = PathView(*[_ptr(out[k]) for k in ("tx", "rx", "n", "type", "label", "material", "ie", "pts", "length",
                                              "delay", "grad", "iters", "status")])
        self._check(self.L.nimbus_query(self.h, paths, which, C.byref(c), C.byref(v), _stream(stream)), "query")
        out["counts"] = c.as_dict()
        return out

    # -- scene checkpoint
    def scene_save(self, scene: int, path: str, stream=None):
        """Write the scene's current cloud, edges, parameters and grid to `path`."""
        self._check(self.L.nimbus_scene_save(self.h, scene, os.fsencode(path), _stream(stream)), "scene_save")

    def scene_load(self, path: str, stream=None) -> int:
        """A new scene from a checkpoint; its tables equal the saved scene's."""
        out = C.c_uint64(0)
        self._check(self.L.nimbus_scene_load(self.h, os.fsencode(path), C.byref(out), _stream(stream)), "scene_load")
        return out.value

    # -- launch layout (result-neutral)
    def get_tuning(self) -> dict:
        t = Tuning()
        self._check(self.L.nimbus_get_tuning(self.h, C.byref(t)), "get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw) -> dict:
        t = Tuning()
        self._check(self.L.nimbus_get_tuning(self.h, C.byref(t)), "get_tuning")
        for k, v in kw.items():
            setattr(t, k, v)
        self._check(self.L.nimbus_set_tuning(self.h, C.byref(t)), "set_tuning")
        return t.as_dict()

    def set_wait_limit(self, cycles: int):
        """Limit, in SM cycles, of the propagation levels' bounded waits (0: defaults);
        for tests of the timeout path (nimbus_set_wait_limit)."""
        self._check(self.L.nimbus_set_wait_limit(self.h, int(cycles)), "set_wait_limit")

    def autotune(self, scene: int, tx, rx, params: Params = None, stream=None) -> dict:
        """Time the launch layouts on a TX/RX sample and keep the fastest (nimbus_autotune)."""
        params = params or Params()
        t = _host(tx, np.float64, (-1, 3))
        r = _host(rx, np.float64, (-1, 3))
        tp, rp, out = trace_params(params), refine_params(params), Tuning()
        self._check(self.L.nimbus_autotune(self.h, scene, _ptr(t), int(t.shape[0]), _ptr(r), int(r.shape[0]),
                                           C.byref(tp), C.byref(rp), C.byref(out), _stream(stream)), "autotune")
        return out.as_dict()

    def coarse_counts(self, coarse: int, stream=None) -> dict:
        """Sizes and counters of a coarse set (no path arrays copied)."""
        c = Counts()
        self._check(self.L.nimbus_query_coarse(self.h, coarse, C.byref(c), None, _stream(stream)), "query_coarse")
        return c.as_dict()

    def query_coarse(self, coarse: int, stream=None) -> dict:
        c = Counts()
        self._check(self.L.nimbus_query_coarse(self.h, coarse, C.byref(c), None, _stream(stream)), "query_coarse")
        n = c.n_coarse
        out = dict(tx=np.zeros(n, np.int32), rx=np.zeros(n, np.int32), n=np.zeros(n, np.int32),
                   ie=np.zeros((n, MAXI), np.int64), type=np.zeros((n, MAXI), np.int32),
                   label=np.zeros((n, MAXI), np.uint32), miss=np.zeros(n, np.float32))
        v = CoarseView(*[_ptr(out[k]) for k in ("tx", "rx", "n", "ie", "type", "label", "miss")])
        self._check(self.L.nimbus_query_coarse(self.h, coarse, C.byref(c), C.byref(v), _stream(stream)),
                    "query_coarse")
        out["counts"] = c.as_dict()
        return out

    def scene_info(self, scene: int) -> dict:
        o = (C.c_double * 3)()
        d = (C.c_int32 * 3)()
        ni = C.c_int64()
        npt = C.c_int64()
        self._check(self.L.nimbus_scene_info(self.h, scene, o, d, C.byref(ni), C.byref(npt)), "scene_info")
        return dict(origin=np.array(o[:]), dims=np.array(d[:], np.int32), n_ie=ni.value, n_points=npt.value)

    def scene_tables(self, scene: int, stream=None) -> dict:
        info = self.scene_info(scene)
        n = info["n_ie"]
        nc = int(np.prod(info["dims"].astype(np.int64)))
        out = dict(kind=np.zeros(n, np.int32), label=np.zeros(n, np.uint32), cell=np.zeros(n, np.int64),
                   gs=np.zeros((n, 3), np.int32), prange=np.zeros((n, 2), np.int64), rp=np.zeros((n, 3), np.float32),
                   normal=np.zeros((n, 3), np.float32), bbc=np.zeros((n, 3), np.float32),
                   material=np.zeros(n, np.uint8), cell_begin=np.zeros(nc, np.int64),
                   cell_count=np.zeros(nc, np.int32), march=np.zeros(nc, np.int32),
                   slab=np.zeros((n, 4), np.float32))
        v = SceneView(*[_ptr(out[k]) for k in ("kind", "label", "cell", "gs", "prange", "rp", "normal", "bbc",
                                               "material", "cell_begin", "cell_count", "march", "slab")])
        self._check(self.L.nimbus_scene_tables(self.h, scene, C.byref(v), _stream(stream)), "scene_tables")
        out.update(info)
        return out

    def voxelize_static(self, xyz, nrm, label, out: dict, material=None, params: Params = None, region=None,
                        stream=None, allow_overflow=False) -> dict:
        """Voxelise into caller-owned device buffers without any device allocation.

        For callers that cannot allocate while they run (device memory carved up in
        advance by another allocator, real-time loops that must not wait on the
        allocator): the inputs must be device tensors
        and ``out`` holds device tensors named as in nimbus_static_tables, sized by
        the capacities ``out['ie_capacity']`` and ``out['cell_capacity']``.
        Calls that overlap on the GPU share one fixed scratch array and race.  The
        call synchronises its stream (it reads counters back), so it cannot run
        inside a CUDA host function or under stream capture.
        """
        params = params or Params()
        cl = Cloud(_ptr(xyz), _ptr(nrm), _ptr(label), _ptr(material), int(xyz.shape[0]))
        t = StaticTables(*[_ptr(out[k]) for k in ("kind", "label", "gs", "pcount", "rp", "normal", "bbc",
                                                  "material")],
                         int(out["ie_capacity"]),
                         *[_ptr(out[k]) for k in ("cell_begin", "cell_count", "march")], int(out["cell_capacity"]))
        vp = vox_params(params, region)
        info = StaticInfo()
        rc = self.L.nimbus_voxelize_static(self.h, C.byref(cl), C.byref(vp), C.byref(t), C.byref(info),
                                           _stream(stream))
        res = dict(origin=np.array(info.origin[:]), dims=np.array(info.dims[:], np.int32), n_ie=info.n_ie,
                   n_cells=info.n_cells, overflow=rc == ERR_OVERFLOW)
        if rc == ERR_OVERFLOW and allow_overflow:
            return res   # the needed sizes; the outputs are untouched
        self._check(rc, "voxelize_static")
        return res

    def release(self, h: int):
        self._check(self.L.nimbus_release(self.h, h), "release")

    def memory_used(self) -> int:
        b = C.c_size_t()
        self._check(self.L.nimbus_memory_used(self.h, C.byref(b)), "memory_used")
        return b.value

    # -- whole pipeline
    def run(self, sc, params: Params = None, stream=None, release=True) -> dict:
        """Voxelise, trace and refine one scene; returns the exact paths (host dict)."""
        params = params or Params(max_refl=sc.max_refl, max_diff=sc.max_diff)
        s = self.voxelize_scene(sc, params, stream)
        c = self.trace(s, sc.tx, sc.rx, params, stream=stream)
        p = self.refine(s, c, params, stream)
        out = self.query(p, 0, stream)
        if release:
            for h in (p, c, s):
                self.release(h)
        return out
