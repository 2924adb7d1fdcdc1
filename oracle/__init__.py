"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It wraps ``nimbus_oracle.cpp`` -- a plain,
slow, single-threaded FP64 implementation of voxelisation (Section 2.1), coarse path
tracing (Section 2.2) and path refinement (Section 2.3) -- through ctypes.  It
shares no code with the CUDA library.

Parity pins (tests/test_oracle_pins.py):
- the image method on the box room, with both transmission phases;
- the LOS length, and the normal-incidence images of an RX placed on the TX;
- the Keller diffraction point on a sampled wedge, and a floor reflection next to that
  diffraction in either order (the floor image of the lower end and its Keller point);
- brute-force visibility and a closed-form plane patch;
- a brute-force chessboard distance for the march field;
- the exact-plane SDF and the continuity of a label's surface;
- a Monte-Carlo cone-sphere test and the Fibonacci lattice properties;
- integer re-derivation of the voxel keys, and the reflection law at refined points;
- the first Fresnel zone radius of the duplicate removal, just inside and just outside;
- Eq. 1's Gaussian weights on two points (a tanh profile), the image-method paths with
  faces turned away, the self-hit rule of the visibility test, the lattice's equal-area
  zones and golden-angle turns, and delay = length / c;
- the depth limits, the LOS miss against the brute-force nearest launch axis, the rho /
  delta validity rule, diffractions refined off their edge, the shortest path per label
  sequence, the image method with an occluding panel, the march's segment of one
  subvoxel diameter, and paths that move with the scene.
- the secant placement after a sign change of f, in an entity's march and in the
  re-projection, on two sheets whose Eq. 1 surface is f = u - h tanh(2uh/sigma^2);
  the final visibility check, which alone removes a path passing 0.0545 m outside a
  panel's border; the RX reception sphere centred on the RX, on one launch cone; the
  re-projection of a target already on the surface (one Newton step from it).
tests/test_oracle_mutants.py plants one mistake at a time in a copy of the source and
checks that these pins catch it.

The coarse-path set and the kappa choice on noisy scenes have no closed form: parity
unpinned beyond those invariants.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nimbus_oracle.cpp")
_LIB = os.path.join(_HERE, "libnimbus_oracle.so")
MAXI = 8
NONE_LABEL = 0xFFFFFFFF
STATUS = {0: "valid", 1: "miss", 2: "not_converged", 3: "occluded", 4: "off_edge"}


class OracleParams(C.Structure):
    _fields_ = [
        ("voxel_size", C.c_double), ("cone_half_angle", C.c_double), ("launch_spacing", C.c_double),
        ("sdf_sigma", C.c_double), ("sdf_eps", C.c_double), ("vis_ignore", C.c_double),
        ("sep_eps", C.c_double), ("delta", C.c_double), ("gamma", C.c_double),
        ("grad_stop", C.c_double), ("freq_hz", C.c_double),
        ("dv", C.c_int32), ("max_refl", C.c_int32), ("max_diff", C.c_int32), ("max_int", C.c_int32),
        ("kappa", C.c_int32), ("n_launch", C.c_int32), ("sdf_max_steps", C.c_int32), ("rho", C.c_int32),
        ("launch_mode", C.c_int32),
    ]


def to_struct(p) -> OracleParams:
    """Any object with the configuration attributes -> the oracle's parameter block."""
    s = OracleParams()
    s.voxel_size = p.voxel_size
    s.cone_half_angle = math.radians(p.cone_half_angle_deg)
    s.launch_spacing = math.radians(p.launch_spacing_deg)
    s.sdf_sigma = p.sdf_sigma
    s.sdf_eps = p.sdf_eps
    s.vis_ignore = p.ignore_dist
    s.sep_eps = p.sep_eps
    s.delta = p.delta
    s.gamma = p.gamma
    s.grad_stop = p.grad_stop
    s.freq_hz = p.freq_hz
    s.dv = p.dv
    s.max_refl = p.max_refl
    s.max_diff = p.max_diff
    s.max_int = p.max_interactions
    s.kappa = p.kappa
    s.n_launch = p.launch_count
    s.sdf_max_steps = p.sdf_max_steps
    s.rho = p.rho
    s.launch_mode = getattr(p, "launch_mode", 0)
    return s


def build_from(src: str, out: str) -> str:
    """Compile an oracle source with g++ (no FP contraction: FP32 binning must be exact)."""
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", src, "-o", out]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libnimbus_oracle.so when its source is newer."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        build_from(_SRC, _LIB)
    return _LIB


_lib = None


def lib():
    """The loaded oracle library.  NIMBUS_ORACLE_LIB names another build of this same
    interface instead: the mutation tests plant one mistake in a copy of the source,
    build it with build_from() and run the pins against it."""
    global _lib
    if _lib is None:
        path = os.environ.get("NIMBUS_ORACLE_LIB") or build()
        L = C.CDLL(path)
        vp, i64, i32, u32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32, C.c_double
        P = C.POINTER
        L.oracle_voxelize.restype = vp
        L.oracle_voxelize.argtypes = [vp, vp, vp, vp, i64, vp, vp, i64, vp, P(OracleParams)]
        L.oracle_scene_free.argtypes = [vp]
        L.oracle_scene_info.restype = i64
        L.oracle_scene_info.argtypes = [vp, vp, vp, vp]
        L.oracle_scene_ies.argtypes = [vp] * 13
        L.oracle_scene_cells.argtypes = [vp, vp, vp, vp]
        L.oracle_scene_points.argtypes = [vp, vp, vp]
        L.oracle_trace.restype = vp
        L.oracle_trace.argtypes = [vp, vp, i32, vp, i32]
        L.oracle_coarse_free.argtypes = [vp]
        L.oracle_coarse_stats.argtypes = [vp, vp, i32]
        L.oracle_coarse_get.argtypes = [vp] * 8
        L.oracle_refine.restype = vp
        L.oracle_refine.argtypes = [vp, vp]
        L.oracle_exact_free.argtypes = [vp]
        L.oracle_refine_given.argtypes = [vp, vp, i32, vp, i32, i64] + [vp] * 11
        L.oracle_exact_count.restype = i64
        L.oracle_exact_count.argtypes = [vp, i32]
        L.oracle_exact_get.argtypes = [vp, i32] + [vp] * 14
        L.oracle_sdf.restype = i32
        L.oracle_sdf.argtypes = [vp, i64, vp, vp, vp]
        L.oracle_sdf_label.restype = i32
        L.oracle_sdf_label.argtypes = [vp, u32, vp, vp, vp]
        L.oracle_sdf_hit.restype = i32
        L.oracle_sdf_hit.argtypes = [vp, i64, vp, vp, vp]
        L.oracle_reproject.restype = i32
        L.oracle_reproject.argtypes = [vp, vp, vp, u32, vp, vp]
        L.oracle_visible.restype = i32
        L.oracle_visible.argtypes = [vp, vp, vp, i32, u32, i32, u32, i32]
        L.oracle_cone_sphere.restype = i32
        L.oracle_cone_sphere.argtypes = [vp, vp, d, vp, d]
        L.oracle_fibonacci.argtypes = [i64, vp]
        L.oracle_onb.argtypes = [vp, vp, vp]
        L.oracle_dda_cells.restype = i64
        L.oracle_dda_cells.argtypes = [vp, vp, vp, vp, i64]
        L.oracle_fresnel_dedup.restype = i64
        L.oracle_fresnel_dedup.argtypes = [i64] + [vp] * 8 + [i32, d, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Scene:
    """Oracle voxelisation of a labelled point cloud (Section 2.1)."""

    def __init__(self, xyz, nrm, label, material, edges, edge_label, params, region=None):
        L = lib()
        self._keep = [_c(xyz, np.float32), _c(nrm, np.float32), _c(label, np.uint32),
                      _c(material, np.uint8), _c(np.asarray(edges).reshape(-1, 12), np.float64),
                      _c(edge_label, np.uint32)]
        self.params = params
        self._ps = to_struct(params)
        x, n, l, m, e, el = self._keep
        self._region = None if region is None else _c(np.asarray(region).reshape(6), np.float64)
        self.h = L.oracle_voxelize(_p(x), _p(n), _p(l), _p(m), x.shape[0], _p(e), _p(el), e.shape[0],
                                   None if self._region is None else _p(self._region), C.byref(self._ps))
        origin = np.zeros(3, np.float64)
        dims = np.zeros(3, np.int32)
        npg = np.zeros(1, np.int64)
        self.n_ie = int(L.oracle_scene_info(self.h, _p(origin), _p(dims), _p(npg)))
        self.origin, self.dims = origin, dims
        self.n_points_grouped = int(npg[0])

    @classmethod
    def from_scene(cls, sc, params):
        return cls(sc.xyz, sc.nrm, sc.label, sc.material, sc.edges, sc.edge_label, params,
                   region=getattr(sc, "region", None))

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_scene_free(self.h)
            self.h = None

    def ies(self) -> dict:
        n = self.n_ie
        out = dict(kind=np.zeros(n, np.int32), label=np.zeros(n, np.uint32), cell=np.zeros(n, np.int64),
                   gs=np.zeros((n, 3), np.int32), prange=np.zeros((n, 2), np.int64),
                   rp=np.zeros((n, 3)), normal=np.zeros((n, 3)), bbc=np.zeros((n, 3)), sc=np.zeros((n, 3)),
                   edge=np.zeros(n, np.int32), trange=np.zeros((n, 2)), material=np.zeros(n, np.uint8))
        lib().oracle_scene_ies(self.h, *[_p(out[k]) for k in ("kind", "label", "cell", "gs", "prange", "rp",
                                                               "normal", "bbc", "sc", "edge", "trange",
                                                               "material")])
        return out

    def points(self):
        """(positions, normals) of the points in the grouped order of the IE point ranges."""
        xyz = np.zeros((self.n_points_grouped, 3))
        nrm = np.zeros((self.n_points_grouped, 3))
        lib().oracle_scene_points(self.h, _p(xyz), _p(nrm))
        return xyz, nrm

    def cells(self) -> dict:
        nc = int(np.prod(self.dims.astype(np.int64)))
        out = dict(begin=np.zeros(nc, np.int64), count=np.zeros(nc, np.int32), march=np.zeros(nc, np.int32))
        lib().oracle_scene_cells(self.h, _p(out["begin"]), _p(out["count"]), _p(out["march"]))
        return out

    def trace(self, tx, rx) -> "Coarse":
        tx = _c(np.asarray(tx).reshape(-1, 3), np.float64)
        rx = _c(np.asarray(rx).reshape(-1, 3), np.float64)
        h = lib().oracle_trace(self.h, _p(tx), tx.shape[0], _p(rx), rx.shape[0])
        if not h:
            raise ValueError("a TX or RX lies outside the voxel grid")
        return Coarse(h, self)

    def refine(self, coarse: "Coarse") -> "Exact":
        return Exact(lib().oracle_refine(self.h, coarse.h), coarse)

    def refine_given(self, tx, rx, paths: dict) -> dict:
        """Refine the given coarse paths one by one (tx, rx, n, ie, type, label arrays)."""
        tx = _c(np.asarray(tx).reshape(-1, 3), np.float64)
        rx = _c(np.asarray(rx).reshape(-1, 3), np.float64)
        m = len(paths["n"])
        a = {k: _c(paths[k], dt) for k, dt in (("tx", np.int32), ("rx", np.int32), ("n", np.int32),
                                                ("ie", np.int64), ("type", np.int32), ("label", np.uint32))}
        out = dict(status=np.zeros(m, np.int32), iters=np.zeros(m, np.int32), grad=np.zeros(m),
                   pts=np.zeros((m, MAXI, 3)), length=np.zeros(m))
        lib().oracle_refine_given(self.h, _p(tx), tx.shape[0], _p(rx), rx.shape[0], m, _p(a["tx"]), _p(a["rx"]),
                                  _p(a["n"]), _p(a["ie"]), _p(a["type"]), _p(a["label"]), _p(out["status"]),
                                  _p(out["iters"]), _p(out["grad"]), _p(out["pts"]), _p(out["length"]))
        return out

    # building blocks for pins
    def sdf(self, ie, x):
        f = np.zeros(1)
        n = np.zeros(3)
        ok = lib().oracle_sdf(self.h, int(ie), _p(_c(x, np.float64)), _p(f), _p(n))
        return (float(f[0]), n) if ok else (None, None)

    def sdf_label(self, label, x):
        """Eq. 1 on the nearby points of one label (the refinement's surface)."""
        f = np.zeros(1)
        n = np.zeros(3)
        ok = lib().oracle_sdf_label(self.h, int(label), _p(_c(x, np.float64)), _p(f), _p(n))
        return (float(f[0]), n) if ok else (None, None)

    def sdf_hit(self, ie, P, d):
        t = np.zeros(1)
        ok = lib().oracle_sdf_hit(self.h, int(ie), _p(_c(P, np.float64)), _p(_c(d, np.float64)), _p(t))
        return float(t[0]) if ok else None

    def reproject(self, P, R, label):
        """Section 2.3's re-projection alone: the ray from P toward R on the surface of
        `label`; (new point, normal), or (None, None) on a miss."""
        c = np.zeros(3)
        n = np.zeros(3)
        ok = lib().oracle_reproject(self.h, _p(_c(P, np.float64)), _p(_c(R, np.float64)), int(label), _p(c), _p(n))
        return (c, n) if ok else (None, None)

    def visible(self, a, b, mode_a=0, label_a=NONE_LABEL, mode_b=0, label_b=NONE_LABEL, brute=False):
        return bool(lib().oracle_visible(self.h, _p(_c(a, np.float64)), _p(_c(b, np.float64)), mode_a,
                                         label_a, mode_b, label_b, 1 if brute else 0))

    def dda_cells(self, a, b, cap=4096):
        out = np.zeros(cap, np.int64)
        k = lib().oracle_dda_cells(self.h, _p(_c(a, np.float64)), _p(_c(b, np.float64)), _p(out), cap)
        return out[:min(k, cap)]


class Coarse:
    def __init__(self, h, scene):
        self.h = h
        self.scene = scene
        st = np.zeros(32, np.int64)
        lib().oracle_coarse_stats(h, _p(st), 32)
        self.stats = dict(n_paths=int(st[0]), n_before_kappa=int(st[1]), n_cones=int(st[2]),
                          n_vis=int(st[3]), n_evals=int(st[4]),
                          nodes_per_level=[int(x) for x in st[6:6 + int(st[5])]])

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_coarse_free(self.h)
            self.h = None

    def paths(self) -> dict:
        n = self.stats["n_paths"]
        out = dict(tx=np.zeros(n, np.int32), rx=np.zeros(n, np.int32), n=np.zeros(n, np.int32),
                   ie=np.zeros((n, MAXI), np.int64), type=np.zeros((n, MAXI), np.int32),
                   label=np.zeros((n, MAXI), np.uint32), miss=np.zeros(n))
        lib().oracle_coarse_get(self.h, *[_p(out[k]) for k in ("tx", "rx", "n", "ie", "type", "label", "miss")])
        return out


class Exact:
    def __init__(self, h, coarse):
        self.h = h
        self.coarse = coarse

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_exact_free(self.h)
            self.h = None

    def paths(self, all_refined: bool = False) -> dict:
        w = 1 if all_refined else 0
        n = int(lib().oracle_exact_count(self.h, w))
        out = dict(tx=np.zeros(n, np.int32), rx=np.zeros(n, np.int32), n=np.zeros(n, np.int32),
                   type=np.zeros((n, MAXI), np.int32), label=np.zeros((n, MAXI), np.uint32),
                   material=np.zeros((n, MAXI), np.uint8), ie=np.zeros((n, MAXI), np.int64),
                   pts=np.zeros((n, MAXI, 3)), length=np.zeros(n), delay=np.zeros(n), grad=np.zeros(n),
                   iters=np.zeros(n, np.int32), status=np.zeros(n, np.int32), coarse=np.zeros(n, np.int64))
        lib().oracle_exact_get(self.h, w, *[_p(out[k]) for k in (
            "tx", "rx", "n", "type", "label", "material", "ie", "pts", "length", "delay", "grad", "iters",
            "status", "coarse")])
        return out


def cone_sphere(apex, axis, half_angle, c, r) -> bool:
    return bool(lib().oracle_cone_sphere(_p(_c(apex, np.float64)), _p(_c(axis, np.float64)), float(half_angle),
                                         _p(_c(c, np.float64)), float(r)))


def fibonacci(n: int) -> np.ndarray:
    out = np.zeros((n, 3))
    lib().oracle_fibonacci(n, _p(out))
    return out


def onb(n):
    u = np.zeros(3)
    v = np.zeros(3)
    lib().oracle_onb(_p(_c(n, np.float64)), _p(u), _p(v))
    return u, v


def fresnel_dedup(paths: dict, tx_pos, lam: float) -> np.ndarray:
    """First-Fresnel-zone duplicate removal alone (Section 2.3) on given exact paths
    (tx, rx, n, type, label, pts, length as returned by paths()); 1 = kept."""
    m = len(paths["n"])
    arrs = [_c(paths["tx"], np.int32), _c(paths["rx"], np.int32), _c(paths["n"], np.int32),
            _c(paths["type"], np.int32).reshape(m, MAXI), _c(paths["label"], np.uint32).reshape(m, MAXI),
            _c(paths["pts"], np.float64).reshape(m, MAXI, 3), _c(paths["length"], np.float64)]
    txp = _c(tx_pos, np.float64).reshape(-1, 3)
    keep = np.zeros(m, np.int32)
    lib().oracle_fresnel_dedup(m, *[_p(a) for a in arrs], _p(txp), int(txp.shape[0]), float(lam), _p(keep))
    return keep


def run(scene, params):
    """Voxelise, trace and refine one scene; returns (oracle Scene, Coarse, Exact)."""
    s = Scene.from_scene(scene, params)
    c = s.trace(scene.tx, scene.rx)
    e = s.refine(c)
    return s, c, e


def path_key(types, labels, n):
    """(type, label) sequence of one path as a hashable tuple."""
    return tuple((int(types[q]), int(labels[q])) for q in range(int(n)))
