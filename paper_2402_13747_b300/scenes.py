"""Seeded synthetic scenes: labelled point clouds, diffraction edges, TX/RX sets.

This module only *samples geometry*.  It holds none of the method's arithmetic
(no voxelisation, tracing or refinement), so both the CUDA path and the FP64
oracle may take their inputs from it.

A labelled point cloud is the simulator's input (Section 2): each point has a
position, a normal and a label, where a label is one segmented surface.  Edges
for diffraction are inserted by hand (Section 2), each with the outward normals
of its two faces so that only exterior edges are diffracted (Section 3.2).

The paper's corridor cloud (2,745,513 points, Section 3.1) is not available, so
these seeded scenes stand in for it:

* ``room_tiny``   — 10x10x3 m box room, 6 exact planes on a 10 cm lattice.
* ``room_noisy``  — the same room at 5 cm with 5 mm position noise, 2 degree
  normal tilt and a 1x1x2 m box obstacle with 8 exterior edges.
* ``indoor``      — 3x2 grid of 8x7x3 m rooms, doorways, 40 furniture boxes.
* ``street``      — 200x50 m street canyon with two rows of box buildings.
* ``wedge``       — a sampled 90 degree convex corner with its edge (diffraction).
* ``serving_requests`` — a Poisson request stream over resident scenes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Scene", "room_tiny", "room_noisy", "indoor", "street", "wedge", "plane_patch",
    "serving_requests", "moving_box", "merge_clouds",
]


@dataclass
class Scene:
    """A labelled point cloud plus edges and transmitter/receiver positions.

    Layout (all C-contiguous):
      xyz      (N,3) float32  point positions [m]
      nrm      (N,3) float32  unit normals
      label    (N,)  uint32   surface id (segmentation cluster)
      material (N,)  uint8    material id carried to the output
      edges    (E,12) float64 p0(3) p1(3) n_face0(3) n_face1(3), outward normals
      edge_label (E,) uint32  label of each edge
      tx (T,3) float64, rx (R,3) float64
      region  optional (2,3) float64 box [min; max] the voxel grid must also cover
              (transmitters and receivers must lie inside the grid)
    """

    name: str
    xyz: np.ndarray
    nrm: np.ndarray
    label: np.ndarray
    material: np.ndarray
    edges: np.ndarray = field(default_factory=lambda: np.zeros((0, 12), np.float64))
    edge_label: np.ndarray = field(default_factory=lambda: np.zeros((0,), np.uint32))
    tx: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.float64))
    rx: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.float64))
    max_refl: int = 2
    max_diff: int = 0
    meta: dict = field(default_factory=dict)
    region: np.ndarray | None = None   # optional (2,3) box the voxel grid must also cover

    @property
    def n_points(self) -> int:
        return int(self.xyz.shape[0])

    def with_pairs(self, tx, rx) -> "Scene":
        return Scene(self.name, self.xyz, self.nrm, self.label, self.material, self.edges,
                     self.edge_label, np.ascontiguousarray(np.asarray(tx, np.float64).reshape(-1, 3)),
                     np.ascontiguousarray(np.asarray(rx, np.float64).reshape(-1, 3)),
                     self.max_refl, self.max_diff, dict(self.meta), self.region)


# --------------------------------------------------------------------------- sampling helpers

def plane_patch(origin, u, v, len_u, len_v, spacing, normal, label, material=0, hole=None):
    """Square lattice on the rectangle origin + a*u + b*v, a in [0,len_u], b in [0,len_v].

    Lattice nodes are a = i*spacing (i = 0..round(len_u/spacing)), likewise b, so the
    rectangle's border rows are included.  ``hole`` = (a0, a1, b0, b1) removes the
    nodes with a0 < a < a1 and b0 <= b < b1 (a doorway cut into a wall).
    """
    origin = np.asarray(origin, np.float64)
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    nu = int(round(len_u / spacing))
    nv = int(round(len_v / spacing))
    a = np.arange(nu + 1, dtype=np.float64) * (len_u / nu)
    b = np.arange(nv + 1, dtype=np.float64) * (len_v / nv)
    A, B = np.meshgrid(a, b, indexing="ij")
    A = A.ravel()
    B = B.ravel()
    if hole is not None:
        a0, a1, b0, b1 = hole
        keep = ~((A > a0) & (A < a1) & (B >= b0) & (B < b1))
        A, B = A[keep], B[keep]
    pts = origin[None, :] + A[:, None] * u[None, :] + B[:, None] * v[None, :]
    n = np.broadcast_to(np.asarray(normal, np.float64), pts.shape)
    lab = np.full(pts.shape[0], label, np.uint32)
    mat = np.full(pts.shape[0], material, np.uint8)
    return pts, np.array(n), lab, mat


def merge_clouds(parts):
    xyz = np.concatenate([p[0] for p in parts]).astype(np.float32)
    nrm = np.concatenate([p[1] for p in parts]).astype(np.float32)
    lab = np.concatenate([p[2] for p in parts]).astype(np.uint32)
    mat = np.concatenate([p[3] for p in parts]).astype(np.uint8)
    return (np.ascontiguousarray(xyz), np.ascontiguousarray(nrm), np.ascontiguousarray(lab),
            np.ascontiguousarray(mat))


def _box_room_parts(L, W, H, spacing, labels, materials, floor_hole_fn=None):
    """Six inward-facing faces of the axis-aligned room [0,L]x[0,W]x[0,H]."""
    X, Y, Z = np.eye(3)
    parts = [
        plane_patch([0, 0, 0], X, Y, L, W, spacing, [0, 0, 1], labels[4], materials[4]),   # floor
        plane_patch([0, 0, H], X, Y, L, W, spacing, [0, 0, -1], labels[5], materials[5]),  # ceiling
        plane_patch([0, 0, 0], Y, Z, W, H, spacing, [1, 0, 0], labels[0], materials[0]),   # x = 0
        plane_patch([L, 0, 0], Y, Z, W, H, spacing, [-1, 0, 0], labels[1], materials[1]),  # x = L
        plane_patch([0, 0, 0], X, Z, L, H, spacing, [0, 1, 0], labels[2], materials[2]),   # y = 0
        plane_patch([0, W, 0], X, Z, L, H, spacing, [0, -1, 0], labels[3], materials[3]),  # y = W
    ]
    if floor_hole_fn is not None:
        p = parts[0]
        keep = floor_hole_fn(p[0])
        parts[0] = (p[0][keep], p[1][keep], p[2][keep], p[3][keep])
    return parts


def _box_parts(lo, hi, spacing, label0, material):
    """Four side faces and the top of a closed box standing on z = lo[2] (outward normals).

    Labels: x-min side, x-max side, y-min side, y-max side, top = label0 .. label0+4.
    """
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    ext = hi - lo
    X, Y, Z = np.eye(3)
    return [
        plane_patch([lo[0], lo[1], lo[2]], Y, Z, ext[1], ext[2], spacing, [-1, 0, 0], label0 + 0, material),
        plane_patch([hi[0], lo[1], lo[2]], Y, Z, ext[1], ext[2], spacing, [1, 0, 0], label0 + 1, material),
        plane_patch([lo[0], lo[1], lo[2]], X, Z, ext[0], ext[2], spacing, [0, -1, 0], label0 + 2, material),
        plane_patch([lo[0], hi[1], lo[2]], X, Z, ext[0], ext[2], spacing, [0, 1, 0], label0 + 3, material),
        plane_patch([lo[0], lo[1], hi[2]], X, Y, ext[0], ext[1], spacing, [0, 0, 1], label0 + 4, material),
    ]


def _box_edges(lo, hi, label0):
    """The 8 exterior edges of a box standing on the floor: 4 vertical + 4 top.

    The 4 floor-contact edges are concave (box against floor) and are left out.
    Each row: p0, p1, outward normal of face 0, outward normal of face 1.
    """
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    mx, px, my, py, pz = [-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, 1]
    rows = [
        ([x0, y0, z0], [x0, y0, z1], mx, my),
        ([x1, y0, z0], [x1, y0, z1], px, my),
        ([x0, y1, z0], [x0, y1, z1], mx, py),
        ([x1, y1, z0], [x1, y1, z1], px, py),
        ([x0, y0, z1], [x1, y0, z1], my, pz),
        ([x0, y1, z1], [x1, y1, z1], py, pz),
        ([x0, y0, z1], [x0, y1, z1], mx, pz),
        ([x1, y0, z1], [x1, y1, z1], px, pz),
    ]
    e = np.array([np.concatenate([np.asarray(a, float) for a in r]) for r in rows], np.float64)
    lab = np.arange(label0, label0 + 8, dtype=np.uint32)
    return e, lab


def _perturb(xyz, nrm, rng, pos_sigma, nrm_sigma_deg):
    """Gaussian position noise and a Gaussian tilt of each normal (renormalised)."""
    xyz = xyz + rng.normal(0.0, pos_sigma, size=xyz.shape)
    if nrm_sigma_deg > 0:
        s = math.radians(nrm_sigma_deg)
        n = nrm.astype(np.float64)
        g = rng.normal(0.0, s, size=n.shape)
        g -= (g * n).sum(1, keepdims=True) * n      # tilt within the tangent plane
        n = n + g
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        nrm = n
    return xyz, nrm


def _uniform_points(rng, n, lo, hi, reject=None):
    out = []
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    while len(out) < n:
        p = lo + (hi - lo) * rng.random(3)
        if reject is not None and reject(p):
            continue
        out.append(p)
    return np.array(out, np.float64)


# --------------------------------------------------------------------------- scenes

def room_tiny() -> Scene:
    """10x10x3 m box room, 6 planar surfaces on a 10 cm lattice (~32.9k points).

    Exact unit normals, labels 0..5 (x=0, x=10, y=0, y=10, floor, ceiling),
    one TX at (2,3,1.5) and one RX at (7,6,1.5), up to 2 reflections.
    """
    parts = _box_room_parts(10.0, 10.0, 3.0, 0.10, labels=[0, 1, 2, 3, 4, 5],
                            materials=[0, 0, 0, 0, 1, 2])
    xyz, nrm, lab, mat = merge_clouds(parts)
    return Scene("room_tiny", xyz, nrm, lab, mat,
                 tx=np.array([[2.0, 3.0, 1.5]]), rx=np.array([[7.0, 6.0, 1.5]]),
                 max_refl=2, max_diff=0, meta={"spacing": 0.10, "room": (10.0, 10.0, 3.0)})


BOX_LO = (4.5, 6.5, 0.0)
BOX_HI = (5.5, 7.5, 2.0)


def room_noisy(seed: int = 1, n_tx: int = 4, n_rx: int = 16, spacing: float = 0.05) -> Scene:
    """The 10x10x3 m room at 5 cm (~130k points) with noise and a box obstacle.

    Position noise N(0, 5 mm), normal tilt N(0, 2 deg); a 1x1x2 m box at
    [4.5,5.5]x[6.5,7.5]x[0,2] (labels 6..10, no floor points under it) with its
    8 exterior edges (labels 11..18).  n_tx TX and n_rx RX are drawn uniformly in
    the room, >= 0.3 m from the walls and outside the box; <= 3 reflections and
    <= 1 diffraction.
    """
    rng = np.random.default_rng(seed)

    def outside_box_footprint(p):
        return ~((p[:, 0] >= BOX_LO[0]) & (p[:, 0] <= BOX_HI[0]) &
                 (p[:, 1] >= BOX_LO[1]) & (p[:, 1] <= BOX_HI[1]))

    parts = _box_room_parts(10.0, 10.0, 3.0, spacing, labels=[0, 1, 2, 3, 4, 5],
                            materials=[0, 0, 0, 0, 1, 2], floor_hole_fn=outside_box_footprint)
    parts += _box_parts(BOX_LO, BOX_HI, spacing, 6, 3)
    xyz, nrm, lab, mat = merge_clouds(parts)
    xyz64, nrm64 = _perturb(xyz.astype(np.float64), nrm.astype(np.float64), rng, 0.005, 2.0)
    edges, elab = _box_edges(BOX_LO, BOX_HI, 11)

    tx, rx = _noisy_room_pairs(rng, n_tx, n_rx)
    return Scene("room_noisy", np.ascontiguousarray(xyz64.astype(np.float32)),
                 np.ascontiguousarray(nrm64.astype(np.float32)), lab, mat, edges, elab, tx, rx,
                 max_refl=3, max_diff=1, meta={"spacing": spacing, "room": (10.0, 10.0, 3.0)})


def _near_box(p):
    m = 0.3
    return (BOX_LO[0] - m <= p[0] <= BOX_HI[0] + m and BOX_LO[1] - m <= p[1] <= BOX_HI[1] + m
            and p[2] <= BOX_HI[2] + m)


def _noisy_room_pairs(rng, n_tx, n_rx):
    tx = _uniform_points(rng, n_tx, [0.3, 0.3, 0.3], [9.7, 9.7, 2.7], _near_box)
    rx = _uniform_points(rng, n_rx, [0.3, 0.3, 0.3], [9.7, 9.7, 2.7], _near_box)
    return tx, rx


def room_noisy_pairs(seed: int, n_tx: int = 4, n_rx: int = 16):
    """Another seeded TX/RX draw for the noisy room (same rules as room_noisy)."""
    return _noisy_room_pairs(np.random.default_rng(seed), n_tx, n_rx)


def indoor(seed: int = 2, n_rx: int = 256, target_points: int = 2_000_000) -> Scene:
    """Indoor scan: 3x2 grid of 8x7x3 m rooms with doorways and 40 furniture boxes.

    Interior walls are 0.1 m thick and sampled on both sides with 1.0x2.1 m
    doorways; 40 axis-aligned boxes of seeded size U(0.4,2.0)^3 stand on the
    floors; 8 materials; U(+-1 cm) jitter.  The lattice spacing starts at 3 cm and is
    scaled so the cloud holds ``target_points`` (+-5%).  1 TX, ``n_rx`` RX.
    """
    rng = np.random.default_rng(seed)
    RX_, RY_, H = 8.0, 7.0, 3.0

    def build(spacing):
        parts = []
        lab = 0
        X, Y, Z = np.eye(3)
        walls_x = [0.0, 8.0, 16.0, 24.0]
        walls_y = [0.0, 7.0, 14.0]
        for i in range(3):
            for j in range(2):
                x0, x1 = walls_x[i], walls_x[i + 1]
                y0, y1 = walls_y[j], walls_y[j + 1]
                # inner faces of interior walls sit 0.05 m off the wall axis
                fx0 = x0 + (0.05 if i > 0 else 0.0)
                fx1 = x1 - (0.05 if i < 2 else 0.0)
                fy0 = y0 + (0.05 if j > 0 else 0.0)
                fy1 = y1 - (0.05 if j < 1 else 0.0)
                Lx, Ly = fx1 - fx0, fy1 - fy0
                parts.append(plane_patch([fx0, fy0, 0], X, Y, Lx, Ly, spacing, [0, 0, 1], lab, 0)); lab += 1
                parts.append(plane_patch([fx0, fy0, H], X, Y, Lx, Ly, spacing, [0, 0, -1], lab, 1)); lab += 1
                # doorways: in the x-walls shared with a neighbour room, in the y-wall
                hx = (Ly / 2 - 0.5, Ly / 2 + 0.5, 0.0, 2.1)
                hy = (Lx / 2 - 0.5, Lx / 2 + 0.5, 0.0, 2.1)
                parts.append(plane_patch([fx0, fy0, 0], Y, Z, Ly, H, spacing, [1, 0, 0], lab, 2,
                                         hole=hx if i > 0 else None)); lab += 1
                parts.append(plane_patch([fx1, fy0, 0], Y, Z, Ly, H, spacing, [-1, 0, 0], lab, 2,
                                         hole=hx if i < 2 else None)); lab += 1
                parts.append(plane_patch([fx0, fy0, 0], X, Z, Lx, H, spacing, [0, 1, 0], lab, 3,
                                         hole=hy if j > 0 else None)); lab += 1
                parts.append(plane_patch([fx0, fy1, 0], X, Z, Lx, H, spacing, [0, -1, 0], lab, 3,
                                         hole=hy if j < 1 else None)); lab += 1
        return parts, lab

    # furniture boxes: seeded sizes and positions, kept inside one room and off the doorways
    boxes = []
    brng = np.random.default_rng(seed + 1000)
    while len(boxes) < 40:
        size = brng.uniform(0.4, 2.0, 3)
        room_i, room_j = brng.integers(0, 3), brng.integers(0, 2)
        x0 = room_i * RX_ + 0.4 + brng.random() * (RX_ - 0.8 - size[0])
        y0 = room_j * RY_ + 0.4 + brng.random() * (RY_ - 0.8 - size[1])
        if x0 < room_i * RX_ + 0.4 or y0 < room_j * RY_ + 0.4:
            continue
        lo = np.array([x0, y0, 0.0])
        hi = lo + size
        hi[2] = min(hi[2], H - 0.4)
        clash = any(np.all(lo < b[1] + 0.2) and np.all(b[0] < hi + 0.2) for b in boxes)
        if not clash:
            boxes.append((lo, hi))

    def with_boxes(spacing, lab):
        parts = []
        edges = []
        elab = []
        for k, (lo, hi) in enumerate(boxes):
            parts += _box_parts(lo, hi, spacing, lab, 4 + (k % 4))
            lab += 5
        for k, (lo, hi) in enumerate(boxes):
            e, el = _box_edges(lo, hi, lab)
            edges.append(e)
            elab.append(el)
            lab += 8
        return parts, np.concatenate(edges), np.concatenate(elab)

    spacing = 0.03
    for _ in range(3):
        parts, lab = build(spacing)
        bparts, edges, elab = with_boxes(spacing, lab)
        n = sum(p[0].shape[0] for p in parts + bparts)
        if abs(n - target_points) <= 0.02 * target_points:
            break
        spacing *= math.sqrt(n / target_points)
    xyz, nrm, labv, mat = merge_clouds(parts + bparts)
    # drop floor points under boxes
    keep = np.ones(xyz.shape[0], bool)
    for lo, hi in boxes:
        keep &= ~((xyz[:, 2] == 0.0) & (xyz[:, 0] >= lo[0]) & (xyz[:, 0] <= hi[0]) &
                  (xyz[:, 1] >= lo[1]) & (xyz[:, 1] <= hi[1]))
    xyz, nrm, labv, mat = xyz[keep], nrm[keep], labv[keep], mat[keep]
    jit = rng.uniform(-0.01, 0.01, size=xyz.shape)
    xyz = (xyz.astype(np.float64) + jit).astype(np.float32)

    def in_box(p):
        return any(np.all(p >= b[0] - 0.3) and np.all(p <= b[1] + 0.3) for b in boxes)

    tx = _uniform_points(rng, 1, [0.5, 0.5, 1.0], [7.5, 6.5, 2.0], in_box)
    rx = _uniform_points(rng, n_rx, [0.5, 0.5, 0.5], [23.5, 13.5, 2.5], in_box)
    return Scene("indoor", np.ascontiguousarray(xyz), np.ascontiguousarray(nrm), labv, mat,
                 edges, elab, tx, rx, max_refl=3, max_diff=1,
                 meta={"spacing": spacing, "boxes": [(b[0].tolist(), b[1].tolist()) for b in boxes]})


def street(seed: int = 3, n_tx: int = 16, n_rx: int = 1024, target_points: int = 20_000_000) -> Scene:
    """Street canyon over 200x50 m: two rows of box buildings (10-30 m wide and tall).

    Rows occupy y in [0,15] and [35,50]; facades toward the street, roofs and the
    street ground are sampled; 4 materials (ground, facade, roof, side wall).
    Lattice spacing starts at 3 cm and is scaled to hold ``target_points`` (+-5%).
    Edges: street-side vertical building corners and facade-roof edges.
    TX and RX at 1.5 m height in the street.
    """
    rng = np.random.default_rng(seed)
    X, Y, Z = np.eye(3)
    rows = []
    for side in (0, 1):
        x = 0.0
        blds = []
        while x < 200.0 - 1e-9:
            w = min(rng.uniform(10, 30), 200.0 - x)
            h = rng.uniform(10, 30)
            blds.append((x, x + w, h))
            x += w
        rows.append(blds)

    def build(spacing):
        parts = []
        edges = []
        elab = []
        lab = 0
        parts.append(plane_patch([0, 15, 0], X, Y, 200.0, 20.0, spacing, [0, 0, 1], lab, 0)); lab += 1
        for side, blds in enumerate(rows):
            yf = 15.0 if side == 0 else 35.0
            fn = [0, 1, 0] if side == 0 else [0, -1, 0]
            y_back = 0.0 if side == 0 else 50.0
            for k, (x0, x1, h) in enumerate(blds):
                parts.append(plane_patch([x0, yf, 0], X, Z, x1 - x0, h, spacing, fn, lab, 1)); lab += 1
                lo_y = min(yf, y_back)
                parts.append(plane_patch([x0, lo_y, h], X, Y, x1 - x0, 15.0, spacing, [0, 0, 1], lab, 2)); lab += 1
                # exposed side walls where the neighbour is lower (or the row ends)
                for nb, xs, sn in ((blds[k - 1] if k > 0 else None, x0, [-1, 0, 0]),
                                   (blds[k + 1] if k + 1 < len(blds) else None, x1, [1, 0, 0])):
                    hn = nb[2] if nb is not None else 0.0
                    if h > hn + 1e-6:
                        parts.append(plane_patch([xs, lo_y, hn], Y, Z, 15.0, h - hn, spacing, sn, lab, 3)); lab += 1
                        edges.append(np.concatenate([[xs, yf, hn], [xs, yf, h], fn, sn]))
                edges.append(np.concatenate([[x0, yf, h], [x1, yf, h], fn, [0, 0, 1]]))
        e = np.array(edges, np.float64)
        elab = np.arange(lab, lab + e.shape[0], dtype=np.uint32)
        return parts, e, elab

    spacing = 0.03
    for _ in range(3):
        parts, edges, elab = build(spacing)
        n = sum(p[0].shape[0] for p in parts)
        if abs(n - target_points) <= 0.02 * target_points:
            break
        spacing *= math.sqrt(n / target_points)
    xyz, nrm, lab, mat = merge_clouds(parts)
    tx = np.column_stack([rng.uniform(5, 195, n_tx), rng.uniform(17, 33, n_tx), np.full(n_tx, 1.5)])
    rx = np.column_stack([rng.uniform(2, 198, n_rx), rng.uniform(16, 34, n_rx), np.full(n_rx, 1.5)])
    return Scene("street", xyz, nrm, lab, mat, edges, elab, tx, rx, max_refl=4, max_diff=1,
                 meta={"spacing": spacing})


def wedge(spacing: float = 0.05, z_tx: float = 0.5, z_rx: float = 2.5) -> Scene:
    """A sampled 90 degree convex corner: the solid is x<=0, y<=0 (0 <= z <= 3).

    Face x=0 (y in [-4,0], outward normal +x, label 0) and face y=0 (x in [-4,0],
    outward normal +y, label 1) meet at the edge x=y=0 (label 2).  TX at
    (1,-3,z_tx) and RX at (-3,1,z_rx) see each other only by diffraction at the
    edge; the Keller point is at z = z_tx + (z_rx - z_tx) * r1/(r1 + r2) with
    r1 = r2 = sqrt(10).
    """
    X, Y, Z = np.eye(3)
    parts = [plane_patch([0, -4, 0], Y, Z, 4.0, 3.0, spacing, [1, 0, 0], 0, 0),
             plane_patch([-4, 0, 0], X, Z, 4.0, 3.0, spacing, [0, 1, 0], 1, 0)]
    xyz, nrm, lab, mat = merge_clouds(parts)
    edges = np.array([[0, 0, 0, 0, 0, 3.0, 1, 0, 0, 0, 1, 0]], np.float64)
    return Scene("wedge", xyz, nrm, lab, mat, edges, np.array([2], np.uint32),
                 tx=np.array([[1.0, -3.0, z_tx]]), rx=np.array([[-3.0, 1.0, z_rx]]),
                 max_refl=0, max_diff=1, meta={"spacing": spacing},
                 region=np.array([[-4.0, -4.0, 0.0], [1.5, 1.5, 3.0]]))


def wedge_on_floor(z_tx: float = 0.8, z_rx: float = 2.0, spacing: float = 0.05) -> Scene:
    """The convex corner of ``wedge`` standing on a sampled floor (z = 0, label 3).

    The floor covers x in [-4, 2], y in [-4, 2] outside the solid (x <= 0, y <= 0).
    Besides the pure diffraction, TX and RX are joined by one path that mixes a floor
    reflection and the edge diffraction, the floor taken next to the lower end.  With
    z_tx < z_rx the floor comes first: unfolding it puts the TX at (1, -3, -z_tx), its
    Keller point on the edge is at z = (z_rx - z_tx) / 2 (both ends sqrt(10) m from
    the edge), and the floor point is where that unfolded segment meets z = 0.  With
    z_tx > z_rx the RX is unfolded instead and the edge comes first.
    """
    w = wedge(spacing=spacing, z_tx=z_tx, z_rx=z_rx)
    X, Y, _ = np.eye(3)
    floor = [plane_patch([0, -4, 0], X, Y, 2.0, 6.0, spacing, [0, 0, 1], 3),
             plane_patch([-4, 0, 0], X, Y, 4.0 - spacing, 2.0, spacing, [0, 0, 1], 3)]
    fx, fn, fl, fm = merge_clouds(floor)
    return Scene("wedge_on_floor", np.vstack([w.xyz, fx]), np.vstack([w.nrm, fn]), np.concatenate([w.label, fl]),
                 np.concatenate([w.material, fm]), w.edges, w.edge_label, tx=w.tx, rx=w.rx, max_refl=1,
                 max_diff=1, meta={"spacing": spacing}, region=np.array([[-4.0, -4.0, 0.0], [2.0, 2.0, 3.0]]))


def box_cloud(lo, size: float = 2.0, spacing: float = 0.05, label0: int = 100, material: int = 5):
    """A closed box of side `size` standing at lo (its five visible faces sampled at
    `spacing`, labels label0..label0+4): (xyz, nrm, label, material, aabb_lo, aabb_hi)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = lo + size
    xyz, nrm, lab, mat = merge_clouds(_box_parts(lo, hi, spacing, label0, material))
    return xyz, nrm, lab, mat, lo, hi


def moving_box(room: Scene, step: int, seed: int = 4, size: float = 2.0, spacing: float = 0.05):
    """A 2x2x2 m box on a seeded random walk in the 10x10 m room (dynamic scenes).

    Returns (xyz, nrm, label, material, aabb_lo, aabb_hi) for the box at walk
    ``step``; labels 100..104.
    """
    rng = np.random.default_rng(seed)
    pos = np.array([2.0, 2.0])
    for _ in range(step):
        pos = np.clip(pos + rng.normal(0, 0.5, 2), 0.5, 10.0 - size - 0.5)
    lo = np.array([pos[0], pos[1], 0.0])
    hi = lo + size
    xyz, nrm, lab, mat = merge_clouds(_box_parts(lo, hi, spacing, 100, 5))
    return xyz, nrm, lab, mat, lo, hi


def serving_requests(n: int, rate_hz: float, scene_ids, seed: int = 4, max_pairs: int = 64,
                     depth_range=(2, 5), room=(10.0, 10.0, 3.0), pools: dict | None = None,
                     depth_caps: dict | None = None):
    """Poisson request stream: arrival time, scene id, 1 TX, 1..max_pairs RX, max depth.

    Each request picks a resident scene uniformly and a max interaction depth in
    depth_range (lowered to the scene's entry in depth_caps, if any).  With pools,
    its TX and RXs are distinct positions drawn from the scene's pool (free-space
    positions made by the scene's own generator); without, they are uniform in the
    room box, 0.3 m from the walls.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        sid = scene_ids[int(rng.integers(0, len(scene_ids)))]
        k = int(rng.integers(1, max_pairs + 1))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        if depth_caps and sid in depth_caps:
            depth = min(depth, int(depth_caps[sid]))
        if pools and sid in pools:
            pool = pools[sid]
            pick = rng.choice(pool.shape[0], size=min(k + 1, pool.shape[0]), replace=False)
            tx, rx = pool[pick[:1]], pool[pick[1:]]
        else:
            lo = np.array([0.3, 0.3, 0.3])
            hi = np.array(room) - 0.3
            tx = lo + (hi - lo) * rng.random((1, 3))
            rx = lo + (hi - lo) * rng.random((k, 3))
        out.append({"id": i, "t": t, "scene": sid, "tx": tx, "rx": rx, "depth": depth})
    return out
