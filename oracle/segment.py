"""Automatic surface labels and exterior edges for unlabelled point clouds: the plain FP64
reference.

TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct statement that the CUDA
labelling (nimbus_segment) is checked against.  Only tests/, the smoke check and the
benchmark's CPU leg may import it.

The paper's method starts from a labelled cloud.  Its labels come from a segmentation
whose clusters are distinct surfaces (Section 2; the experiments of Section 3 used a
plane-fitting algorithm from PCL), its diffraction edges are inserted by hand
(Section 2), and raw sensor clouds are left to future work (Section 3.3).  The paper
fixes no algorithm for either step, so the reading used here is stated in full:

1. Binning.  Points fall into subvoxels exactly as in the voxelisation (Section 2.1):
   FP32 (x - o), then / h_s, then floor.  The points of one subvoxel, in input order,
   form a group; groups are ordered by (voxel, subvoxel).
2. Plane of a group.  FP64 centroid c and covariance C (two passes).  The normal n is
   the eigenvector of C's smallest eigenvalue, turned to agree with the sum of the
   group's input normals.  The group is planar when it holds at least min_points
   points, trace(C) > 0, the smallest eigenvalue is at most flat_max * trace(C) and the
   middle one at least spread_min * trace(C) (a single row of points has no plane).
3. Surfaces.  Two planar groups in 26-adjacent subvoxels are joined when
   n_a . n_b >= cos(join_angle) and each centroid lies within join_dist of the other's
   plane.  The connected sets of joined groups are the surfaces; a non-planar group is
   a surface of its own.  Surfaces are numbered 0, 1, ... in the order of their first
   group.
4. Point labels.  A group fits a point p with input normal n_p when the group is planar,
   n . n_p >= cos(join_angle) and |n . (p - c)| <= join_dist.  A point takes its own
   group's surface when its group fits it; otherwise the surface of the fitting
   26-neighbour group whose plane is nearest (ties: the lower group); with none, it keeps
   its own group's surface.  (A subvoxel on a room's edge can hold a wall's bottom and
   the floor's last row in one plane: the floor points then go to the floor.)
5. Exterior edges.  A surface with planar groups has the plane of their pooled FP64
   moments, its normal turned to agree with the sum of the groups' normals.  Two
   surfaces meet where a planar group of each lies in 26-adjacent subvoxels.  They form
   an exterior (convex) edge when each has at least edge_min_groups planar groups,
   n_A . n_B <= cos(edge_angle) and each surface's centroid lies strictly behind the
   other's plane.  The edge lies on the line where
   the two planes meet, at the point of that line nearest the mean centroid of the
   meeting groups, and spans the projections of those groups' centroids onto the line.
   Its face normals are n_A and n_B.  Edges are ordered by (A, B); edge e gets label
   n_surfaces + e.

Pinned (tests/test_segment_oracle.py) on clouds sampled from exact planes -- the box
room's six faces, the wedge's convex edge, sheets folded at 5 to 40 degrees and sheets
offset by 1 and 10 cm, boxes too small to have edges, the numbering of two sheets --
and on the noisy room's box, whose eight exterior edges are known.
tests/test_oracle_mutants.py checks that planted mistakes in this module fail them.
"""
from __future__ import annotations

import math
from types import SimpleNamespace

import numpy as np

import oracle as _oracle

# 26-neighbour offsets, in (dz, dy, dx) loop order
_NEIGHBOURS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
               if (dx, dy, dz) != (0, 0, 0)]


def grid_of(xyz, nrm, sp):
    """Origin and voxel dims of the voxelisation grid of this cloud (the oracle's own
    voxelisation; only the grid parameters matter here)."""
    n = xyz.shape[0]
    hs = sp.voxel_size / sp.dv
    vp = SimpleNamespace(voxel_size=sp.voxel_size, dv=sp.dv, cone_half_angle_deg=4.0, launch_spacing_deg=0.5,
                         sdf_sigma=hs / 2, sdf_eps=1e-3, ignore_dist=hs * math.sqrt(3.0), sep_eps=hs / 4,
                         delta=1e-4, gamma=0.5, grad_stop=1e-6, freq_hz=60e9, max_refl=0, max_diff=0,
                         max_interactions=0, kappa=1, launch_count=1, sdf_max_steps=1, rho=0)
    s = _oracle.Scene(xyz, nrm, np.zeros(n, np.uint32), np.zeros(n, np.uint8), np.zeros((0, 12)),
                      np.zeros(0, np.uint32), vp)
    return np.asarray(s.origin, np.float64), np.asarray(s.dims, np.int64)


def groups(xyz, origin, dims, sp):
    """Step 1: subvoxel of every point; groups in (voxel, subvoxel) order."""
    dv = sp.dv
    x32 = np.asarray(xyz, np.float32)
    o32 = np.asarray(origin, np.float64).astype(np.float32)
    hs32 = np.float32(sp.voxel_size / sp.dv)
    t = (x32 - o32[None, :]) / hs32              # FP32 subtract, then FP32 divide
    gs = np.floor(t).astype(np.int64)
    hi = dims[None, :] * dv - 1
    gs = np.minimum(np.maximum(gs, 0), hi)
    vox = gs // dv
    sub = gs % dv
    cell = (vox[:, 2] * dims[1] + vox[:, 1]) * dims[0] + vox[:, 0]
    key = cell * dv ** 3 + (sub[:, 2] * dv + sub[:, 1]) * dv + sub[:, 0]
    order = np.argsort(key, kind="stable")
    k_sorted = key[order]
    starts = np.flatnonzero(np.r_[True, k_sorted[1:] != k_sorted[:-1]])
    ends = np.r_[starts[1:], len(order)]
    g_of_point = np.empty(len(order), np.int64)
    for g, (a, b) in enumerate(zip(starts, ends)):
        g_of_point[order[a:b]] = g
    return order, starts, ends, gs[order[starts]], g_of_point


def fit_group(p, nr, sp):
    """Step 2 for one group: centroid, covariance, oriented normal, planarity."""
    m = p.shape[0]
    c = p.sum(axis=0) / m
    d = p - c
    C = d.T @ d / m
    w, V = np.linalg.eigh(C)                      # ascending eigenvalues
    n = V[:, 0].copy()
    if n @ nr.sum(axis=0) < 0.0:
        n = -n
    tr = float(np.trace(C))
    planar = m >= sp.min_points and tr > 0.0 and w[0] <= sp.flat_max * tr and w[1] >= sp.spread_min * tr
    return c, n, C, planar


def segment(xyz, nrm, sp):
    """Labels (one per input point) and exterior edges of an unlabelled cloud.

    sp: any object with the attributes of the labelling parameters (voxel_size, dv,
    min_points, flat_max, spread_min, join_angle_deg, join_dist, edge_angle_deg,
    edge_min_groups).  Returns
    (labels uint32[n], edges float64[m, 12] = p0, p1, n_face0, n_face1,
    edge_labels uint32[m], n_surfaces).
    """
    xyz = np.asarray(xyz, np.float32)
    nrm = np.asarray(nrm, np.float32)
    origin, dims = grid_of(xyz, nrm, sp)
    order, starts, ends, ggs, g_of_point = groups(xyz, origin, dims, sp)
    G = len(starts)
    P = xyz.astype(np.float64)
    N = nrm.astype(np.float64)
    cos_join = math.cos(math.radians(sp.join_angle_deg))
    cos_edge = math.cos(math.radians(sp.edge_angle_deg))

    # step 2
    cen = np.zeros((G, 3))
    nor = np.zeros((G, 3))
    cov = np.zeros((G, 3, 3))
    cnt = (ends - starts).astype(np.int64)
    planar = np.zeros(G, bool)
    for g in range(G):
        idx = order[starts[g]:ends[g]]
        cen[g], nor[g], cov[g], planar[g] = fit_group(P[idx], N[idx], sp)

    # subvoxel -> group
    index = {tuple(int(v) for v in ggs[g]): g for g in range(G)}

    def neighbours(g):
        x, y, z = (int(v) for v in ggs[g])
        for dx, dy, dz in _NEIGHBOURS:
            h = index.get((x + dx, y + dy, z + dz))
            if h is not None:
                yield h

    # step 3: union-find whose root is always the lowest group of the set
    parent = list(range(G))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    def joined(a, b):
        return (nor[a] @ nor[b] >= cos_join and abs(nor[a] @ (cen[b] - cen[a])) <= sp.join_dist
                and abs(nor[b] @ (cen[a] - cen[b])) <= sp.join_dist)

    for a in range(G):
        if not planar[a]:
            continue
        for b in neighbours(a):
            if b > a and planar[b] and joined(a, b):
                ra, rb = find(a), find(b)
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
    root = np.array([find(g) for g in range(G)], np.int64)
    is_root = root == np.arange(G)
    surf_of_root = np.cumsum(is_root) - 1
    surf = surf_of_root[root]
    n_surf = int(is_root.sum())

    # step 4
    def fits(h, i):
        return planar[h] and nor[h] @ N[i] >= cos_join and abs(nor[h] @ (P[i] - cen[h])) <= sp.join_dist

    labels = np.zeros(xyz.shape[0], np.uint32)
    for g in range(G):
        cand = sorted(h for h in neighbours(g) if planar[h])
        for i in order[starts[g]:ends[g]]:
            if fits(g, i):
                labels[i] = surf[g]
                continue
            best, best_d = -1, math.inf
            for h in cand:
                if fits(h, i):
                    dist = abs(nor[h] @ (P[i] - cen[h]))
                    if dist < best_d:
                        best, best_d = h, dist
            labels[i] = surf[best] if best >= 0 else surf[g]

    # step 5: planes of the surfaces from the pooled moments of their planar groups
    members = {}
    for g in range(G):
        if planar[g]:
            members.setdefault(int(surf[g]), []).append(g)
    splane = {}
    for A, gl in members.items():
        m = sum(int(cnt[g]) for g in gl)
        c = sum(cnt[g] * cen[g] for g in gl) / m
        S = sum(cnt[g] * (cov[g] + np.outer(cen[g] - c, cen[g] - c)) for g in gl) / m
        w, V = np.linalg.eigh(S)
        n = V[:, 0].copy()
        if n @ sum(nor[g] for g in gl) < 0.0:
            n = -n
        splane[A] = (c, n)
    meet = {}
    for a in range(G):
        if not planar[a]:
            continue
        for b in neighbours(a):
            if b > a and planar[b] and surf[a] != surf[b]:
                A, B = sorted((int(surf[a]), int(surf[b])))
                meet.setdefault((A, B), set()).update((a, b))
    edges = []
    for (A, B) in sorted(meet):
        if len(members[A]) < sp.edge_min_groups or len(members[B]) < sp.edge_min_groups:
            continue
        (cA, nA), (cB, nB) = splane[A], splane[B]
        if not (nA @ nB <= cos_edge and nA @ (cB - cA) < 0.0 and nB @ (cA - cB) < 0.0):
            continue
        gl = sorted(meet[(A, B)])
        mid = sum(cen[g] for g in gl) / len(gl)
        w = np.cross(nA, nB)
        w /= np.linalg.norm(w)
        # nearest point to mid on both planes: mid + alpha nA + beta nB
        M = np.array([[nA @ nA, nA @ nB], [nA @ nB, nB @ nB]])
        r = np.array([nA @ cA - nA @ mid, nB @ cB - nB @ mid])
        al, be = np.linalg.solve(M, r)
        x0 = mid + al * nA + be * nB
        t = [w @ (cen[g] - x0) for g in gl]
        edges.append(np.concatenate([x0 + min(t) * w, x0 + max(t) * w, nA, nB]))
    E = np.array(edges, np.float64).reshape(-1, 12)
    return labels, E, (n_surf + np.arange(len(E))).astype(np.uint32), n_surf
