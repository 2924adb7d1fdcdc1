"""Pins of the labelling oracle (oracle/segment.py) against clouds whose surfaces and
exterior edges are known: sampled exact planes and the noisy room's box.  CPU only."""
from collections import Counter

import numpy as np
import pytest

import oracle.segment as seg
from paper_2402_13747_b300 import config, scenes
from tests import segclouds

SP = config.SegmentParams()


def _partition_matches(auto, true):
    """Every auto label lies inside one true label and vice versa (a relabelling)."""
    pairs = set(zip(auto.tolist(), true.tolist()))
    return len(pairs) == len(set(auto.tolist())) == len(set(true.tolist()))


def _segment_dist(p, a, b):
    """Distance from point p to the segment a-b."""
    ab = b - a
    t = np.clip((p - a) @ ab / (ab @ ab), 0.0, 1.0)
    return float(np.linalg.norm(a + t * ab - p))


def test_box_room_faces_are_the_surfaces():
    """Six exact faces sampled with shared border rows: the labels are the faces, and
    every edge of the room is concave, so none is extracted."""
    sc = scenes.room_tiny()
    lab, E, EL, ns = seg.segment(sc.xyz, sc.nrm, SP)
    assert _partition_matches(lab, sc.label)
    assert len(E) == 0 and len(EL) == 0
    assert lab.max() < ns


@pytest.mark.parametrize("with_floor", [False, True])
def test_convex_corner_edge(with_floor):
    """The corner x = y = 0 of two exact faces: one exterior edge on the z axis with the
    faces' normals; on a floor, the floor's junctions with the faces are concave."""
    sc = scenes.wedge_on_floor() if with_floor else scenes.wedge()
    lab, E, EL, ns = seg.segment(sc.xyz, sc.nrm, SP)
    assert _partition_matches(lab, sc.label)
    assert len(E) == 1 and EL.tolist() == [ns]
    p0, p1, n0, n1 = E[0, :3], E[0, 3:6], E[0, 6:9], E[0, 9:]
    np.testing.assert_allclose(p0[:2], 0.0, atol=1e-9)
    np.testing.assert_allclose(p1[:2], 0.0, atol=1e-9)
    lo, hi = sorted((p0[2], p1[2]))
    assert lo <= SP.h_s + (0.25 if with_floor else 0.0) and hi >= 3.0 - SP.h_s
    assert {tuple(np.round(n0, 9)), tuple(np.round(n1, 9))} == {(1.0, 0.0, 0.0), (0.0, 1.0, 0.0)}


def test_noisy_room_box_edges_and_faces():
    """The noisy room (5 mm position noise, 2 degree normal tilt): the eight exterior
    edges of the box and no other, each within 2 cm of the generator's edge and covering
    most of it; the labels reproduce the generator's faces for all but a few points."""
    sc = scenes.room_noisy(n_tx=1, n_rx=1)
    lab, E, EL, ns = seg.segment(sc.xyz, sc.nrm, SP)
    assert len(E) == 8
    matched = set()
    for e in E:
        p0, p1 = e[:3], e[3:6]
        best = min(range(len(sc.edges)), key=lambda k: _segment_dist(p0, sc.edges[k, :3], sc.edges[k, 3:6]) +
                   _segment_dist(p1, sc.edges[k, :3], sc.edges[k, 3:6]))
        a, b = sc.edges[best, :3], sc.edges[best, 3:6]
        assert _segment_dist(p0, a, b) < 0.02 and _segment_dist(p1, a, b) < 0.02
        assert np.linalg.norm(p1 - p0) >= 0.7 * np.linalg.norm(b - a)
        normals = {tuple(np.round(e[6:9])), tuple(np.round(e[9:]))}
        assert normals == {tuple(sc.edges[best, 6:9]), tuple(sc.edges[best, 9:])}
        matched.add(best)
    assert len(matched) == 8
    # faces: the majority true label of each auto label
    cnt = Counter(zip(lab.tolist(), sc.label.tolist()))
    major = {}
    for (a, t), c in cnt.items():
        if a not in major or c > major[a][1]:
            major[a] = (t, c)
    wrong = sum(c for (a, t), c in cnt.items() if major[a][0] != t)
    assert wrong <= 1e-4 * len(lab)
    assert {t for t, _ in major.values()} == set(sc.label.tolist())


def test_labels_do_not_depend_on_point_order():
    """Surfaces are numbered by their first subvoxel, not by input order: a shuffled
    cloud gets the same label per point."""
    sc = scenes.wedge_on_floor()
    lab, E, _, _ = seg.segment(sc.xyz, sc.nrm, SP)
    perm = np.random.default_rng(5).permutation(len(lab))
    lab2, E2, _, _ = seg.segment(sc.xyz[perm], sc.nrm[perm], SP)
    np.testing.assert_array_equal(lab2, lab[perm])
    np.testing.assert_allclose(E2, E, atol=1e-12)



@pytest.mark.parametrize("deg", [5, -5, 11, -11, 20, -20, 40, -40])
def test_folded_sheet_joins_within_the_join_angle(deg):
    """Two planar sheets meeting along a line join into one surface when their normals
    agree within the join angle (10 degrees) and stay two otherwise (at 11 degrees the
    groups next to the fold still lie within the join distance of each other's plane,
    so the angle alone keeps them apart); the fold is an exterior edge only when it is
    convex and at least the edge angle (30 degrees), and then it lies on the fold line
    with the two sheets' normals."""
    xyz, nrm, lab, n = segclouds.folded_sheet(deg)
    L, E, EL, ns = seg.segment(xyz, nrm, SP)
    if abs(deg) < SP.join_angle_deg:
        assert len(set(L.tolist())) == 1 and len(E) == 0
        return
    assert _partition_matches(L, lab)
    if deg > -SP.edge_angle_deg:
        assert len(E) == 0
        return
    assert len(E) == 1
    p0, p1 = E[0, :3], E[0, 3:6]
    for p in (p0, p1):
        np.testing.assert_allclose(p[[0, 2]], [2.0, 0.6], atol=1e-9)
    assert min(p0[1], p1[1]) <= SP.h_s and max(p0[1], p1[1]) >= 2.0 - SP.h_s
    faces = sorted([E[0, 6:9], E[0, 9:]], key=lambda v: v[0])    # planes fitted to FP32 points
    np.testing.assert_allclose(faces[0], [0.0, 0.0, 1.0], atol=1e-6)
    np.testing.assert_allclose(faces[1], n, atol=1e-6)


@pytest.mark.parametrize("dz,surfaces", [(0.01, 1), (0.1, 2)])
def test_offset_sheets_join_within_the_join_distance(dz, surfaces):
    """Two parallel sheets side by side, one raised by dz: within the join distance
    (3 cm) their groups join across the seam, beyond it they are two surfaces."""
    xyz, nrm, lab = segclouds.offset_sheets(dz)
    L, E, _, _ = seg.segment(xyz, nrm, SP)
    assert len(set(L.tolist())) == surfaces and len(E) == 0
    if surfaces == 2:
        assert _partition_matches(L, lab)


@pytest.mark.parametrize("size,edges", [(0.3, 0), (0.5, 0), (1.0, 8)])
def test_small_boxes_have_no_edges(size, edges):
    """A box on a floor: a face needs edge_min_groups (4) planar subvoxel groups before
    its edges count, so boxes of a subvoxel or two across give none, and a 1 m box gives
    its eight exterior edges (four vertical, four on top; the floor's are concave)."""
    xyz, nrm, _ = segclouds.box_on_floor(size)
    _, E, _, _ = seg.segment(xyz, nrm, SP)
    assert len(E) == edges


def test_surfaces_are_numbered_by_their_first_subvoxel():
    """Surface numbers follow each surface's first subvoxel group in (voxel, subvoxel)
    order, whatever its other groups: sheet A starts in the first grid row before
    sheet B, so A's number is lower, although B's last subvoxel comes long before A's."""
    xyz, nrm, lab = segclouds.two_sheets_in_row_order()
    L, _, _, _ = seg.segment(xyz, nrm, SP)
    assert _partition_matches(L, lab)
    assert L[lab == 0][0] < L[lab == 1][0]
