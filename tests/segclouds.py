"""Synthetic clouds for the labelling tests: exact planar sheets and boxes whose
surfaces and exterior edges are known.  Input generators only (no method arithmetic)."""
import numpy as np

from paper_2402_13747_b300 import scenes

X, Y = np.eye(3)[0], np.eye(3)[1]


def folded_sheet(deg):
    """A 2 x 2 m sheet at z = 0.6 (label 0) continued past x = 2 by a second 2 x 2 m
    sheet (label 1) turned by deg about the fold line x = 2, z = 0.6 (up: concave,
    down: convex).  Returns xyz, nrm, label and the second sheet's normal."""
    a = np.radians(deg)
    u = np.array([np.cos(a), 0.0, np.sin(a)])
    n = np.array([-np.sin(a), 0.0, np.cos(a)])
    parts = [scenes.plane_patch([0, 0, 0.6], X, Y, 2.0, 2.0, 0.05, [0, 0, 1], 0),
             scenes.plane_patch([2.0, 0, 0.6], u, Y, 2.0, 2.0, 0.05, n, 1)]
    xyz, nrm, lab, _ = scenes.merge_clouds(parts)
    return xyz, nrm, lab, n


def offset_sheets(dz):
    """Two parallel sheets side by side, x in [0, 1.95] at z = 0.6 (label 0) and
    x in [2, 4] at z = 0.6 + dz (label 1)."""
    parts = [scenes.plane_patch([0, 0, 0.6], X, Y, 1.95, 2.0, 0.05, [0, 0, 1], 0),
             scenes.plane_patch([2.0, 0, 0.6 + dz], X, Y, 2.0, 2.0, 0.05, [0, 0, 1], 1)]
    xyz, nrm, lab, _ = scenes.merge_clouds(parts)
    return xyz, nrm, lab


def box_on_floor(size):
    """A size^3 box standing on a 3 x 3 m floor (labels: floor 0, box faces 1..5)."""
    lo = np.array([0.4, 0.4, 0.0])
    parts = [scenes.plane_patch([-1, -1, 0], X, Y, 3.0, 3.0, 0.05, [0, 0, 1], 0)]
    parts += scenes._box_parts(lo, lo + size, 0.05, 1, 0)
    xyz, nrm, lab, _ = scenes.merge_clouds(parts)
    return xyz, nrm, lab


def two_sheets_in_row_order():
    """Sheet A (x in [0, 1], y in [0, 4], label 0) and sheet B (x in [3, 4], y in [0, 1],
    label 1) at z = 0.6: A's first subvoxel comes first, B's last long before A's."""
    parts = [scenes.plane_patch([0, 0, 0.6], X, Y, 1.0, 4.0, 0.05, [0, 0, 1], 0),
             scenes.plane_patch([3.0, 0, 0.6], X, Y, 1.0, 1.0, 0.05, [0, 0, 1], 1)]
    xyz, nrm, lab, _ = scenes.merge_clouds(parts)
    return xyz, nrm, lab
