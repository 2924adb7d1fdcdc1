"""Scenes of the refinement and visibility pins that both the oracle pins and the GPU
parity tests run: the box room with an occluding panel, the box room with two walls
sharing a label, and the wedge with room above its edge.  Input generators only."""
import dataclasses

import numpy as np

from paper_2402_13747_b300 import scenes

# the free-standing panel: the plane x = PANEL_X, y in [y0, y1], z in [z0, z1], label 6
PANEL_X, PANEL_Y, PANEL_Z = 4.0, (3.6, 5.4), (0.5, 2.5)


def room_with_panel(room_tiny):
    Y, Z = np.eye(3)[1], np.eye(3)[2]
    (y0, y1), (z0, z1) = PANEL_Y, PANEL_Z
    panel = scenes.plane_patch([PANEL_X, y0, z0], Y, Z, y1 - y0, z1 - z0, 0.1, [-1, 0, 0], 6)
    rt = room_tiny
    xyz, nrm, lab, mat = scenes.merge_clouds([(rt.xyz, rt.nrm, rt.label, rt.material), panel])
    return scenes.Scene("room_panel", xyz, nrm, lab, mat, tx=rt.tx, rx=rt.rx, max_refl=2, max_diff=0)


def room_with_merged_labels(room_tiny):
    """The walls x = 0 (label 0) and y = 0 (label 2) share label 0."""
    lab = room_tiny.label.copy()
    lab[lab == 2] = 0
    return scenes.Scene("room_tiny_merged", room_tiny.xyz, room_tiny.nrm, lab, room_tiny.material,
                        tx=room_tiny.tx, rx=room_tiny.rx, max_refl=2, max_diff=0)


def tall_wedge(z_tx, z_rx):
    """scenes.wedge with its grid reaching z = 4, so TX and RX may sit above the edge's
    end at z = 3."""
    return dataclasses.replace(scenes.wedge(z_tx=z_tx, z_rx=z_rx),
                               region=np.array([[-4.0, -4.0, 0.0], [1.5, 1.5, 4.0]]))


def panel_margin(tx, rx, labels, pts):
    """How a path meets the panel: (deepest, margin).  deepest: the largest distance
    inside the panel's rectangle at which a segment crosses the panel's plane (-inf when
    none crosses; > 0 means the segment passes through the panel).  margin: the smallest
    distance, inside or outside, from the panel's border of any crossing of the plane
    and of any reflection point on the panel (inf when the path meets neither)."""
    x0, (y0, y1), (z0, z1) = PANEL_X, PANEL_Y, PANEL_Z

    def inside(q):
        return min(q[1] - y0, y1 - q[1], q[2] - z0, z1 - q[2])

    nodes = [np.asarray(tx, float)] + [np.asarray(q, float) for q in pts] + [np.asarray(rx, float)]
    deepest, margin = -np.inf, np.inf
    for a, b in zip(nodes[:-1], nodes[1:]):
        if (a[0] - x0) * (b[0] - x0) < 0:
            d = inside(a + (x0 - a[0]) / (b[0] - a[0]) * (b - a))
            deepest = max(deepest, d)
            margin = min(margin, abs(d))
    for q, l in zip(pts, labels):
        if l == 6:
            margin = min(margin, abs(inside(q)))
    return deepest, margin
