"""Closed-form image method for reflections on axis-aligned bounded rectangles.

Independent of the oracle: mirror the TX across each plane of a sequence, back-trace
from the RX to get the reflection points, keep the sequence when every point lies on
its bounded rectangle and every segment meets its plane in order.  Section 2.3 names
the image method as the standard refinement for reflections.
"""
import itertools

import numpy as np


def box_room_planes(L, W, H):
    """(axis, value, label, extent lo, extent hi) of the six faces of [0,L]x[0,W]x[0,H].

    Labels follow the scene generator: x=0, x=L, y=0, y=W, floor, ceiling.
    """
    lo, hi = np.zeros(3), np.array([L, W, H], float)
    return [(0, 0.0, 0, lo, hi), (0, L, 1, lo, hi), (1, 0.0, 2, lo, hi), (1, W, 3, lo, hi),
            (2, 0.0, 4, lo, hi), (2, H, 5, lo, hi)]


def image_paths(planes, tx, rx, max_order):
    """{label sequence: (points (n,3), length)} of all valid specular paths."""
    tx = np.asarray(tx, float)
    rx = np.asarray(rx, float)
    out = {}
    for n in range(max_order + 1):
        for seq in itertools.product(range(len(planes)), repeat=n):
            if any(seq[i] == seq[i + 1] for i in range(n - 1)):
                continue
            imgs = [tx]
            for k in seq:
                a, v = planes[k][0], planes[k][1]
                q = imgs[-1].copy()
                q[a] = 2 * v - q[a]
                imgs.append(q)
            pts = [None] * n
            target = rx
            ok = True
            for k in range(n - 1, -1, -1):
                a, v, _, lo, hi = planes[seq[k]]
                src = imgs[k + 1]
                d = target - src
                if abs(d[a]) < 1e-12:
                    ok = False
                    break
                t = (v - src[a]) / d[a]
                if not (0 < t < 1):
                    ok = False
                    break
                q = src + t * d
                if not all(lo[i] - 1e-9 <= q[i] <= hi[i] + 1e-9 for i in range(3)):
                    ok = False
                    break
                pts[k] = q
                target = q
            if not ok:
                continue
            path = [tx] + pts + [rx]
            length = sum(np.linalg.norm(path[i + 1] - path[i]) for i in range(len(path) - 1))
            out[tuple(planes[k][2] for k in seq)] = (np.array(pts, float).reshape(-1, 3), length)
    return out


def corner_on_floor_mixed_path(tx, rx):
    """Closed form of the one path that mixes a floor reflection and an edge diffraction
    on the corner standing on a floor (edge on the z axis, floor z = 0, floor label 3,
    edge label 2): the law of reflection unfolds the floor, so the path is a straight
    line from the floor image of its first or last end, and the edge point is the
    Keller point of that line (Section 2.3: equal angles to the edge).

    The floor comes first when the TX is the lower end and last when the RX is; the
    other order would put the Keller point below the floor.  Returns (labels, types,
    points (2, 3), length).
    """
    tx, rx = np.asarray(tx, float), np.asarray(rx, float)
    floor_first = tx[2] < rx[2]
    a, b = (tx, rx) if floor_first else (rx, tx)       # a is reflected in the floor
    a_img = a * np.array([1.0, 1.0, -1.0])
    r_a, r_b = np.hypot(a_img[0], a_img[1]), np.hypot(b[0], b[1])
    D = np.array([0.0, 0.0, a_img[2] + (b[2] - a_img[2]) * r_a / (r_a + r_b)])
    F = a_img + (0.0 - a_img[2]) / (D[2] - a_img[2]) * (D - a_img)
    length = float(np.linalg.norm(D - a_img) + np.linalg.norm(b - D))
    if floor_first:
        return (3, 2), (0, 1), np.array([F, D]), length
    return (2, 3), (1, 0), np.array([D, F]), length
