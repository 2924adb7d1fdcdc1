"""Pins of the FP64 oracle against things other than itself.

Closed forms (image method, Keller diffraction point, LOS length), a library
distance transform, brute force on tiny scenes, Monte-Carlo geometry and the
paper's Table 1.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2402_13747_b300 import config, scenes
from tests import cases
from tests.imagemethod import box_room_planes, corner_on_floor_mixed_path, image_paths

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _exact_by_labels(P):
    out = {}
    for i in range(len(P["n"])):
        n = int(P["n"][i])
        key = (int(P["tx"][i]), int(P["rx"][i]), tuple(int(l) for l in P["label"][i][:n]))
        assert key not in out
        out[key] = (P["pts"][i][:n].copy(), float(P["length"][i]), tuple(int(t) for t in P["type"][i][:n]))
    return out


def test_config_defaults_match_table1():
    g = json.load(open(os.path.join(GOLDEN, "table1_params.json")))
    p = config.Params()
    assert p.voxel_size == g["voxel_size_m"]
    assert p.dv == g["voxel_division_factor"]
    assert p.kappa == g["coarse_path_duplicate_limit"]
    assert p.delta == g["convergence_threshold"]
    assert p.rho == g["refinement_iterations"]
    assert p.freq_hz == g["carrier_frequency_hz"]


@pytest.fixture(scope="module")
def tiny_run(room_tiny):
    p = config.params_for(room_tiny, grad_stop=1e-9)
    s, c, e = oracle.run(room_tiny, p)
    return room_tiny, p, s, c, e


def test_image_method_room_tiny(tiny_run):
    """Refined reflection paths equal the image method on the sampled box room (Section 2.3)."""
    sc, p, s, c, e = tiny_run
    ref = image_paths(box_room_planes(10.0, 10.0, 3.0), sc.tx[0], sc.rx[0], max_order=2)
    assert len(ref) == 25  # 1 LOS + 6 single + 18 double on the bounded faces
    got = _exact_by_labels(e.paths())
    assert set(k[2] for k in got) == set(ref)
    for (t, r, lab), (pts, length, types) in got.items():
        assert types == (0,) * len(lab)
        rp, rl = ref[lab]
        np.testing.assert_allclose(pts, rp, atol=1e-6)
        assert abs(length - rl) <= 1e-9 * rl
    # delay = length / c, with c = 299,792,458 m/s exactly (the SI definition of the metre)
    P = e.paths()
    for i in range(len(P["n"])):
        assert P["delay"][i] * 299_792_458.0 == pytest.approx(P["length"][i], rel=1e-15)


@pytest.mark.parametrize("flipped", [(0, 1, 2, 3, 4, 5), (0, 3, 4)])
def test_image_method_with_surfaces_facing_away(room_tiny, flipped):
    """The normals of a scan have no agreed side: a surface whose normals all face
    away from the room reflects the same rays (mirroring about n or -n is the same
    map), so turning whole faces around leaves the image method's 25 paths."""
    sc = room_tiny
    nrm = np.where(np.isin(sc.label, flipped)[:, None], -sc.nrm, sc.nrm).astype(np.float32)
    turned = scenes.Scene("room_tiny_turned", sc.xyz, nrm, sc.label, sc.material, tx=sc.tx, rx=sc.rx,
                          max_refl=2, max_diff=0)
    _, _, e = oracle.run(turned, config.params_for(turned, grad_stop=1e-9))
    ref = image_paths(box_room_planes(10.0, 10.0, 3.0), sc.tx[0], sc.rx[0], max_order=2)
    got = _exact_by_labels(e.paths())
    assert set(k[2] for k in got) == set(ref)
    for (t, r, lab), (pts, length, types) in got.items():
        np.testing.assert_allclose(pts, ref[lab][0], atol=1e-6)
        assert abs(length - ref[lab][1]) <= 1e-9 * ref[lab][1]


def test_reflection_limit_below_interaction_limit(room_tiny):
    """The depth limits count reflections and diffractions apart: at most one
    reflection and one diffraction (two interactions) on the box room, which has no
    edges, leaves LOS and the six single reflections of the image method."""
    p = config.params_for(room_tiny, max_refl=1, max_diff=1, grad_stop=1e-9)
    assert p.max_interactions == 2
    _, _, e = oracle.run(room_tiny, p)
    ref = image_paths(box_room_planes(10.0, 10.0, 3.0), room_tiny.tx[0], room_tiny.rx[0], max_order=1)
    got = _exact_by_labels(e.paths())
    assert set(k[2] for k in got) == set(ref) and len(ref) == 7


def test_rho_iterations_then_delta(room_tiny):
    """Section 2.3: once rho iterations are reached a path is valid only if its
    gradient norm is below delta.  Three iterations leave every reflection path of the
    box room far from stationary (gradient norms up to 0.3), so only LOS remains and
    every refined reflection path is reported not converged."""
    p = config.params_for(room_tiny, rho=3)
    _, _, e = oracle.run(room_tiny, p)
    P, A = e.paths(), e.paths(all_refined=True)
    assert [int(n) for n in P["n"]] == [0]
    refl = A["n"] > 0
    assert refl.sum() > 100
    assert all(oracle.STATUS[int(st)] == "not_converged" for st in A["status"][refl])
    assert np.all(A["grad"][refl] >= p.delta)


def test_label_dedup_keeps_the_shortest(room_tiny):
    """Label-based duplicate removal (Section 2.3) keeps, per TX/RX pair, only the
    shortest path of each interaction and label combination: with the walls x = 0 and
    y = 0 sharing label 0, each merged label sequence keeps its shortest image path
    (20 of the 25)."""
    sc = cases.room_with_merged_labels(room_tiny)
    _, _, e = oracle.run(sc, config.params_for(sc, grad_stop=1e-9))
    best = {}
    for seq, (pts, L) in image_paths(box_room_planes(10.0, 10.0, 3.0), sc.tx[0], sc.rx[0], max_order=2).items():
        k = tuple(0 if l == 2 else l for l in seq)
        if k not in best or L < best[k][1]:
            best[k] = (pts, L)
    got = _exact_by_labels(e.paths())
    assert len(best) == 20 and set(k[2] for k in got) == set(best)
    for (t, r, k), (pts, length, types) in got.items():
        np.testing.assert_allclose(pts, best[k][0], atol=1e-6)
        assert abs(length - best[k][1]) <= 1e-9 * best[k][1]


def test_los_miss_is_the_nearest_launch_axis(tiny_run):
    """The LOS coarse path keeps the smallest miss over the launch cones that see the
    RX: by brute force over the whole lattice, the smallest distance of the RX from a
    launch axis pointing its way."""
    sc, p, s, c, e = tiny_run
    C = c.paths()
    los = [i for i in range(len(C["n"])) if C["n"][i] == 0]
    assert len(los) == 1
    d = oracle.fibonacci(p.launch_count)
    r = sc.rx[0] - sc.tx[0]
    along = d @ r
    perp = np.linalg.norm(r[None, :] - along[:, None] * d, axis=1)
    assert C["miss"][los[0]] == pytest.approx(perp[along > 0].min(), abs=1e-12)


@pytest.mark.parametrize("z_tx,z_rx,on_edge", [(2.6, 3.36, True), (2.6, 3.44, False), (2.8, 3.36, False)])
def test_diffraction_leaving_its_edge_is_dropped(z_tx, z_rx, on_edge):
    """The wedge's edge ends at z = 3: a TX and an RX whose Keller point lies just
    beyond it (z = 3.02, 3.08) get a coarse diffraction path whose refinement walks off
    the edge, and no exact path; with the Keller point at z = 2.98 the path is there at
    its closed form."""
    sc = cases.tall_wedge(z_tx, z_rx)
    _, c, e = oracle.run(sc, config.params_for(sc, grad_stop=1e-10))
    assert len(c.paths()["n"]) == 1
    P, A = e.paths(), e.paths(all_refined=True)
    if on_edge:
        assert len(P["n"]) == 1
        np.testing.assert_allclose(P["pts"][0][0], [0.0, 0.0, (z_tx + z_rx) / 2.0], atol=1e-6)
    else:
        assert len(P["n"]) == 0 and oracle.STATUS[int(A["status"][0])] == "off_edge"


def test_image_method_with_an_occluding_panel(room_tiny):
    """The box room with a free-standing 1.8 x 2 m panel (label 6) at x = 4 between TX
    and RX: the image-method paths whose segments all pass the panel at least 0.3 m
    outside its border are found at their image points, and none whose segment crosses
    the panel is found (LOS among them).  Paths within 0.3 m of the panel's border are
    left out of the comparison: the point set's implicit surface reaches a little past its
    last row."""
    x0, (y0, y1), (z0, z1) = cases.PANEL_X, cases.PANEL_Y, cases.PANEL_Z
    sc = cases.room_with_panel(room_tiny)
    _, _, e = oracle.run(sc, config.params_for(sc, grad_stop=1e-9))
    planes = box_room_planes(10.0, 10.0, 3.0) + [(0, x0, 6, np.array([x0, y0, z0]), np.array([x0, y1, z1]))]
    ref = image_paths(planes, sc.tx[0], sc.rx[0], max_order=2)

    def inside(q):            # signed distance of a point of the plane x = x0 inside the panel
        return min(q[1] - y0, y1 - q[1], q[2] - z0, z1 - q[2])

    clear, blocked, near = {}, set(), set()
    for seq, (pts, L) in ref.items():
        nodes = [sc.tx[0]] + list(pts) + [sc.rx[0]]
        cross = []
        for a, b in zip(nodes[:-1], nodes[1:]):
            if (a[0] - x0) * (b[0] - x0) < 0:
                cross.append(inside(a + (x0 - a[0]) / (b[0] - a[0]) * (b - a)))
        on_panel = [inside(pts[k]) for k in range(len(seq)) if seq[k] == 6]
        if any(d > 0 for d in cross):
            blocked.add(seq)
        elif all(d < -0.3 for d in cross) and all(d > 0.3 for d in on_panel):
            clear[seq] = (pts, L)
        else:
            near.add(seq)
    assert () in blocked and len(clear) >= 8 and len(blocked) >= 4
    got = {k[2]: v for k, v in _exact_by_labels(e.paths()).items()}
    assert not blocked & set(got)
    assert set(clear) <= set(got)
    for k, (pts, length, types) in got.items():
        if k in clear:
            np.testing.assert_allclose(pts, clear[k][0], atol=1e-6)
            assert abs(length - clear[k][1]) <= 1e-9 * clear[k][1]
        elif k not in near:   # a panel reflection the image method bounds out: within the border's reach
            kp = [q for q, l in zip(pts, k) if l == 6]
            assert kp and all(abs(inside(q)) < 0.3 for q in kp), k


def test_paths_move_with_the_scene(tiny_run):
    """Nothing depends on where the scene sits: the box room, its TX and its RX shifted
    by whole voxels (1, -2, 0.5) m give the same paths, each point shifted by the same
    amount and each length unchanged."""
    rt, p, s, c, e = tiny_run
    shift = np.array([1.0, -2.0, 0.5])
    moved = scenes.Scene("room_tiny_moved", (rt.xyz.astype(np.float64) + shift).astype(np.float32), rt.nrm,
                         rt.label, rt.material, tx=rt.tx + shift, rx=rt.rx + shift, max_refl=2, max_diff=0)
    _, _, e2 = oracle.run(moved, config.params_for(moved, grad_stop=1e-9))
    a, b = _exact_by_labels(e.paths()), _exact_by_labels(e2.paths())
    assert a.keys() == b.keys() and len(a) == 25
    for k in a:
        np.testing.assert_allclose(b[k][0], a[k][0] + shift, atol=1e-7)
        assert b[k][1] == pytest.approx(a[k][1], rel=1e-12)


def test_image_method_room_tiny_paper_launch(room_tiny):
    """The paper's own transmission phase (a ray toward every IE and RX, Section 2.2.2)
    finds the same 25 image-method paths in the sampled box room."""
    p = config.params_for(room_tiny, grad_stop=1e-9, launch_mode=1)
    s, c, e = oracle.run(room_tiny, p)
    ref = image_paths(box_room_planes(10.0, 10.0, 3.0), room_tiny.tx[0], room_tiny.rx[0], max_order=2)
    got = _exact_by_labels(e.paths())
    assert set(k[2] for k in got) == set(ref)
    for (t, r, lab), (pts, length, types) in got.items():
        rp, rl = ref[lab]
        np.testing.assert_allclose(pts, rp, atol=1e-6)
        assert abs(length - rl) <= 1e-9 * rl
    assert got[(0, 0, ())][1] == pytest.approx(math.sqrt(25 + 9), rel=1e-15)   # LOS


def test_los_length(tiny_run):
    sc, p, s, c, e = tiny_run
    got = _exact_by_labels(e.paths())
    assert got[(0, 0, ())][1] == pytest.approx(math.sqrt(25 + 9), rel=1e-15)


@pytest.mark.parametrize("launch_mode", [0, 1])
@pytest.mark.parametrize("z_tx,z_rx", [(0.5, 2.5), (0.5, 2.0), (2.2, 0.7)])
def test_keller_point_on_sampled_wedge(z_tx, z_rx, launch_mode):
    """Diffraction at an exterior edge: the refined point is the closed-form Keller point.

    TX and RX are both sqrt(10) m from the edge line, so the point divides the
    height difference in the ratio r1/(r1+r2) = 1/2; the path obeys the equal-angle law.
    """
    sc = scenes.wedge(z_tx=z_tx, z_rx=z_rx)
    p = config.params_for(sc, grad_stop=1e-10, launch_mode=launch_mode)
    s, c, e = oracle.run(sc, p)
    P = e.paths()
    assert len(P["n"]) == 1
    assert P["n"][0] == 1 and P["type"][0][0] == 1 and P["label"][0][0] == 2
    r1 = r2 = math.sqrt(10.0)
    z = z_tx + (z_rx - z_tx) * r1 / (r1 + r2)
    np.testing.assert_allclose(P["pts"][0][0], [0.0, 0.0, z], atol=1e-6)
    L = math.sqrt(r1 ** 2 + (z - z_tx) ** 2) + math.sqrt(r2 ** 2 + (z_rx - z) ** 2)
    assert P["length"][0] == pytest.approx(L, rel=1e-9)
    ein = P["pts"][0][0] - sc.tx[0]
    eout = sc.rx[0] - P["pts"][0][0]
    w = np.array([0, 0, 1.0])
    assert abs(ein @ w / np.linalg.norm(ein) - eout @ w / np.linalg.norm(eout)) < 1e-6


@pytest.mark.parametrize("z_tx,z_rx", [(0.8, 2.0), (1.0, 2.2), (0.6, 1.8), (2.0, 0.8), (1.8, 0.6)])
def test_reflection_and_diffraction_closed_form(z_tx, z_rx):
    """Paths mixing both interaction kinds, in either order: the floor point and the
    edge point are those of the floor image of the lower end joined to the other end
    through its Keller point, each obeys its own law (mirror reflection; equal angles
    to the edge), and the order whose Keller point would lie below the floor is absent."""
    sc = scenes.wedge_on_floor(z_tx=z_tx, z_rx=z_rx)
    p = config.params_for(sc, grad_stop=1e-10)
    _, _, e = oracle.run(sc, p)
    got = _exact_by_labels(e.paths())
    tx, rx = sc.tx[0], sc.rx[0]
    labels, types, want, L = corner_on_floor_mixed_path(tx, rx)
    pts, length, got_types = got[(0, 0, labels)]
    assert got_types == types
    np.testing.assert_allclose(pts, want, atol=1e-6)
    assert length == pytest.approx(L, rel=1e-9)
    assert (0, 0, labels[::-1]) not in got
    nodes = [tx, pts[0], pts[1], rx]
    d = [(nodes[k + 1] - nodes[k]) / np.linalg.norm(nodes[k + 1] - nodes[k]) for k in range(3)]
    kf = types.index(0)                   # floor: mirror law about z
    np.testing.assert_allclose(d[kf + 1], d[kf] * np.array([1.0, 1.0, -1.0]), atol=1e-6)
    kd = types.index(1)                   # edge (z axis): equal angles
    assert abs(d[kd][2] - d[kd + 1][2]) < 1e-6
    # the pure diffraction is there too, at the Keller point of TX and RX themselves
    dpts, dlen, dtypes = got[(0, 0, (2,))]
    np.testing.assert_allclose(dpts[0], [0.0, 0.0, (z_tx + z_rx) / 2.0], atol=1e-6)


def _tiny_occluder_scene():
    X, Y, Z = np.eye(3)
    parts = [scenes.plane_patch([0.5, 0.5, 1.0], X, Y, 2.0, 2.0, 0.1, [0, 0, 1], 0),
             scenes.plane_patch([1.5, 0.0, 0.0], Y, Z, 3.0, 2.0, 0.1, [1, 0, 0], 1),
             scenes.plane_patch([0.0, 2.2, 0.5], X, Z, 1.2, 1.5, 0.1, [0, -1, 0], 2)]
    xyz, nrm, lab, mat = scenes.merge_clouds(parts)
    assert xyz.shape[0] < 2000
    return scenes.Scene("tiny", xyz, nrm, lab, mat)


def test_visibility_traversal_matches_brute_force():
    """The voxel traversal visits exactly the voxels a brute-force slab test finds."""
    sc = _tiny_occluder_scene()
    s = oracle.Scene.from_scene(sc, config.Params())
    rng = np.random.default_rng(7)
    lo = s.origin + 0.3
    hi = s.origin + s.dims * 0.5 - 0.3
    n_block = 0
    for _ in range(400):
        a = lo + (hi - lo) * rng.random(3)
        b = lo + (hi - lo) * rng.random(3)
        v1 = s.visible(a, b)
        v2 = s.visible(a, b, brute=True)
        assert v1 == v2
        n_block += not v1
    assert 40 < n_block < 360


def test_visibility_closed_form_plane_patch():
    """Segments crossing the interior of a sampled plane patch are occluded; others are not."""
    sc = _tiny_occluder_scene()
    s = oracle.Scene.from_scene(sc, config.Params())
    rng = np.random.default_rng(3)
    for _ in range(100):
        x, y = 0.8 + 1.4 * rng.random(2)   # well inside the z=1 patch [0.5,2.5]^2, left of x=1.5 wall
        x = min(x, 1.3)
        a = np.array([x, y, 0.4])
        b = np.array([x + 0.05, y - 0.05, 1.6])
        if 2.0 < y < 2.4:
            continue
        assert not s.visible(a, b)
        c = np.array([x, y, 1.3])
        d = np.array([x - 0.2, y + 0.1, 1.8])
        if y + 0.1 < 2.3:
            assert s.visible(c, d)


def test_visibility_self_hit_rule():
    """Hits near a path node (Sections 2.2.4, 2.3), with the rule read for them: a hit
    closer than r = h_s sqrt(3) to a node is ignored when it lies on that node's own
    label (a reflection) or on any label (a diffraction), and blocks otherwise.  A
    floor (label 0) with a 0.3 m high wall (label 1) at x = 0.2: the ray from the floor
    point F = 0 to (2, 0, 1) crosses the wall 0.22 m from F; the ray from (0, 0, 0.1)
    to (0.2, 0, -0.5) crosses the floor 0.03 m from its start, the ray to
    (-2.9, 0, -0.5) 0.49 m from it (beyond r)."""
    X, Y, Z = np.eye(3)
    parts = [scenes.plane_patch([-3, -2, 0], X, Y, 6.0, 4.0, 0.05, [0, 0, 1], 0),
             scenes.plane_patch([0.2, -2, 0], Y, Z, 4.0, 0.3, 0.05, [-1, 0, 0], 1)]
    xyz, nrm, lab, mat = scenes.merge_clouds(parts)
    sc = scenes.Scene("floor_low_wall", xyz, nrm, lab, mat, region=np.array([[-3.0, -2, -1], [3.0, 2, 1.5]]))
    p = config.Params()
    assert 0.22 < p.ignore_dist < 0.49
    s = oracle.Scene.from_scene(sc, p)
    NONE, LABEL, ANY, NL = 0, 1, 2, oracle.NONE_LABEL

    def vis(a, b, mode, label):   # the rule at either end of the ray
        v = s.visible(a, b, mode, label)
        assert s.visible(b, a, NONE, NL, mode, label) == v
        return v

    F, R = np.zeros(3), np.array([2.0, 0.0, 1.0])
    assert not vis(F, R, LABEL, 0)        # another surface near a reflection blocks
    assert vis(F, R, LABEL, 1)            # ... and is ignored on the node's own label
    assert vis(F, R, ANY, 0)              # ... and near a diffraction on any label
    A, near, far = np.array([0, 0, 0.1]), np.array([0.2, 0, -0.5]), np.array([-2.9, 0, -0.5])
    assert not vis(A, near, NONE, NL)
    assert vis(A, near, LABEL, 0) and vis(A, near, ANY, 0)
    assert not vis(A, near, LABEL, 1)
    for mode, label in ((NONE, NL), (LABEL, 0), (ANY, 0)):
        assert not vis(A, far, mode, label)   # beyond r nothing is ignored


def test_march_field_is_chessboard_distance(room_tiny):
    """March distance (Section 2.2.4) equals scipy's chessboard distance transform."""
    from scipy import ndimage
    s = oracle.Scene.from_scene(room_tiny, config.Params())
    cells = s.cells()
    nx, ny, nz = (int(d) for d in s.dims)
    occ = (cells["count"] > 0).reshape(nz, ny, nx)
    ref = ndimage.distance_transform_cdt(~occ, metric="chessboard")
    np.testing.assert_array_equal(cells["march"].reshape(nz, ny, nx), np.minimum(ref, 255))


def test_voxel_membership_by_integer_arithmetic():
    """Each point lands in the IE of its (subvoxel, label); IEs ordered by voxel, subvoxel, label."""
    rng = np.random.default_rng(11)
    p = config.Params()
    hs = p.h_s
    # cloud whose bounds fix the origin at -0.5: points strictly inside subvoxels
    g = rng.integers(2, 14, size=(600, 3))
    off = rng.uniform(0.2, 0.8, size=(600, 3)) * hs
    org = -0.5
    xyz = org + g * hs + off
    xyz = np.vstack([xyz, [[0.0, 0.0, 0.0], [3.0, 3.0, 3.0]]])
    g = np.vstack([g, [[2, 2, 2], [14, 14, 14]]])
    lab = rng.integers(0, 3, size=xyz.shape[0]).astype(np.uint32)
    nrm = np.tile([0, 0, 1.0], (xyz.shape[0], 1))
    s = oracle.Scene(xyz, nrm, lab, np.zeros(xyz.shape[0], np.uint8), np.zeros((0, 12)),
                     np.zeros(0, np.uint32), p)
    np.testing.assert_allclose(s.origin, [org] * 3)
    I = s.ies()
    groups = {}
    for i in range(xyz.shape[0]):
        groups.setdefault((tuple(g[i]), int(lab[i])), []).append(i)
    assert s.n_ie == len(groups)
    dims = s.dims
    for k in range(s.n_ie):
        key = (tuple(int(v) for v in I["gs"][k]), int(I["label"][k]))
        members = groups[key]
        assert I["prange"][k][1] == len(members)
        np.testing.assert_allclose(I["rp"][k], xyz[members].astype(np.float32).astype(np.float64).mean(0),
                                   atol=1e-12)
        vx, vy, vz = (int(v) // 2 for v in I["gs"][k])
        assert I["cell"][k] == (vz * dims[1] + vy) * dims[0] + vx
    order = [(int(I["cell"][k]), tuple(int(v) % 2 for v in I["gs"][k][::-1]), int(I["label"][k]))
             for k in range(s.n_ie)]
    assert order == sorted(order)


def test_sdf_on_exact_plane(room_tiny):
    """Eq. 1 on coplanar points with exact normals is the plane distance."""
    s = oracle.Scene.from_scene(room_tiny, config.Params())
    I = s.ies()
    floor = np.where((I["label"] == 4) & (I["prange"][:, 1] >= 9))[0][:20]
    rng = np.random.default_rng(0)
    for k in floor:
        for _ in range(5):
            x = I["bbc"][k] + rng.uniform(-0.15, 0.15, 3)
            f, n = s.sdf(k, x)
            assert f == pytest.approx(x[2], abs=1e-12)
            np.testing.assert_allclose(n, [0, 0, 1], atol=1e-12)
        du = np.array([0.3, -0.2, -1.0])
        du /= np.linalg.norm(du)
        target = I["bbc"][k] + np.array([0.05, 0.02, 0.0])   # on the patch
        P = target - 2.0 * du                                 # 2 m back along the ray
        t = s.sdf_hit(k, P, du)
        t_ref = -P[2] / du[2]
        assert t is not None and t == pytest.approx(t_ref, abs=1e-9)


def test_sdf_weights_two_points_closed_form():
    """Eq. 1's weighted average with the Gaussian weights exp(-|x - p_i|^2 / sigma^2)
    (the Adamson-Alexa weights the paper cites) on two points p -/+ h z with a shared
    normal z: the weight ratio is exp(4 z h / sigma^2) at height z above their
    midpoint, whatever the lateral offset, so the weighted position sits at
    h tanh(2 z h / sigma^2) and f = z - h tanh(2 z h / sigma^2).  Any other weight
    profile (a dropped square, another width) moves f off this curve."""
    p = config.Params()
    c, h = np.array([1.125, 1.125, 1.125]), 0.0625      # exact in FP32, one subvoxel
    xyz = np.array([c - [0, 0, h], c + [0, 0, h]], np.float32)
    nrm = np.array([[0, 0, 1], [0, 0, 1]], np.float32)
    sc = scenes.Scene("two_points", xyz, nrm, np.zeros(2, np.uint32), np.zeros(2, np.uint8))
    s = oracle.Scene.from_scene(sc, p)
    I = s.ies()
    assert len(I["label"]) == 1 and I["prange"][0, 1] == 2
    s2 = p.sdf_sigma ** 2
    for z in (-0.1, -0.04, -0.01, 0.0, 0.02, 0.07, 0.1):
        for lat in ((0.0, 0.0), (0.06, -0.03)):
            x = c + np.array([lat[0], lat[1], z])
            f, n = s.sdf(0, x)
            assert f == pytest.approx(z - h * math.tanh(2 * z * h / s2), abs=1e-12)
            np.testing.assert_allclose(n, [0, 0, 1], atol=1e-12)


def test_sdf_hit_marches_one_subvoxel_diameter(room_tiny):
    """Section 2.2.1: the march covers a segment one subvoxel diameter long (h_s sqrt 3)
    centred on the projection of the point set's bounding-box centre onto the ray.
    Rays 10 degrees above a floor entity's plane meet it 0.049 to 0.197 m along the ray
    from that projection -- found, at the exact plane crossing -- or 0.246 and 0.295 m
    from it, beyond the half length of 0.2165 m -- no intersection."""
    p = config.Params()
    s = oracle.Scene.from_scene(room_tiny, p)
    I = s.ies()
    k = np.where((I["label"] == 4) & (I["prange"][:, 1] >= 9))[0][0]
    th = math.radians(10.0)
    d = np.array([math.cos(th), 0.0, -math.sin(th)])
    for delta, found in ((0.05, True), (0.15, True), (0.2, True), (0.25, False), (0.3, False)):
        assert (delta * math.cos(th) < 0.5 * p.voxel_size / p.dv * math.sqrt(3.0)) == found
        P = I["bbc"][k] + np.array([delta, 0.0, 0.0]) - 2.0 * d     # 2 m back from the plane crossing
        t = s.sdf_hit(k, P, d)
        if found:
            assert t == pytest.approx(2.0, abs=1e-9)
        else:
            assert t is None


def test_cone_sphere_against_sampling():
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(300):
        apex = rng.normal(size=3)
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        alpha = rng.uniform(0.01, 0.3)
        c = apex + rng.normal(size=3) * 2.0
        r = rng.uniform(0.05, 0.6)
        u = rng.normal(size=(20000, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        pts = c + r * u * rng.random((20000, 1)) ** (1 / 3)
        pts = np.vstack([pts, c + r * u])
        v = pts - apex
        ang = np.arccos(np.clip(v @ axis / np.linalg.norm(v, axis=1), -1, 1))
        amin = ang.min()
        got = oracle.cone_sphere(apex, axis, alpha, c, r)
        if amin < alpha - 2e-3:
            assert got
            checked += 1
        elif amin > alpha + 2e-2:
            assert not got
            checked += 1
    assert checked > 250


def test_fibonacci_lattice():
    n = config.Params().launch_count
    assert n == 165012  # round(4 pi / (0.5 deg)^2)
    d = oracle.fibonacci(n)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    # equal area: z is uniform on [-1, 1]
    hist, _ = np.histogram(d[:, 2], bins=20, range=(-1, 1))
    assert hist.min() >= n / 20 - 2 and hist.max() <= n / 20 + 2
    # the lattice's construction: by Archimedes' hat-box theorem, zones of equal height
    # on the unit sphere have equal area, and each point sits at the middle height of
    # one of N such zones (so the set is symmetric about z = 0, nothing at the poles);
    # successive points turn about z by the golden angle pi (3 - sqrt 5)
    z = np.sort(d[:, 2])
    np.testing.assert_allclose(np.diff(z), 2.0 / n, atol=1e-12)
    assert z[-1] == pytest.approx(1.0 - 1.0 / n, abs=1e-15) and z[0] == pytest.approx(-1.0 + 1.0 / n, abs=1e-15)
    np.testing.assert_allclose(d.mean(axis=0), 0.0, atol=1e-5)
    turn = np.mod(np.diff(np.arctan2(d[:, 1], d[:, 0])), 2 * math.pi)
    np.testing.assert_allclose(turn, math.pi * (3.0 - math.sqrt(5.0)), atol=1e-9)
    rng = np.random.default_rng(1)
    sample = rng.integers(0, n, 100)
    delta = math.radians(0.5)
    for i in sample:
        cosang = d @ d[i]
        cosang[i] = -2
        nn = math.acos(min(1.0, cosang.max()))
        assert 0.5 * delta < nn < 1.2 * delta


def test_orthonormal_basis():
    rng = np.random.default_rng(2)
    ns = [np.array([0, 0, -1.0]), np.array([0, 0, 1.0]), np.array([1.0, 0, 0])]
    ns += [v / np.linalg.norm(v) for v in rng.normal(size=(50, 3))]
    for n in ns:
        u, v = oracle.onb(n)
        M = np.stack([u, v, n])
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-12)
        np.testing.assert_allclose(np.cross(u, v), n, atol=1e-12)


def test_fresnel_removes_label_split_duplicates():
    """Section 2.3: a reflection near a label boundary is found under two labels and the
    first-Fresnel-zone step keeps one.  Floor split at x = 4.5, through three specular points."""
    sc = scenes.room_tiny()
    lab = sc.label.copy()
    lab[(lab == 4) & (sc.xyz[:, 0] >= 4.5)] = 6
    sc2 = scenes.Scene("split", sc.xyz, sc.nrm, lab, sc.material, tx=sc.tx, rx=sc.rx, max_refl=2)
    p = config.params_for(sc2, grad_stop=1e-9)
    s, c, e = oracle.run(sc2, p)
    A = e.paths(True)
    valid_single = {int(A["label"][i][0]) for i in range(len(A["n"])) if A["status"][i] == 0 and A["n"][i] == 1}
    assert {4, 6} <= valid_single                # the floor reflection under both labels
    P = e.paths()
    got = _exact_by_labels(P)
    assert len(got) == 25                        # ... but only once after Fresnel removal
    ref = image_paths(box_room_planes(10.0, 10.0, 3.0), sc.tx[0], sc.rx[0], max_order=2)
    pts_sorted = sorted(round(v[1], 6) for v in got.values())
    assert pts_sorted == sorted(round(v[1], 6) for v in ref.values())


def _paths(tx, rx, chains, types):
    """Exact-path arrays for given interaction points (one list per path)."""
    m = len(chains)
    out = dict(tx=np.zeros(m, np.int32), rx=np.zeros(m, np.int32), n=np.zeros(m, np.int32),
               type=np.zeros((m, oracle.MAXI), np.int32), label=np.zeros((m, oracle.MAXI), np.uint32),
               pts=np.zeros((m, oracle.MAXI, 3)), length=np.zeros(m))
    for i, (pts, t) in enumerate(zip(chains, types)):
        nodes = [tx] + list(pts) + [rx]
        out["n"][i] = len(pts)
        out["type"][i][:len(pts)] = t
        out["label"][i][:len(pts)] = np.arange(len(pts)) + 10 * i   # distinct label sequences
        out["pts"][i][:len(pts)] = pts
        out["length"][i] = sum(np.linalg.norm(np.subtract(b, a)) for a, b in zip(nodes[:-1], nodes[1:]))
    return out


def test_fresnel_zone_radius():
    """Section 2.3: a later path duplicates a kept one of the same interaction types when
    each of its points lies within the kept path's first Fresnel zone radius
    r_k = sqrt(lambda a_k b_k / (a_k + b_k)), a_k the kept path's length from the TX to
    its k-th point and b_k the rest.  Points at 0.99 r are removed, at 1.01 r kept."""
    lam = 299792458.0 / 60e9
    tx, rx = np.array([0.0, 0.0, 1.0]), np.array([10.0, 0.0, 1.0])
    y = np.array([0.0, 1.0, 0.0])
    # one reflection: a = b = sqrt(26)
    A1 = [np.array([5.0, 0.0, 0.0])]
    r = math.sqrt(lam * math.sqrt(26.0) / 2.0)
    chains = [A1, [A1[0] + 0.99 * r * y], [A1[0] - 1.01 * r * y], [A1[0] + 0.5 * r * y]]
    keep = oracle.fresnel_dedup(_paths(tx, rx, chains, [[0], [0], [0], [1]]), tx[None], lam)
    assert keep.tolist() == [1, 0, 1, 1]          # the diffraction at the same place is another chain
    # two interactions, asymmetric: a_k accumulates along the kept path
    P1, P2 = np.array([3.0, 0.0, 0.0]), np.array([7.0, 0.0, 3.0])
    a1 = np.linalg.norm(P1 - tx)
    a2 = a1 + np.linalg.norm(P2 - P1)
    L = a2 + np.linalg.norm(rx - P2)
    r1, r2 = (math.sqrt(lam * a * (L - a) / L) for a in (a1, a2))
    chains = [[P1, P2],
              [P1 + 0.99 * r1 * y, P2 + 0.99 * r2 * y],
              [P1 + 0.99 * r1 * y, P2 + 1.01 * r2 * y],
              [P1 - 1.01 * r1 * y, P2]]
    keep = oracle.fresnel_dedup(_paths(tx, rx, chains, [[0, 0]] * 4), tx[None], lam)
    assert keep.tolist() == [1, 0, 1, 1]
    # the shorter of two duplicates is the one kept, whatever the input order
    keep = oracle.fresnel_dedup(_paths(tx, rx, [[P1 + 0.5 * r1 * y, P2], [P1, P2]], [[0, 0]] * 2), tx[None], lam)
    assert keep.tolist() == [0, 1]


def test_kappa_keeps_nearest_axis(tiny_run):
    """kappa = 1 keeps, per (TX, RX, label sequence), the coarse path with the smallest miss."""
    sc, p, s, c, e = tiny_run
    full = c.paths()
    c1 = oracle.Scene.from_scene(sc, p.replace(kappa=1)).trace(sc.tx, sc.rx).paths()
    best = {}
    for i in range(len(full["n"])):
        k = oracle.path_key(full["type"][i], full["label"][i], full["n"][i])
        if k not in best or full["miss"][i] < best[k]:
            best[k] = full["miss"][i]
    got = {oracle.path_key(c1["type"][i], c1["label"][i], c1["n"][i]): c1["miss"][i]
           for i in range(len(c1["n"]))}
    assert len(got) == len(c1["n"])
    assert got.keys() == best.keys()
    for k in got:
        assert got[k] == pytest.approx(best[k], abs=1e-12)


def test_stationarity_on_noisy_room():
    """Every refined path is stationary: at a reflection e_in + e_out is parallel to the
    surface normal of Eq. 1 there; at a diffraction the equal-angle law holds and the
    point lies on its edge."""
    full = scenes.room_noisy(n_tx=1, n_rx=2)
    sc = full.with_pairs(full.tx[:1], full.rx[:2])
    p = config.params_for(sc, max_refl=1, max_diff=1, n_launch=20000)
    s, c, e = oracle.run(sc, p)
    P = e.paths()
    assert len(P["n"]) >= 3
    I = s.ies()
    n_checked = 0
    for i in range(len(P["n"])):
        n = int(P["n"][i])
        nodes = [sc.tx[P["tx"][i]]] + list(P["pts"][i][:n]) + [sc.rx[P["rx"][i]]]
        for k in range(n):
            x = nodes[k + 1]
            ein = (x - nodes[k]) / np.linalg.norm(x - nodes[k])
            eout = (x - nodes[k + 2]) / np.linalg.norm(x - nodes[k + 2])
            ie = int(P["ie"][i][k])
            if P["type"][i][k] == 0:
                # the point lies on its label's Eq. 1 surface and e_in + e_out is parallel to
                # that surface's normal there (the reflection law)
                f, nn = s.sdf_label(int(P["label"][i][k]), x)
                assert f is not None and abs(f) < 1e-4
                assert np.linalg.norm(np.cross(ein + eout, nn)) < 1e-4
            else:
                e_ = sc.edges[I["edge"][ie]]
                p0, p1 = e_[:3], e_[3:6]
                w = (p1 - p0) / np.linalg.norm(p1 - p0)
                assert abs((ein + eout) @ w) < 2e-4
                off = (x - p0) - ((x - p0) @ w) * w
                assert np.linalg.norm(off) < 1e-9
            n_checked += 1
    assert n_checked >= 2


def test_label_surface_is_plane_distance_and_continuous(room_tiny):
    """Eq. 1 on a label's nearby points: the plane distance on an exact plane, across
    subvoxel boundaries; on a noisy wall it varies smoothly (no jumps at boundaries)."""
    s = oracle.Scene.from_scene(room_tiny, config.Params())
    rng = np.random.default_rng(4)
    for _ in range(50):
        x = np.array([rng.uniform(1, 9), rng.uniform(1, 9), rng.uniform(-0.2, 0.2)])
        f, n = s.sdf_label(4, x)
        assert f == pytest.approx(x[2], abs=1e-12)
        np.testing.assert_allclose(n, [0, 0, 1], atol=1e-12)
    noisy = scenes.room_noisy(n_tx=1, n_rx=1)
    s2 = oracle.Scene.from_scene(noisy, config.Params())
    ys = np.linspace(2.0, 4.0, 801)          # crosses 8 subvoxel boundaries, 2.5 mm steps
    fs = np.array([s2.sdf_label(0, np.array([0.01, y, 1.3]))[0] for y in ys])
    assert np.all(np.isfinite(fs))
    assert np.max(np.abs(np.diff(fs))) < 1e-3   # no step at subvoxel faces


def test_rx_on_the_tx_gives_normal_incidence_images(room_tiny):
    """Degenerate pair: the RX at the TX.  The exact paths are the LOS of length 0 and
    the six normal-incidence reflections, of length twice the distance to each face
    (image method); a duplicated RX gets the same set."""
    tx = room_tiny.tx[0]
    sc = room_tiny.with_pairs(room_tiny.tx, np.vstack([tx, room_tiny.rx[0], room_tiny.rx[0]]))
    p = config.params_for(sc, max_refl=1, grad_stop=1e-9)
    _, _, e = oracle.run(sc, p)
    P = e.paths()
    on = np.sort(P["length"][P["rx"] == 0])
    want = np.sort([0.0] + [2 * d for d in (tx[0], 10 - tx[0], tx[1], 10 - tx[1], tx[2], 3 - tx[2])])
    np.testing.assert_allclose(on, want, atol=1e-6)
    a = np.sort(P["length"][P["rx"] == 1])
    b = np.sort(P["length"][P["rx"] == 2])
    np.testing.assert_array_equal(a, b)


# ------------------------------------------------- the march's secant placement
def _sheet_pair(zs, lo, hi, spacing):
    """Horizontal sheets of one label with normals +z at heights zs, on one lattice
    (all coordinates exact in FP32)."""
    g = np.arange(lo, hi + 1e-12, spacing)
    X, Y = np.meshgrid(g, g, indexing="ij")
    xyz = np.vstack([np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1) for z in zs]).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (xyz.shape[0], 1))
    return scenes.Scene("sheet_pair", xyz, nrm, np.zeros(xyz.shape[0], np.uint32), np.zeros(xyz.shape[0], np.uint8))


def _march_closed_form(f, u0, cos_t, length, eps):
    """The |f| march of Section 2.2.1 on a closed-form f(u), u = u0 - t cos_t: step
    t += |f| until |f| < eps or the sign of f changes, then place the hit by the
    secant through the last two march points.  Returns (branch, t)."""
    t, fv = 0.0, f(u0)
    for _ in range(64):
        if abs(fv) < eps:
            return "near_zero", t
        tn = t + abs(fv)
        if tn > length:
            return "miss", None
        fn = f(u0 - tn * cos_t)
        if (fn < 0) != (fv < 0):
            return "secant", t - fv * (tn - t) / (fn - fv)
        t, fv = tn, fn
    return "budget", None


def test_sdf_hit_secant_after_a_sign_change():
    """Two sheets 2h apart inside one subvoxel with shared normals: Eq. 1 gives
    f = u - h tanh(2uh/sigma^2) at height u above their middle plane, whatever the
    lateral position (both sheets share one lattice, so the lateral weight sums
    cancel).  With h > sigma the slope of f exceeds 1 along a ray 70 degrees off the
    normal, so the |f| march steps over the middle zero and the hit is the secant
    through the two march points around it.  The closed-form f, marched by the same
    rule, fixes that point."""
    p = config.Params(sdf_sigma=0.05)
    c, h = 0.375, 0.09375
    s = oracle.Scene.from_scene(_sheet_pair([c - h, c + h], 0.25, 0.4375, 0.0625), p)
    I = s.ies()
    assert len(I["label"]) == 1 and I["prange"][0, 1] == 32
    f = lambda u: u - h * math.tanh(2.0 * u * h / p.sdf_sigma ** 2)  # noqa: E731
    th = math.radians(70.0)
    d = np.array([math.sin(th), 0.0, -math.cos(th)])
    half = 0.5 * p.voxel_size / p.dv * math.sqrt(3.0)
    assert (2 * h * h / p.sdf_sigma ** 2 - 1.0) * math.cos(th) > 1.0 and half * math.cos(th) < h
    branch, t_ref = _march_closed_form(f, half * math.cos(th), math.cos(th), 2 * half, p.sdf_eps)
    assert branch == "secant"
    bbc = I["bbc"][0]
    np.testing.assert_allclose(bbc, [0.34375, 0.34375, c], atol=1e-7)
    for lat in (0.0, 0.05):
        P = bbc + np.array([0.0, lat, 0.0]) - 2.0 * d
        t = s.sdf_hit(0, P, d)
        assert t == pytest.approx(2.0 - half + t_ref, abs=1e-9)


def _sheet_pair_surface():
    """The sheet pair 2h = 0.375 m apart across three subvoxel layers (one label,
    default sigma) and its closed-form Eq. 1: f = u - h tanh(2uh/sigma^2), odd in u,
    wherever the 3x3x3 block of the evaluated point holds both sheets."""
    p = config.Params()
    c, h = 0.375, 0.1875
    s = oracle.Scene.from_scene(_sheet_pair([c - h, c + h], 0.0, 2.0, 0.0625), p)
    f = lambda u: u - h * math.tanh(2.0 * u * h / p.sdf_sigma ** 2)  # noqa: E731
    return p, c, h, s, f


def test_reprojection_secant_lands_near_the_middle_plane():
    """The re-projection of Section 2.3 on the sheet pair: a ray 60 degrees off the
    normal toward a target 0.01 m above the middle plane, where |f| = 0.034 m is not
    near zero, so the segment is marched from its near end; the march oversteps the
    middle zero (the slope of f along the ray exceeds 1) and the secant places the hit
    at the closed-form march's point, 2.3 mm from the plane (the zero of f by symmetry;
    the secant's error on the curved f), with normal +z."""
    p, c, h, s, f = _sheet_pair_surface()
    th = math.radians(60.0)
    d = np.array([math.sin(th), 0.0, -math.cos(th)])
    half = 0.5 * p.voxel_size / p.dv * math.sqrt(3.0)
    u_R = 0.01
    assert (2 * h * h / p.sdf_sigma ** 2 - 1.0) * math.cos(th) > 1.0 and abs(f(u_R)) >= p.sdf_eps
    assert u_R + half * math.cos(th) < p.voxel_size / p.dv / 2 and u_R - half * math.cos(th) > -p.voxel_size / p.dv / 2
    branch, t_ref = _march_closed_form(f, u_R + half * math.cos(th), math.cos(th), 2 * half, p.sdf_eps)
    assert branch == "secant"
    u_ref = u_R + half * math.cos(th) - t_ref * math.cos(th)
    assert abs(u_ref) < 5e-3
    for R in ([1.03125, 1.0625, c + u_R], [0.96875, 1.125, c + u_R]):
        R = np.array(R)
        cn, nn = s.reproject(R - 3.0 * d, R, 0)
        assert cn is not None
        np.testing.assert_allclose(cn, R + ((u_R - u_ref) / math.cos(th)) * d, atol=1e-9)
        np.testing.assert_allclose(nn, [0, 0, 1], atol=1e-12)


def test_reprojection_of_a_target_on_the_surface():
    """Re-projection reading: a target R where Eq. 1 is already near zero (|f(R)| <
    eps) is met by one Newton step along the ray from R itself, t = -f(R) / (n . d),
    as at the end of a march.  On the sheet pair's middle plane f(R) = 0 and the hit is
    R; 2e-4 m above it f(R) = -7.0e-4 m and the hit is R - f(R) / (n . d) d with
    n = +z, both in closed form."""
    p, c, h, s, f = _sheet_pair_surface()
    th = math.radians(60.0)
    d = np.array([math.sin(th), 0.0, -math.cos(th)])
    for u_R in (0.0, 2e-4):
        assert abs(f(u_R)) < p.sdf_eps
        R = np.array([1.03125, 1.0625, c + u_R])
        cn, nn = s.reproject(R - 3.0 * d, R, 0)
        assert cn is not None
        np.testing.assert_allclose(cn, R - (f(u_R) / np.dot([0.0, 0.0, 1.0], d)) * d, atol=1e-9)
        np.testing.assert_allclose(nn, [0, 0, 1], atol=1e-12)
    assert abs(f(2e-4) + 7.0e-4) < 1e-5


# ------------------------------------------------- final visibility (Section 2.3)
def test_final_visibility_removes_a_path_past_the_panel_border(room_tiny):
    """Section 2.3 ends with a visibility check of every refined segment.  On the box
    room with the panel, the ceiling-then-far-wall image path crosses the panel's
    plane 0.0545 m outside its border: the image method lets it through, but an exact
    plane's Eq. 1 surface is the whole plane (f = distance to it), and the crossing
    lies within half a subvoxel diameter of the border entities' marched segments, so
    the segment is blocked.  The coarse path refines to its image points, is marked
    occluded, and no exact path has its label sequence -- the final check alone
    decides it."""
    x0, (y0, y1), (z0, z1) = cases.PANEL_X, cases.PANEL_Y, cases.PANEL_Z
    sc = cases.room_with_panel(room_tiny)
    p = config.params_for(sc, grad_stop=1e-9)
    s, _, e = oracle.run(sc, p)
    planes = box_room_planes(10.0, 10.0, 3.0)
    ref = image_paths(planes, sc.tx[0], sc.rx[0], max_order=2)
    seq = (5, 1)
    pts, L = ref[seq]
    deepest, margin = cases.panel_margin(sc.tx[0], sc.rx[0], seq, pts)
    assert deepest < 0 and margin == pytest.approx(0.0545, abs=5e-4)          # clear of the panel
    assert margin < 0.5 * p.voxel_size / p.dv * math.sqrt(3.0)                 # within a border entity's reach
    A = e.paths(all_refined=True)
    rows = [i for i in range(len(A["n"])) if tuple(int(l) for l in A["label"][i][:A["n"][i]]) == seq]
    assert rows
    for i in rows:
        assert oracle.STATUS[int(A["status"][i])] == "occluded"
        np.testing.assert_allclose(A["pts"][i][:2], pts, atol=1e-6)
    nodes = [sc.tx[0]] + list(pts) + [sc.rx[0]]
    ends = [(0, oracle.NONE_LABEL), (1, 5), (1, 1), (0, oracle.NONE_LABEL)]
    blocked = [k for k in range(3) if not s.visible(nodes[k], nodes[k + 1], *ends[k], *ends[k + 1], brute=True)]
    assert blocked == [0]                       # brute force over every entity: TX to the ceiling
    assert seq not in {tuple(int(l) for l in e.paths()["label"][i][:n]) for i, n in enumerate(e.paths()["n"])}


# ------------------------------------------------- RX reception sphere (reading C10b)
def test_rx_sphere_is_centred_on_the_rx(room_tiny):
    """One launch cone (n_launch = 1: the Fibonacci lattice's single direction is +x)
    of half-angle 4 degrees from (2, 5, 1.5).  An RX at (7, 5.52, 1.5) lies 5.94
    degrees off the axis; a sphere of the subvoxel radius h_s sqrt(3)/2 around it
    reaches the cone (limit 4 + asin(r/|v|) = 6.47 degrees), one around its subvoxel's
    centre (7.125, 5.625, 1.625) does not (7.09 against 6.40 degrees).  The oracle
    finds the LOS path with the miss distance of the RX itself, 0.52 m, and its
    exact length |TX - RX|."""
    p = config.Params(max_refl=0, max_diff=0, n_launch=1)
    tx, rx = np.array([2.0, 5.0, 1.5]), np.array([7.0, 5.52, 1.5])
    sc = room_tiny.with_pairs(tx[None], rx[None])
    np.testing.assert_allclose(oracle.fibonacci(1)[0], [1, 0, 0], atol=1e-15)
    r = p.voxel_size / p.dv * math.sqrt(3.0) / 2.0
    alpha = math.radians(max(p.cone_half_angle_deg, p.launch_spacing_deg / math.sqrt(2.0)))

    def reaches(cen):
        v = np.asarray(cen) - tx
        ang = math.acos(v[0] / np.linalg.norm(v))
        return ang <= alpha + math.asin(r / np.linalg.norm(v))

    s = oracle.Scene.from_scene(sc, p)
    centre = s.origin + (np.floor((rx - s.origin) / (p.voxel_size / p.dv)) + 0.5) * (p.voxel_size / p.dv)
    np.testing.assert_allclose(centre, [7.125, 5.625, 1.625])
    assert reaches(rx) and not reaches(centre)
    c = s.trace(sc.tx, sc.rx)
    C = c.paths()
    assert list(C["n"]) == [0]
    assert C["miss"][0] == pytest.approx(0.52, abs=1e-9)
    P = s.refine(c).paths()
    assert len(P["n"]) == 1 and P["length"][0] == pytest.approx(np.linalg.norm(rx - tx), rel=1e-12)
