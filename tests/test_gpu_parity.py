"""CUDA library vs FP64 oracle, through the C ABI (needs a B300)."""
import numpy as np
import pytest

import oracle
from paper_2402_13747_b300 import config, scenes
from tests import cases
from tests.imagemethod import box_room_planes, corner_on_floor_mixed_path, image_paths
from tests.pathsets import compare, confirm_alternates, keyed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2402_13747_b300 import _abi
    c = _abi.Context(0)
    yield c
    c.close()


def _tables_match(ctx, sc, params):
    h = ctx.voxelize_scene(sc, params)
    G = ctx.scene_tables(h)
    s = oracle.Scene.from_scene(sc, params)
    R = s.ies()
    Rc = s.cells()
    np.testing.assert_allclose(G["origin"], s.origin, rtol=0, atol=0)
    np.testing.assert_array_equal(G["dims"], s.dims)
    assert G["n_ie"] == s.n_ie
    # integer / index work: bit-exact
    np.testing.assert_array_equal(G["kind"], R["kind"])
    np.testing.assert_array_equal(G["label"], R["label"])
    np.testing.assert_array_equal(G["cell"], R["cell"])
    np.testing.assert_array_equal(G["gs"], R["gs"])
    np.testing.assert_array_equal(G["prange"][:, 1], R["prange"][:, 1])
    np.testing.assert_array_equal(G["cell_count"], Rc["count"])
    occ = Rc["count"] > 0
    np.testing.assert_array_equal(G["cell_begin"][occ], Rc["begin"][occ])
    np.testing.assert_array_equal(G["march"], Rc["march"])
    # FP32 records of FP64 sums: within one FP32 rounding
    np.testing.assert_allclose(G["rp"], R["rp"], atol=2e-6)
    pt = R["kind"] == 0
    np.testing.assert_allclose(G["normal"][pt], R["normal"][pt], atol=2e-6)
    np.testing.assert_allclose(G["bbc"][pt], R["bbc"][pt], atol=2e-6)
    np.testing.assert_array_equal(G["material"][pt], R["material"][pt])
    ctx.release(h)


@pytest.mark.parametrize("name", ["room_tiny", "room_noisy", "wedge"])
def test_voxel_tables_match_oracle(ctx, name):
    sc = {"room_tiny": scenes.room_tiny, "room_noisy": lambda: scenes.room_noisy(n_tx=1, n_rx=1),
          "wedge": scenes.wedge}[name]()
    _tables_match(ctx, sc, config.params_for(sc))


def test_voxel_tables_ragged_sizes(ctx):
    """Clouds that leave a ragged last tile in every kernel, down to a single point."""
    rng = np.random.default_rng(3)
    p = config.Params()
    for n in (1, 2, 31, 33, 4095, 4097, 70001):
        xyz = rng.uniform(0, 6, size=(n, 3)).astype(np.float32)
        nrm = rng.normal(size=(n, 3)).astype(np.float32)
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        lab = rng.integers(0, 7, n).astype(np.uint32)
        sc = scenes.Scene("rand", xyz, nrm, lab, (lab % 3).astype(np.uint8))
        _tables_match(ctx, sc, p)


@pytest.mark.parametrize("launch_mode", [0, 1])
def test_room_tiny_exact_paths(ctx, room_tiny, launch_mode):
    """The tiny room: the same 25 paths as the oracle and the image method, with the
    uniform launch (0) and with the paper's ray toward every IE and RX (1)."""
    p = config.params_for(room_tiny, launch_mode=launch_mode)
    G = ctx.run(room_tiny, p)
    _, _, e = oracle.run(room_tiny, p)
    R = e.paths()
    cmp = compare(G, R, atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [], cmp
    assert cmp["bad"] == [], cmp
    ref = image_paths(box_room_planes(10.0, 10.0, 3.0), room_tiny.tx[0], room_tiny.rx[0], max_order=2)
    got = keyed(G)
    assert {k[3] for k in got} == set(ref)
    for k, (pts, L) in got.items():
        np.testing.assert_allclose(pts, ref[k[3]][0], atol=1e-3)
        assert abs(L - ref[k[3]][1]) <= 1e-6 * ref[k[3]][1]


def test_room_tiny_faces_turned_away(ctx, room_tiny):
    """The tiny room with three faces' normals turned away from the room (a scan's
    normals have no agreed side): the oracle's paths and the 25 image-method paths."""
    sc = room_tiny
    nrm = np.where(np.isin(sc.label, (0, 3, 4))[:, None], -sc.nrm, sc.nrm).astype(np.float32)
    turned = scenes.Scene("room_tiny_turned", sc.xyz, nrm, sc.label, sc.material, tx=sc.tx, rx=sc.rx,
                          max_refl=2, max_diff=0)
    p = config.params_for(turned)
    G = ctx.run(turned, p)
    _, _, e = oracle.run(turned, p)
    cmp = compare(G, e.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [] and cmp["bad"] == [], cmp
    ref = image_paths(box_room_planes(10.0, 10.0, 3.0), sc.tx[0], sc.rx[0], max_order=2)
    got = keyed(G)
    assert {k[3] for k in got} == set(ref)
    for k, (pts, L) in got.items():
        np.testing.assert_allclose(pts, ref[k[3]][0], atol=1e-3)
        assert abs(L - ref[k[3]][1]) <= 1e-6 * ref[k[3]][1]


def test_wedge_keller_point(ctx):
    sc = scenes.wedge(z_tx=0.5, z_rx=2.0)
    p = config.params_for(sc)
    G = ctx.run(sc, p)
    assert len(G["n"]) == 1 and G["n"][0] == 1 and G["type"][0][0] == 1
    np.testing.assert_allclose(G["pts"][0][0], [0.0, 0.0, 1.25], atol=1e-3)


@pytest.mark.parametrize("z_tx,z_rx", [(0.8, 2.0), (1.0, 2.2), (2.0, 0.8)])
def test_reflection_and_diffraction(ctx, z_tx, z_rx):
    """The corner on a floor: the oracle's paths exactly, and the path mixing a floor
    reflection and the edge diffraction (floor first when the TX is the lower end,
    edge first otherwise) at the closed-form points of the floor image and its
    Keller point."""
    sc = scenes.wedge_on_floor(z_tx=z_tx, z_rx=z_rx)
    p = config.params_for(sc)
    G = ctx.run(sc, p)
    _, _, e = oracle.run(sc, p)
    cmp = compare(G, e.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [] and cmp["bad"] == [], cmp
    labels, types, want, L = corner_on_floor_mixed_path(sc.tx[0], sc.rx[0])
    rd = [i for i in range(len(G["n"])) if G["n"][i] == 2 and tuple(G["label"][i][:2]) == labels]
    assert len(rd) == 1
    i = rd[0]
    assert tuple(G["type"][i][:2]) == types
    np.testing.assert_allclose(G["pts"][i][:2], want, atol=1e-3)
    assert abs(G["length"][i] - L) <= 1e-6 * L


@pytest.mark.parametrize("case", ["panel", "merged_labels", "rho3", "refl1_diff1", "edge_end_inside",
                                  "edge_end_beyond"])
def test_pinned_cases_match_oracle(ctx, room_tiny, case):
    """The scenes of the oracle's refinement and visibility pins, on the CUDA path: the
    oracle's path set exactly (points 1e-3 m, lengths 1e-6 relative), and each case's
    own expectation -- no path through the occluding panel (LOS among them), the
    shortest path per merged label sequence, only LOS after three iterations, only
    first-order paths under a one-reflection limit, a Keller point on the edge and none
    beyond its end."""
    if case == "panel":
        sc, kw = cases.room_with_panel(room_tiny), {}
    elif case == "merged_labels":
        sc, kw = cases.room_with_merged_labels(room_tiny), {}
    elif case == "rho3":
        sc, kw = room_tiny, {"rho": 3}
    elif case == "refl1_diff1":
        sc, kw = room_tiny, {"max_refl": 1, "max_diff": 1}
    else:
        sc, kw = cases.tall_wedge(2.6, 3.36 if case == "edge_end_inside" else 3.44), {}
    p = config.params_for(sc, **kw)
    G = ctx.run(sc, p)
    _, _, e = oracle.run(sc, p)
    cmp = compare(G, e.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["bad"] == [], cmp
    labels = {tuple(int(l) for l in G["label"][i][:G["n"][i]]) for i in range(len(G["n"]))}
    if case == "panel":
        # FP32 against FP64 may decide the paths within the implicit surface's reach of
        # the panel's border either way; every other path is the same on both sides,
        # and none that crosses the panel is found
        g, r = keyed(G), keyed(e.paths())
        for k in cmp["only_gpu"] + cmp["only_ref"]:
            pts = (g[k] if k in g else r[k])[0]
            assert cases.panel_margin(sc.tx[0], sc.rx[0], k[3], pts)[1] < 0.3, (k, cmp)
        for k, (pts, L) in g.items():   # through the panel, past its last rows' reach
            assert cases.panel_margin(sc.tx[0], sc.rx[0], k[3], pts)[0] < 0.05, k
        assert () not in labels and cmp["n_common"] >= 8
        return
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [], cmp
    if case == "merged_labels":
        assert len(labels) == 20
    elif case == "rho3":
        assert labels == {()}
    elif case == "refl1_diff1":
        assert len(labels) == 7 and all(len(k) <= 1 for k in labels)
    elif case == "edge_end_inside":
        assert len(G["n"]) == 1
        np.testing.assert_allclose(G["pts"][0][0], [0.0, 0.0, 2.98], atol=1e-3)
    else:
        assert len(G["n"]) == 0


def test_final_visibility_removes_the_path_past_the_panel_border(ctx, room_tiny):
    """Section 2.3's last step on the CUDA path: the panel scene's ceiling-then-far-wall
    path crosses the panel's plane 0.0545 m outside its border.  Its coarse paths
    refine to the image points and the final visibility check marks every one
    occluded, as in the oracle, so no exact path has its label sequence.  A refinement
    that skipped the check would report it."""
    sc = cases.room_with_panel(room_tiny)
    p = config.params_for(sc)
    s = ctx.voxelize_scene(sc, p)
    c = ctx.trace(s, sc.tx, sc.rx, p)
    P = ctx.refine(s, c, p)
    A, F = ctx.query(P, 1), ctx.query(P, 0)
    for h in (P, c, s):
        ctx.release(h)
    seq = (5, 1)
    pts, _ = image_paths(box_room_planes(10.0, 10.0, 3.0), sc.tx[0], sc.rx[0], max_order=2)[seq]
    rows = [i for i in range(len(A["n"])) if tuple(int(l) for l in A["label"][i][:A["n"][i]]) == seq]
    assert rows
    for i in rows:
        assert int(A["status"][i]) == 3, (i, A["status"][i])     # occluded
        np.testing.assert_allclose(A["pts"][i][:2], pts, atol=1e-3)
    assert seq not in {tuple(int(l) for l in F["label"][i][:n]) for i, n in enumerate(F["n"])}


def test_rx_sphere_is_centred_on_the_rx(ctx, room_tiny):
    """One launch cone along +x (n_launch = 1) of half-angle 4 degrees from (2, 5, 1.5)
    reaches the reception sphere around the RX at (7, 5.52, 1.5) but not one around
    its subvoxel's centre: the LOS coarse path exists with the RX's own miss distance
    0.52 m, and refines to the length |TX - RX|, as in the oracle."""
    p = config.Params(max_refl=0, max_diff=0, n_launch=1)
    tx, rx = np.array([[2.0, 5.0, 1.5]]), np.array([[7.0, 5.52, 1.5]])
    sc = room_tiny.with_pairs(tx, rx)
    s = ctx.voxelize_scene(sc, p)
    c = ctx.trace(s, sc.tx, sc.rx, p)
    C = ctx.query_coarse(c)
    P = ctx.refine(s, c, p)
    F = ctx.query(P, 0)
    for h in (P, c, s):
        ctx.release(h)
    assert list(C["n"]) == [0] and C["miss"][0] == pytest.approx(0.52, abs=1e-5)
    assert len(F["n"]) == 1 and F["length"][0] == pytest.approx(np.linalg.norm(rx - tx), rel=1e-9)


def test_memory_returns_after_release(ctx, room_tiny):
    """The context's device-memory accounting: a scene, a coarse set and a path set
    each hold memory while alive, the scratch of a call is freed by the call itself,
    and releasing the three returns the context to where it started."""
    p = config.params_for(room_tiny)
    ctx.run(room_tiny, p)                      # whatever a first call leaves in place exists from here on
    before = ctx.memory_used()
    s = ctx.voxelize_scene(room_tiny, p)
    held_s = ctx.memory_used()
    c = ctx.trace(s, room_tiny.tx, room_tiny.rx, p)
    held_c = ctx.memory_used()
    P = ctx.refine(s, c, p)
    held_p = ctx.memory_used()
    assert before < held_s < held_c < held_p
    for h in (P, c, s):
        ctx.release(h)
    assert ctx.memory_used() == before
    assert set(ctx.get_tuning()) >= {"level_block", "refine_blocks", "refine_order", "graph"}


def test_noisy_room_subset_matches_oracle(ctx):
    """Noisy room with the box: 1 TX x 3 RX, <= 2 reflections + 1 diffraction.  The same
    (TX, RX, types, labels) set; every path within 1e-3 m and 1e-6 relative length but
    for oracle-confirmed alternate stationary points (at most 1 %)."""
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:3])
    p = config.params_for(sc, max_refl=2, max_diff=1)
    G = ctx.run(sc, p)
    _, _, e = oracle.run(sc, p)
    cmp = compare(G, e.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["n_ref"] > 20
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [], cmp
    confirm_alternates(G, cmp["bad"], sc, p, max(1, cmp["n_common"] // 100))


def test_noisy_room_subset_paper_launch(ctx):
    """The paper's transmission phase (a ray toward every IE and RX) on the noisy room:
    the coarse sets match in size and the exact path sets as for the uniform launch."""
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:3])
    p = config.params_for(sc, max_refl=2, max_diff=1, launch_mode=1)
    G = ctx.run(sc, p)
    _, c, e = oracle.run(sc, p)
    cmp = compare(G, e.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["n_ref"] > 20
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [], cmp
    confirm_alternates(G, cmp["bad"], sc, p, max(1, cmp["n_common"] // 100))
    # initial interactions: every IE visible from the TX, on both sides
    assert abs(G["counts"]["n_coarse_raw"] - c.stats["n_before_kappa"]) <= 0.02 * c.stats["n_before_kappa"]


def test_deterministic(ctx, room_tiny):
    p = config.params_for(room_tiny)
    a = ctx.run(room_tiny, p)
    b = ctx.run(room_tiny, p)
    ka, kb = keyed(a), keyed(b)
    assert ka.keys() == kb.keys()
    for k in ka:
        assert np.array_equal(ka[k][0], kb[k][0]) and ka[k][1] == kb[k][1]


def test_edge_cases(ctx, room_tiny):
    from paper_2402_13747_b300._abi import NimbusError
    p = config.params_for(room_tiny)
    s = ctx.voxelize_scene(room_tiny, p)
    # no RX: no paths
    c = ctx.trace(s, room_tiny.tx, np.zeros((0, 3)), p)
    P = ctx.refine(s, c, p)
    assert ctx.counts(P)["n_paths"] == 0
    # no interactions allowed: LOS only
    p0 = p.replace(max_refl=0, max_diff=0)
    c = ctx.trace(s, room_tiny.tx, room_tiny.rx, p0)
    out = ctx.query(ctx.refine(s, c, p0))
    assert list(out["n"]) == [0]
    assert out["length"][0] == pytest.approx(np.sqrt(34.0), rel=1e-12)
    # TX outside the grid
    with pytest.raises(NimbusError):
        ctx.trace(s, np.array([[50.0, 0, 0]]), room_tiny.rx, p)
    # overflow is reported with the needed size
    with pytest.raises(NimbusError) as ei:
        ctx.trace(s, room_tiny.tx, room_tiny.rx, p, max_nodes=100)
    assert "overflow" in str(ei.value)
    # bad handle kind
    with pytest.raises(NimbusError):
        ctx.refine(s, s, p)
    ctx.release(s)


def test_degenerate_pairs_and_parameters(ctx, room_tiny):
    """RX on the TX, a duplicated RX and kappa = 1 give the oracle's paths; an unknown
    launch mode and too many interactions are argument errors."""
    from paper_2402_13747_b300._abi import NimbusError
    tx = room_tiny.tx[0]
    sc = room_tiny.with_pairs(room_tiny.tx, np.vstack([tx, room_tiny.rx[0], room_tiny.rx[0]]))
    p = config.params_for(sc, max_refl=1)
    G = ctx.run(sc, p)
    _, _, e = oracle.run(sc, p)
    cmp = compare(G, e.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [] and cmp["bad"] == [], cmp
    on = np.sort(G["length"][G["rx"] == 0])
    want = np.sort([0.0] + [2 * d for d in (tx[0], 10 - tx[0], tx[1], 10 - tx[1], tx[2], 3 - tx[2])])
    np.testing.assert_allclose(on, want, atol=1e-5)
    np.testing.assert_array_equal(np.sort(G["length"][G["rx"] == 1]), np.sort(G["length"][G["rx"] == 2]))
    p1 = config.params_for(room_tiny, kappa=1)
    G1 = ctx.run(room_tiny, p1)
    _, _, e1 = oracle.run(room_tiny, p1)
    cmp = compare(G1, e1.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["only_gpu"] == [] and cmp["only_ref"] == [] and len(G1["n"]) == 25, cmp
    s = ctx.voxelize_scene(room_tiny, p1)
    for bad in (p1.replace(launch_mode=2), p1.replace(max_int=9, max_refl=9)):
        with pytest.raises(NimbusError, match="ERR_ARG"):
            ctx.trace(s, room_tiny.tx, room_tiny.rx, bad)
    ctx.release(s)


def test_empty_cloud_with_region(ctx):
    p = config.Params(max_refl=1)
    s = ctx.voxelize(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros(0, np.uint32),
                     params=p, region=np.array([[0, 0, 0], [4, 4, 4.0]]))
    c = ctx.trace(s, np.array([[1.0, 1, 1]]), np.array([[3.0, 3, 3]]), p)
    out = ctx.query(ctx.refine(s, c, p))
    assert list(out["n"]) == [0]


@pytest.mark.parametrize("case", ["moving_box", "remove_fixed_box", "remove_only", "replacement_outside"])
def test_update_region_equals_rebuild(ctx, case):
    """Dynamic scene: a region update re-bins only the voxels that lose or gain points
    and splices them into the tables; the result equals a full build of the new cloud
    on the same grid entry for entry (every table, the point ranges and the march
    field), and the paths traced on both are identical.  Cases: the moving box; the
    fixed box removed (its voxels hold edge entities, which stay); a region emptied
    with no replacement; replacement points outside the region box."""
    room = scenes.room_noisy(n_tx=1, n_rx=2)
    p = config.params_for(room, max_refl=2, max_diff=1)
    s = ctx.voxelize_scene(room, p)
    info = ctx.scene_info(s)
    # a region box that reproduces this grid: one voxel inside the padded origin
    h = p.voxel_size
    region = np.array([info["origin"] + h + 1e-6, info["origin"] + (info["dims"] - 1) * h - 1e-6])
    xyz, nrm, lab, mat, lo, hi = scenes.moving_box(room, step=7)
    lo, hi = lo - 0.01, hi + 0.01
    if case == "remove_fixed_box":
        lo, hi = np.array([4.45, 6.45, 0.02]), np.array([5.55, 7.55, 2.1])
        xyz = nrm = lab = mat = None
    elif case == "remove_only":
        xyz = nrm = lab = mat = None
    elif case == "replacement_outside":
        lo, hi = np.array([1.0, 1.0, -0.02]), np.array([1.6, 1.6, 0.6])   # a floor patch; the box lies elsewhere
    ctx.update_region(s, lo, hi, xyz, nrm, lab, mat)
    A = ctx.scene_tables(s)
    # the same cloud built from scratch on the same grid
    keep = ~np.all((room.xyz >= lo.astype(np.float32)) & (room.xyz <= hi.astype(np.float32)), axis=1)
    parts = [(room.xyz[keep], room.nrm[keep], room.label[keep], room.material[keep])]
    if xyz is not None:
        parts.append((xyz, nrm, lab, mat))
    sc2 = scenes.Scene("upd", *[np.concatenate([q[k] for q in parts]) for k in range(4)], room.edges, room.edge_label,
                       tx=room.tx, rx=room.rx, region=region)
    assert (~keep).sum() > 0
    s2 = ctx.voxelize_scene(sc2, p)
    B = ctx.scene_tables(s2)
    np.testing.assert_array_equal(A["dims"], B["dims"])
    assert A["n_ie"] == B["n_ie"] and A["n_points"] == B["n_points"]
    for k in ("kind", "label", "cell", "gs", "prange", "cell_count", "cell_begin", "march", "material", "rp", "normal",
              "bbc"):
        np.testing.assert_array_equal(A[k], B[k], err_msg=k)
    got = [ctx.query(ctx.refine(h_, ctx.trace(h_, room.tx, room.rx, p), p), 0) for h_ in (s, s2)]
    assert len(got[0]["n"]) > 0
    for k in ("tx", "rx", "n", "type", "label", "pts", "length"):
        np.testing.assert_array_equal(got[0][k], got[1][k])
    ctx.release(s)
    ctx.release(s2)


def test_autotune_keeps_results(ctx):
    """The autotuner only changes launch layouts: after it, and under every layout it
    can pick, the noisy-room subset gives bit-identical exact paths."""
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:3])
    p = config.params_for(sc, max_refl=2, max_diff=1)
    base = ctx.run(sc, p)
    s = ctx.voxelize_scene(sc, p)
    t = ctx.autotune(s, sc.tx, sc.rx[:2], p)
    ctx.release(s)
    assert t["level_block"] in (128, 256, 512)
    assert t["refine_blocks"] in (0, 4) and t["refine_order"] in (0, 1, 2) and t["refine_ms"] > 0
    assert t["level_queue"] in (0, 1)
    assert t["refine_split"] in (0, 64, 128, 512) and t["refine_split_key"] in (0, 1)
    assert t["level_help"] in (0, 1) and not (t["level_help"] and t["level_queue"])
    assert t["level_rx_first"] in (0, 1)
    for layout in (dict(level_block=128, refine_blocks=3, refine_order=0, level_queue=1, refine_split=0),
                   dict(level_block=256, refine_blocks=0, refine_order=2, level_queue=0, refine_split=0),
                   dict(level_block=512, refine_blocks=0, refine_order=1, level_queue=1, refine_split=0),
                   dict(level_block=512, refine_blocks=0, refine_order=1, level_queue=0, refine_split=0,
                        level_help=1, level_rx_first=1),
                   dict(level_block=256, refine_blocks=0, refine_order=1, level_queue=0, refine_split=5),
                   dict(level_block=256, refine_blocks=2, refine_order=2, level_queue=0, refine_split=64),
                   dict(level_block=256, refine_blocks=0, refine_order=0, level_queue=0, refine_split=7,
                        refine_split_key=1), t):
        ctx.set_tuning(**{k: layout.get(k, 0) for k in ("level_block", "refine_blocks", "refine_order", "level_queue",
                                                        "refine_split", "refine_split_key", "level_help",
                                                        "level_rx_first")})
        G = ctx.run(sc, p)
        assert len(G["n"]) == len(base["n"])
        for k in ("tx", "rx", "n", "type", "label", "pts", "length"):
            np.testing.assert_array_equal(G[k], base[k])
    ctx.set_tuning(level_block=512, refine_blocks=0, refine_order=1, level_queue=0, refine_split=0, refine_split_key=0,
                   level_help=1, level_rx_first=1)
    with pytest.raises(Exception):
        ctx.set_tuning(level_block=96)
    with pytest.raises(Exception):
        ctx.set_tuning(level_help=2)
    with pytest.raises(Exception):
        ctx.set_tuning(level_rx_first=2)
    with pytest.raises(Exception):
        ctx.set_tuning(refine_split=-1)
    with pytest.raises(Exception):
        ctx.set_tuning(refine_split_key=2)


def _coarse_rows(cq):
    miss = np.asarray(cq["miss"], np.float32).view(np.uint32)
    return sorted(zip(cq["tx"].tolist(), cq["rx"].tolist(), cq["n"].tolist(), map(tuple, cq["ie"].tolist()),
                      map(tuple, cq["type"].tolist()), map(tuple, cq["label"].tolist()), miss.tolist()))


def test_graph_launch_keeps_results(ctx):
    """Issuing each host-free stretch as one CUDA graph changes nothing but how the
    launches reach the GPU: the same coarse set and exact paths bit for bit, the same
    kernel count, and the stage times still come from events recorded inside the
    graphs.  Covers both launch modes and a request-batched trace (per-RX owner and
    depth)."""
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:2], full.rx[:3])
    s = None
    try:
        for mode in (0, 1):
            p = config.params_for(sc, max_refl=2, max_diff=1, launch_mode=mode)
            if s is None:
                s = ctx.voxelize_scene(sc, p)
            owner = np.array([0, 1, -1], np.int32)
            depth = np.array([1, 3, 2], np.int32)
            res = {}
            for graph in (0, 1):
                ctx.set_tuning(graph=graph)
                for batched in (False, True):
                    kw = dict(rx_owner=owner, rx_max_int=depth) if batched else {}
                    co = ctx.trace(s, sc.tx, sc.rx, p, **kw)
                    cq = ctx.query_coarse(co)
                    cc = ctx.coarse_counts(co)
                    P = ctx.refine(s, co, p)
                    out = ctx.query(P, 0)
                    pc = ctx.counts(P)
                    ctx.release(P)
                    ctx.release(co)
                    res[graph, batched] = (cq, out, cc, pc)
            for batched in (False, True):
                (cq0, o0, cc0, pc0), (cq1, o1, cc1, pc1) = res[0, batched], res[1, batched]
                assert len(o0["n"]) > 0
                # the coarse records come out in group order, whose ids follow the
                # device's atomics: compare them as a set of rows
                assert _coarse_rows(cq1) == _coarse_rows(cq0)
                for k in ("tx", "rx", "n", "type", "label", "pts", "length"):
                    np.testing.assert_array_equal(o1[k], o0[k], err_msg=k)
                for k in ("n_cones", "n_vis", "n_nodes", "n_coarse", "n_coarse_raw", "launches"):
                    assert cc1[k] == cc0[k], k
                assert pc1["launches"] == pc0["launches"]
                assert cc1["ms_levels"] > 0 and cc1["ms_vis"] > 0
                assert cc1["ms_primary"] > 0 or mode == 1
                assert pc1["ms_refine"] > 0 and pc1["ms_dedup"] > 0
    finally:
        ctx.set_tuning(graph=1)
        if s is not None:
            ctx.release(s)
    with pytest.raises(Exception):
        ctx.set_tuning(graph=2)


@pytest.mark.parametrize("case", ["room_2x3_d3", "wedge_d2", "batched", "rx_only_depth1"])
def test_single_launch_propagation_keeps_results(ctx, case):
    """All depths in one launch (a cone task queue across levels, level_queue=1)
    against one launch per depth: the same coarse rows, exact paths and counters, at
    128-, 256- and 512-thread blocks, with request batching (per-RX owner and depth),
    and at depth 1 where the queue holds only the first level.  With level_help the
    per-depth launches' warps walk one another's visibility rays once their own cones
    are done; the counters (rays walked, bytes) must still be those of each cone
    walking its own rays in order."""
    full = scenes.room_noisy()
    kw = {}
    if case == "wedge_d2":
        sc = scenes.wedge_on_floor(z_tx=0.8, z_rx=2.0)
        p = config.params_for(sc, max_refl=1, max_diff=1)
    else:
        sc = full.with_pairs(full.tx[:2], full.rx[:3])
        p = config.params_for(sc, max_refl=2 if case != "rx_only_depth1" else 1,
                              max_diff=1 if case != "rx_only_depth1" else 0)
        if case == "batched":
            kw = dict(rx_owner=np.array([0, 1, -1], np.int32), rx_max_int=np.array([1, 3, 2], np.int32))
    s = ctx.voxelize_scene(sc, p)
    res = {}
    try:
        for lq, help_ in ((0, 0), (0, 1), (1, 0)):
            for block in (128, 256, 512):
                ctx.set_tuning(level_queue=lq, level_block=block, level_help=help_)
                co = ctx.trace(s, sc.tx, sc.rx, p, **kw)
                cq, cc = ctx.query_coarse(co), ctx.coarse_counts(co)
                P = ctx.refine(s, co, p)
                res[lq, help_, block] = (cq, ctx.query(P, 0), cc)
                ctx.release(P)
                ctx.release(co)
    finally:
        ctx.set_tuning(level_queue=0, level_block=512, level_help=1)
        ctx.release(s)
    cq0, o0, cc0 = res[0, 0, 256]
    assert cc0["n_coarse"] > 0
    for key, (cq, o, cc) in res.items():
        assert _coarse_rows(cq) == _coarse_rows(cq0), key
        for k in ("tx", "rx", "n", "type", "label", "pts", "length"):
            np.testing.assert_array_equal(o[k], o0[k], err_msg=f"{key} {k}")
        for k in ("n_cones", "n_vis", "n_nodes", "n_coarse", "n_coarse_raw", "bytes_levels"):
            assert cc[k] == cc0[k], (key, k)
    with pytest.raises(Exception):
        ctx.set_tuning(level_queue=2)


def test_scene_checkpoint_round_trip(ctx, tmp_path):
    """A saved scene -- including a region update -- loads into another context with
    the same tables and gives the same coarse and exact paths; damaged files fail."""
    from paper_2402_13747_b300 import _abi
    from paper_2402_13747_b300.serve import moved_box_update
    full = scenes.room_noisy()
    sc = full.with_pairs(full.tx[:1], full.rx[:3])
    p = config.params_for(sc, max_refl=2, max_diff=1)
    s = ctx.voxelize_scene(sc, p)
    lo, hi, cloud = moved_box_update(sc, {"box": None}, 3)
    ctx.update_region(s, lo, hi, *cloud)
    path = str(tmp_path / "scene.nimbus")
    ctx.scene_save(s, path)
    other = _abi.Context(0)
    s2 = other.scene_load(path)
    A, B = ctx.scene_tables(s), other.scene_tables(s2)
    for k in ("origin", "dims", "kind", "label", "cell", "gs", "prange", "cell_count", "march", "rp", "normal"):
        np.testing.assert_array_equal(np.asarray(A[k]), np.asarray(B[k]), err_msg=k)
    def paths(c, h):
        co = c.trace(h, sc.tx, sc.rx, p)
        P = c.refine(h, co, p)
        out = c.query(P, 0)
        c.release(P)
        c.release(co)
        return out
    G1, G2 = paths(ctx, s), paths(other, s2)
    for k in ("tx", "rx", "n", "type", "label", "pts", "length"):
        np.testing.assert_array_equal(G1[k], G2[k])
    # a truncated and a foreign file are rejected without creating a scene
    raw = open(path, "rb").read()
    open(tmp_path / "cut.nimbus", "wb").write(raw[: len(raw) // 2])
    open(tmp_path / "foreign.nimbus", "wb").write(b"not a scene" * 10)
    for bad in ("cut.nimbus", "foreign.nimbus", "missing.nimbus"):
        with pytest.raises(_abi.NimbusError, match="ERR_IO"):
            other.scene_load(str(tmp_path / bad))
    ctx.release(s)
    other.close()
