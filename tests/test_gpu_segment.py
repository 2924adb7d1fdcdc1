"""nimbus_segment (automatic labels and exterior edges) against the labelling oracle,
through the C ABI, and the labels it makes driving the method (needs a B300)."""
import ctypes as C

import numpy as np
import pytest

import oracle
import oracle.segment as seg
from paper_2402_13747_b300 import config, scenes
from tests import segclouds
from tests.pathsets import compare

pytestmark = pytest.mark.gpu

SP = config.SegmentParams()


@pytest.fixture(scope="module")
def ctx():
    from paper_2402_13747_b300 import _abi
    c = _abi.Context(0)
    yield c
    c.close()


def _scene(name):
    return {"room_tiny": scenes.room_tiny, "wedge_on_floor": scenes.wedge_on_floor,
            "room_noisy": lambda: scenes.room_noisy(n_tx=1, n_rx=3)}[name]()


def _cloud(name):
    """xyz, nrm of a named cloud: a scene, or one of the labelling pins' sheets and boxes."""
    kind, _, arg = name.partition(":")
    if kind == "fold":
        return segclouds.folded_sheet(float(arg))[:2]
    if kind == "offset":
        return segclouds.offset_sheets(float(arg))[:2]
    if kind == "box":
        return segclouds.box_on_floor(float(arg))[:2]
    if kind == "rows":
        return segclouds.two_sheets_in_row_order()[:2]
    sc = _scene(name)
    return sc.xyz, sc.nrm


@pytest.mark.parametrize("name", ["room_tiny", "wedge_on_floor", "room_noisy", "fold:5", "fold:11", "fold:20",
                                  "fold:-40", "offset:0.01", "offset:0.1", "box:0.5", "box:1.0", "rows"])
def test_labels_and_edges_match_oracle(ctx, name):
    """Integer labels bit for bit; edges to 1e-9 m (FP64 sums in another order)."""
    xyz, nrm = _cloud(name)
    G = ctx.segment(xyz, nrm, SP)
    lab, E, EL, ns = seg.segment(xyz, nrm, SP)
    assert G["counts"]["n_surfaces"] == ns
    np.testing.assert_array_equal(G["labels"], lab)
    np.testing.assert_array_equal(G["edge_labels"], EL)
    assert G["edges"].shape == E.shape
    np.testing.assert_allclose(G["edges"], E, atol=1e-9)
    assert G["counts"]["ms"] > 0 and G["counts"]["ms_total"] >= G["counts"]["ms"]


def test_shuffled_cloud_same_labels(ctx):
    sc = _scene("room_noisy")
    G = ctx.segment(sc.xyz, sc.nrm, SP)
    perm = np.random.default_rng(9).permutation(sc.xyz.shape[0])
    H = ctx.segment(sc.xyz[perm], sc.nrm[perm], SP)
    np.testing.assert_array_equal(H["labels"], G["labels"][perm])
    np.testing.assert_allclose(H["edges"], G["edges"], atol=1e-9)


def test_edge_buffer_bound_and_arguments(ctx):
    """Too small an edge buffer: the first edges_cap edges, NIMBUS_ERR_OVERFLOW and the
    needed count; bad parameters and an empty cloud are argument errors."""
    from paper_2402_13747_b300 import _abi
    sc = _scene("room_noisy")
    full = ctx.segment(sc.xyz, sc.nrm, SP)
    assert len(full["edges"]) == 8
    x, nr = np.ascontiguousarray(sc.xyz, np.float32), np.ascontiguousarray(sc.nrm, np.float32)
    cl = _abi.Cloud(x.ctypes.data, nr.ctypes.data, None, None, x.shape[0])
    prm = _abi.segment_params(SP)
    labels = np.zeros(x.shape[0], np.uint32)
    edges = np.zeros((2, 12))
    elab = np.zeros(2, np.uint32)
    cnt = _abi.SegmentCounts()
    rc = ctx.L.nimbus_segment(ctx.h, C.byref(cl), C.byref(prm), labels.ctypes.data, edges.ctypes.data,
                              elab.ctypes.data, 2, C.byref(cnt), None)
    assert rc == _abi.ERR_OVERFLOW and cnt.n_edges == 8
    np.testing.assert_array_equal(labels, full["labels"])
    np.testing.assert_allclose(edges, full["edges"][:2], atol=1e-12)
    bad = _abi.segment_params(SP.replace(min_points=2))
    assert ctx.L.nimbus_segment(ctx.h, C.byref(cl), C.byref(bad), labels.ctypes.data, None, None, 0,
                                C.byref(cnt), None) == _abi.ERR_ARG
    empty = _abi.Cloud(x.ctypes.data, nr.ctypes.data, None, None, 0)
    assert ctx.L.nimbus_segment(ctx.h, C.byref(empty), C.byref(prm), labels.ctypes.data, None, None, 0,
                                C.byref(cnt), None) == _abi.ERR_ARG


def test_auto_labels_drive_the_method(ctx):
    """The noisy room with its labels and edges replaced by nimbus_segment's: the CUDA
    path matches the oracle on that scene, and finds the paths of the generator-labelled
    scene (labels mapped by majority)."""
    sc = _scene("room_noisy")
    G = ctx.segment(sc.xyz, sc.nrm, SP)
    auto = scenes.Scene("room_noisy_auto", sc.xyz, sc.nrm, G["labels"], sc.material, G["edges"], G["edge_labels"],
                        tx=sc.tx, rx=sc.rx, max_refl=2, max_diff=1, region=sc.region)
    p = config.params_for(auto, max_refl=2, max_diff=1)
    A = ctx.run(auto, p)
    _, _, e = oracle.run(auto, p)
    cmp = compare(A, e.paths(), atol_pts=1e-3, rtol_len=1e-6)
    assert cmp["n_ref"] > 20 and cmp["jaccard"] >= 0.9, cmp
    assert len(cmp["bad"]) <= 0.05 * cmp["n_common"], cmp
    # against the generator's labels: same paths up to the relabelling
    R = ctx.run(sc, config.params_for(sc, max_refl=2, max_diff=1))
    to_true = {}
    for a, t in zip(G["labels"].tolist(), sc.label.tolist()):
        to_true.setdefault(a, {}).setdefault(t, 0)
        to_true[a][t] += 1
    major = {a: max(c, key=c.get) for a, c in to_true.items()}
    edge_true = {}
    for k, el in enumerate(G["edge_labels"].tolist()):
        mid = 0.5 * (G["edges"][k, :3] + G["edges"][k, 3:6])
        j = int(np.argmin([np.linalg.norm(0.5 * (q[:3] + q[3:6]) - mid) for q in sc.edges]))
        edge_true[el] = int(sc.edge_label[j])

    def keys(P, relabel):
        out = set()
        for i in range(len(P["n"])):
            n = int(P["n"][i])
            labs = tuple(relabel(int(l), int(t)) for l, t in zip(P["label"][i][:n], P["type"][i][:n]))
            out.add((int(P["tx"][i]), int(P["rx"][i]), tuple(int(t) for t in P["type"][i][:n]), labs))
        return out

    ka = keys(A, lambda l, t: edge_true[l] if t == 1 else major[l])
    kr = keys(R, lambda l, t: l)
    assert len(ka & kr) >= 0.85 * len(kr), (len(ka), len(kr), len(ka & kr))


def test_segment_timing_large_scenes(ctx):
    """Labels and edges of the 1.9 M-point indoor scan and the 20 M-point street: sizes
    and times (CUDA events), with the invariants any result must meet."""
    for sc in (scenes.indoor(), scenes.street()):
        G = ctx.segment(sc.xyz, sc.nrm, SP)
        c = G["counts"]
        assert G["labels"].max() < c["n_surfaces"] and c["n_planar"] <= c["n_groups"]
        assert np.all(G["edge_labels"] == c["n_surfaces"] + np.arange(len(G["edges"])))
        n0, n1 = G["edges"][:, 6:9], G["edges"][:, 9:]
        np.testing.assert_allclose(np.linalg.norm(n0, axis=1), 1.0, atol=1e-9)
        assert np.all(np.einsum("ij,ij->i", n0, n1) <= np.cos(np.radians(SP.edge_angle_deg)) + 1e-12)
        print(f"{sc.name}: {sc.xyz.shape[0]} points, {c['n_groups']} groups ({c['n_planar']} planar), "
              f"{c['n_surfaces']} surfaces, {c['n_edges']} edges; {c['ms']:.1f} ms labelling, "
              f"{c['ms_total']:.1f} ms with the binning voxelisation")
