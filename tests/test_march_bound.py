"""The visibility rays' march skip.

Before marching a candidate IE (Section 2.2.1), the CUDA visibility walk bounds Eq. 1
over that IE's points from a per-IE record (the smallest cosine between a point
normal and the mean normal, the range of the points' offsets along the mean normal,
their largest distance from the bbox centre) and skips the march when the bound
keeps |f| above eps on the whole segment.  The skip is exact only if the bound is:
here its mathematics is checked in FP64 against the oracle's own march, which
judges every segment, and on the GPU the stored records are checked against the
points they bound.
"""
import numpy as np
import pytest

import oracle
from paper_2402_13747_b300 import config, scenes

MARGIN = 1e-5


def slab_of(xyz, nrm, n0, c):
    """(smallest cosine, smallest offset, largest offset, largest distance) of a point set."""
    p = xyz - c
    cos = (nrm @ n0) / np.linalg.norm(nrm, axis=1)
    off = p @ n0
    return cos.min(), off.min(), off.max(), np.linalg.norm(p, axis=1).max()


def cannot_hit(slab, n0, x0, d, half, eps):
    """The bound: f(x) >= cos(theta) (x.n0 - hi) - sin(theta) (|x| + r) above the slab,
    symmetrically below it, at the extremes of x.n0 and |x| over the segment."""
    cmin, lo, hi, r = slab
    if not cmin > 0.5:
        return False
    s0, sd = x0 @ n0, half * abs(d @ n0)
    D = max(np.linalg.norm(x0 - half * d), np.linalg.norm(x0 + half * d)) + r
    need = eps + MARGIN + np.sqrt(max(0.0, 1.0 - cmin * cmin)) * D
    return (s0 - sd - hi) * cmin > need or (lo - (s0 + sd)) * cmin > need


@pytest.fixture(scope="module")
def noisy_scene():
    sc = scenes.room_noisy(n_tx=1, n_rx=1)
    p = config.params_for(sc)
    s = oracle.Scene.from_scene(sc, p)
    return s, p


@pytest.mark.parametrize("seed", [0, 1])
def test_bound_never_skips_a_hit(noisy_scene, seed):
    """Segments across, beside and grazing 200 IEs of the noisy room (5 mm / 2 degree
    noise): wherever the bound says the march cannot hit, the oracle's march finds no
    hit.  The sample is not vacuous: many segments are skipped, many hit."""
    s, p = noisy_scene
    I = s.ies()
    xyz, nrm = s.points()
    half = 0.5 * s.params.voxel_size / s.params.dv * np.sqrt(3.0)
    rng = np.random.default_rng(seed)
    cand = np.nonzero((I["kind"] == 0) & (I["prange"][:, 1] >= 4))[0]
    skipped = hits = 0
    for ie in rng.choice(cand, size=200, replace=False):
        b, k = I["prange"][ie]
        n0, c = I["normal"][ie], I["bbc"][ie]
        slab = slab_of(xyz[b:b + k], nrm[b:b + k], n0, c)
        t1 = np.cross(n0, [1.0, 0.0, 0.0] if abs(n0[0]) < 0.9 else [0.0, 1.0, 0.0])
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(n0, t1)
        for _ in range(12):
            # a direction from grazing (along the surface) to steep, a closest approach
            # within a few centimetres of the centre along the normal
            elev = rng.choice([rng.uniform(0.0, 0.05), rng.uniform(0.0, 1.5)])
            az = rng.uniform(0, 2 * np.pi)
            d = np.cos(elev) * (np.cos(az) * t1 + np.sin(az) * t2) + np.sin(elev) * n0 * rng.choice([-1, 1])
            d /= np.linalg.norm(d)
            q = c + rng.uniform(-0.05, 0.05) * n0 + rng.uniform(-0.02, 0.02) * t1
            P = q - 3.0 * d
            x0 = (P - c) + ((c - P) @ d) * d
            hit = s.sdf_hit(int(ie), P, d)
            if cannot_hit(slab, n0, x0, d, half, p.sdf_eps):
                skipped += 1
                assert hit is None, (ie, d, q)
            hits += hit is not None
    assert skipped > 150 and hits > 500, (skipped, hits)


def test_bound_on_an_exact_plane():
    """On a noise-free plane (all normals equal) the bound is the plane distance: a
    segment parallel to the plane 2 mm above it (beyond eps = 1 mm plus the margin) is
    skipped, one 0.5 mm above it is not, and the oracle agrees that the first misses."""
    sc = scenes.room_tiny()
    p = config.params_for(sc)
    s = oracle.Scene.from_scene(sc, p)
    I = s.ies()
    xyz, nrm = s.points()
    half = 0.5 * p.voxel_size / p.dv * np.sqrt(3.0)
    floor = np.nonzero((I["kind"] == 0) & (np.abs(I["normal"][:, 2] - 1.0) < 1e-12) & (I["prange"][:, 1] >= 4))[0]
    ie = int(floor[len(floor) // 2])
    b, k = I["prange"][ie]
    n0, c = I["normal"][ie], I["bbc"][ie]
    slab = slab_of(xyz[b:b + k], nrm[b:b + k], n0, c)
    assert slab[0] == pytest.approx(1.0, abs=1e-12) and slab[2] - slab[1] < 1e-9
    d = np.array([1.0, 0.0, 0.0])
    for h, skip in ((2e-3, True), (5e-4, False)):
        q = c + (h + slab[2]) * n0
        x0 = q - c
        assert cannot_hit(slab, n0, x0, d, half, p.sdf_eps) == skip
        if skip:
            assert s.sdf_hit(ie, q - 3.0 * d, d) is None


@pytest.mark.gpu
def test_stored_bounds_cover_the_points():
    """The CUDA voxelisation's per-IE bound records (nimbus_scene_tables 'slab') bound
    the IE's points: the cosine and the lower offset no larger, the upper offset and
    the radius no smaller than the FP64 values from the same points (to FP32
    rounding), on the noisy room and on an exact plane."""
    from paper_2402_13747_b300 import _abi
    ctx = _abi.Context(0)
    for sc in (scenes.room_noisy(n_tx=1, n_rx=1), scenes.room_tiny()):
        p = config.params_for(sc)
        s = ctx.voxelize_scene(sc, p)
        G = ctx.scene_tables(s)
        osc = oracle.Scene.from_scene(sc, p)
        R = osc.ies()
        xyz, nrm = osc.points()
        np.testing.assert_array_equal(G["prange"][:, 1], R["prange"][:, 1])
        for ie in np.nonzero(G["kind"] == 0)[0]:
            b, k = R["prange"][ie]
            n0, c = G["normal"][ie].astype(np.float64), G["bbc"][ie].astype(np.float64)
            cmin, lo, hi, r = slab_of(xyz[b:b + k], nrm[b:b + k], n0, c)
            g = G["slab"][ie].astype(np.float64)
            tol = 1e-6 * (1.0 + r)
            assert g[0] <= cmin + 1e-7 and g[0] >= cmin - 1e-5
            assert g[1] <= lo + tol and g[2] >= hi - tol and g[3] >= r - tol
        assert (G["slab"][G["kind"] == 1] == 0).all()
        ctx.release(s)
    ctx.close()
