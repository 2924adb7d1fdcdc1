"""The last level's walk bound (the CUDA trace's level_cone and march_cone_warp).

A cone of the last level can only emit paths to RXs, and an RX is screened only while
the cone's walk stands in a voxel within one voxel (L-infinity) of the RX's own voxel.
The walk therefore stops once the next voxel it would enter starts more than 4 voxel
edges beyond the farthest RX along the axis: every voxel that can screen an RX is
entered at most 2 sqrt(3) voxel edges beyond that RX's axial distance (its entry point
and the RX lie within two voxel edges of each other on every axis).  Here an exact
voxel walk (FP64, the same stepping rule as the CUDA walk: enter the neighbour across
the nearest boundary) checks that bound on random rays and RXs near them, and that it
is not loose by a whole margin: the entry of a screening voxel can lie more than one
voxel edge beyond the RX.
"""
import numpy as np

H = 0.5


def walk(apex, d, n_steps):
    """Voxels entered by the ray apex + t d (t >= 0) and the parameter at which each is
    entered (0 for the first)."""
    v = np.floor(apex / H).astype(np.int64)
    step = np.where(d >= 0, 1, -1)
    nxt = (v + (step > 0)) * H
    with np.errstate(divide="ignore"):
        tmax = np.where(d != 0, (nxt - apex) / d, np.inf)
        tdelta = np.where(d != 0, H / np.abs(d), np.inf)
    out = [(v.copy(), 0.0)]
    for _ in range(n_steps):
        a = int(np.argmin(tmax))
        t = float(tmax[a])
        v[a] += step[a]
        tmax[a] += tdelta[a]
        out.append((v.copy(), t))
    return out


def test_screening_voxels_start_within_the_bound():
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(3000):
        apex = rng.uniform(0, 20, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        # an RX near the ray, ahead of the apex, within a voxel or two of it
        t_rx = rng.uniform(0.0, 15.0)
        rx = apex + t_rx * d + rng.uniform(-1.5 * H, 1.5 * H, 3)
        u = np.floor(rx / H).astype(np.int64)
        t_axial = float((rx - apex) @ d)
        for v, t_in in walk(apex, d, int(40.0 / H)):
            if np.max(np.abs(v - u)) <= 1:
                assert t_in <= t_axial + 2.0 * np.sqrt(3.0) * H + 1e-9, (t_in, t_axial)
                worst = max(worst, t_in - t_axial)
    # the bound has room to spare against the margin the walk uses (4 edges) and is
    # not far from tight: a screening voxel can start more than one edge beyond the RX
    assert H < worst <= 2.0 * np.sqrt(3.0) * H < 4.0 * H
