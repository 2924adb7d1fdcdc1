"""Method parameters (configuration values only; no arithmetic of the method).

Table 1 of the paper fixes the carrier frequency (60 GHz), voxel size (0.5 m),
division factor D_v (2), duplicate limit kappa (100), the maximum number of
interactions (5), the convergence threshold delta (1e-4) and the number of
refinement iterations rho (2000).  The paper leaves the remaining values open;
the readings chosen here are the defaults of ``Params`` and are used unchanged
by both the CUDA path and the FP64 oracle.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict, replace
import math

__all__ = ["Params", "SegmentParams", "params_for", "NONE_LABEL"]

NONE_LABEL = 0xFFFFFFFF


@dataclass(frozen=True)
class Params:
    # voxelisation (Section 2.1, Table 1)
    voxel_size: float = 0.5          # low-resolution voxel edge h [m]
    dv: int = 2                      # voxel division factor D_v
    # coarse path tracing (Section 2.2)
    max_refl: int = 2
    max_diff: int = 0
    max_int: int = -1                # -1: max_refl + max_diff
    kappa: int = 100                 # duplicate limit per (TX, RX, label sequence)
    cone_half_angle_deg: float = 4.0     # constant cone apex half-angle alpha
    launch_spacing_deg: float = 0.5      # uniform sphere-grid spacing Delta of the TX launch
    n_launch: int = 0                # 0: round(4*pi/Delta^2) Fibonacci directions
    launch_mode: int = 0             # 0: uniform sphere grid; 1: a ray toward every IE and RX (Section 2.2.2)
    # point-set intersection (Section 2.2.1, Eq. 1)
    sdf_sigma: float = 0.125         # Gaussian weight width [m] (h_s / 2)
    sdf_eps: float = 1e-3            # "near zero" |f| threshold [m]
    sdf_max_steps: int = 64
    vis_ignore: float = -1.0         # self-hit ignore distance; -1: h_s*sqrt(3)
    sep_eps: float = 0.0625          # reflection separation-plane offset [m] (h_s / 4)
    # refinement (Section 2.3, Table 1)
    delta: float = 1e-4
    rho: int = 2000
    gamma: float = 0.5               # GD step = gamma / (1/a + 1/b)
    grad_stop: float = 1e-6          # early exit once ||grad|| < grad_stop (< delta)
    freq_hz: float = 60e9

    @property
    def h_s(self) -> float:
        return self.voxel_size / self.dv

    @property
    def max_interactions(self) -> int:
        return self.max_int if self.max_int >= 0 else self.max_refl + self.max_diff

    @property
    def ignore_dist(self) -> float:
        return self.vis_ignore if self.vis_ignore >= 0 else self.h_s * math.sqrt(3.0)

    @property
    def launch_count(self) -> int:
        if self.n_launch > 0:
            return self.n_launch
        d = math.radians(self.launch_spacing_deg)
        return int(round(4.0 * math.pi / (d * d)))

    def replace(self, **kw) -> "Params":
        return replace(self, **kw)

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass(frozen=True)
class SegmentParams:
    """Automatic labels and exterior edges for unlabelled clouds.

    The paper takes its labels from a plane-fitting segmentation and places its
    diffraction edges by hand.  These are the values of the reading used here,
    shared by the CUDA path and the oracle.
    """
    voxel_size: float = 0.5          # the voxel grid of the voxelisation
    dv: int = 2
    min_points: int = 3              # fewest points of a subvoxel that can be planar
    flat_max: float = 0.02           # planar: smallest covariance eigenvalue <= flat_max * trace ...
    spread_min: float = 0.05         # ... and the middle one >= spread_min * trace (not a line of points)
    join_angle_deg: float = 10.0     # neighbouring planes joined when their normals agree this well ...
    join_dist: float = 0.03          # ... and each centroid is this close to the other's plane [m]
    edge_angle_deg: float = 30.0     # exterior edge between surfaces at least this far apart ...
    edge_min_groups: int = 4         # ... each with at least this many planar subvoxels

    @property
    def h_s(self) -> float:
        return self.voxel_size / self.dv

    def replace(self, **kw) -> "SegmentParams":
        return replace(self, **kw)


def params_for(scene, **overrides) -> Params:
    """Defaults for a scene: its reflection/diffraction limits plus overrides."""
    kw = dict(max_refl=scene.max_refl, max_diff=scene.max_diff)
    kw.update(overrides)
    return Params(**kw)
