"""The last level's RX pre-test (rx_in_reach in the CUDA trace).

A cone of the last level emits no child, so it can only produce coarse paths to the
RXs its march screens in; when no RX could pass that screening the march is skipped.
The skip is exact only if the pre-test accepts every RX the screening accepts.  The
screening is cone_sphere(apex, axis, sin_a, cos_a, rx, r_sub) and the separation
planes, computed in FP32; the pre-test is the same inequalities loosened by
1e-5 (|v| + 1) m.  Here both are written out in numpy FP32, as the kernel computes
them, and checked on RXs placed at the cone's and the planes' boundaries (where a
rounding difference could flip the screening) and at distances from 1 cm to 300 m:
wherever the FP32 screening, or the screening in FP64 on the same FP32 inputs,
accepts, the pre-test accepts too.  The GPU side of the claim (the skip drops no
coarse path) is the parity tests', which compare every coarse and exact set with the
oracle at full depth.
"""
import numpy as np

f4 = np.float32


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def screening(apex, axis, sin_a, cos_a, pn, sep, C, r, dt):
    """cone_sphere && the reflection plane test, in dtype dt, on the FP32 values the
    kernel holds (apex, axis, RX position and parameters rounded to FP32 first)."""
    A, ax, P, N = (x.astype(f4).astype(dt) for x in (apex, axis, C, pn))
    r, sin_a, cos_a, sep = (dt(f4(x)) for x in (r, sin_a, cos_a, sep))
    v = P - A
    d2 = np.sum(v * v, axis=-1, dtype=dt)
    r2 = r * r
    t = np.sum(v * ax, axis=-1, dtype=dt)
    cone = (d2 <= r2) | (t + r * sin_a >= cos_a * np.sqrt(np.maximum(d2 - r2, dt(0))))
    return cone & (np.sum(v * N, axis=-1, dtype=dt) > sep)


def pretest(apex, axis, sin_a, cos_a, pn, sep, C, r):
    """The kernel's loosened test, FP32."""
    A, ax, P, N = (x.astype(f4) for x in (apex, axis, C, pn))
    r, sin_a, cos_a, sep = f4(r), f4(sin_a), f4(cos_a), f4(sep)
    v = P - A
    d2 = np.sum(v * v, axis=-1, dtype=f4)
    tol = f4(1e-5) * (np.sqrt(d2) + f4(1))
    r2 = r * r
    cone = (d2 <= r2 * f4(1.001) + f4(1e-6)) | (
        np.sum(v * ax, axis=-1, dtype=f4) + r * sin_a + tol >= cos_a * np.sqrt(np.maximum(d2 - r2, f4(0))))
    return cone & (np.sum(v * N, axis=-1, dtype=f4) > sep - tol)


def test_pretest_accepts_whatever_the_screening_accepts():
    rng = np.random.default_rng(7)
    n = 400_000
    apex = rng.uniform(-150, 150, (n, 3))
    axis = _unit(rng.normal(size=(n, 3)))
    alpha = np.deg2rad(rng.choice([0.25, 0.5, 1.0, 2.0, 4.0], n))
    r = rng.choice([0.0433, 0.0866, 0.2165], n)
    dist = np.exp(rng.uniform(np.log(0.01), np.log(300.0), n))
    # an RX on the boundary of the cone around the sphere (the angle at which the
    # sphere touches the cone), nudged by a few ppm either way
    perp = _unit(np.cross(axis, rng.normal(size=(n, 3))))
    theta = alpha + np.arcsin(np.minimum(r / dist, 1.0)) * rng.uniform(0.999, 1.001, n)
    C = apex + dist[:, None] * (np.cos(theta)[:, None] * axis + np.sin(theta)[:, None] * perp)
    # a reflection plane through the apex whose distance to the RX is near sep_eps
    sep = 1e-3
    v = C - apex
    pn = _unit(rng.normal(size=(n, 3)))
    pn = _unit(pn - (np.sum(pn * v, axis=1) / np.sum(v * v, axis=1))[:, None] * v)   # pn orthogonal to v ...
    pn = _unit(pn + ((sep + rng.uniform(-1e-5, 1e-5, n)) / np.linalg.norm(v, axis=1))[:, None] * _unit(v))
    sin_a, cos_a = np.sin(alpha), np.cos(alpha)
    s32 = screening(apex, axis, sin_a, cos_a, pn, sep, C, r, f4)
    s64 = screening(apex, axis, sin_a, cos_a, pn, sep, C, r, np.float64)
    pre = pretest(apex, axis, sin_a, cos_a, pn, sep, C, r)
    # the sample sits on the boundaries: both outcomes occur often
    assert 0.1 < s32.mean() < 0.9 and 0.1 < s64.mean() < 0.9
    assert not np.any(s32 & ~pre), np.nonzero(s32 & ~pre)[0][:5]
    assert not np.any(s64 & ~pre), np.nonzero(s64 & ~pre)[0][:5]
    # and the pre-test is not vacuous: an RX a metre or more away, 63 degrees off the
    # axis, is rejected
    far = apex + dist[:, None] * _unit(perp + 0.5 * axis)
    away = dist > 1.0
    assert not pretest(apex, axis, sin_a, cos_a, axis, -1.0, far, r)[away].any()
