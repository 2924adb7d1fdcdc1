"""Voxelisation without device allocation (nimbus_voxelize_static), on the GPU.

Some callers cannot allocate device memory while they run: processes whose device
memory another allocator has carved up in advance, real-time loops that must not
wait on the allocator.  For them the library offers one entry point that writes
the voxel tables into buffers the caller owns and keeps every intermediate in a
fixed device array of the library.  These tests call it through the C ABI twice in
a row (two different clouds, so stale contents of the shared array would show) and
compare each result with the regular nimbus_voxelize + nimbus_scene_tables output
for the same cloud; check that a call after the first allocates nothing (the
library's allocation counter, its context's accounting and the device's free
memory are unchanged); and check each documented error.  The file is collected
last so a failing run has already run every other test.
"""
import numpy as np
import pytest

from paper_2402_13747_b300 import config, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2402_13747_b300 import _abi
    c = _abi.Context(0)
    yield c
    c.close()


def _device_cloud(sc):
    import torch
    d = torch.device("cuda", 0)
    return (torch.as_tensor(sc.xyz, device=d), torch.as_tensor(sc.nrm, device=d),
            torch.as_tensor(sc.label.astype(np.int64), device=d).to(torch.int32),
            torch.as_tensor(sc.material, device=d))


def _outputs(n_ie, n_cells):
    import torch
    d = torch.device("cuda", 0)
    z = lambda n, dt: torch.full((n,), -7, dtype=dt, device=d) if dt != torch.uint8 else \
        torch.full((n,), 77, dtype=dt, device=d)  # noqa: E731 (garbage so unwritten slots show)
    return dict(kind=z(n_ie, torch.int32), label=z(n_ie, torch.int32), gs=z(3 * n_ie, torch.int32),
                pcount=z(n_ie, torch.int32), rp=z(3 * n_ie, torch.float32), normal=z(3 * n_ie, torch.float32),
                bbc=z(3 * n_ie, torch.float32), material=z(n_ie, torch.uint8), ie_capacity=n_ie,
                cell_begin=z(n_cells, torch.int32), cell_count=z(n_cells, torch.int32),
                march=z(n_cells, torch.uint8), cell_capacity=n_cells)


def _check_against_regular(ctx, sc, p):
    h = ctx.voxelize_scene(sc, p)
    ref = ctx.scene_tables(h)
    ctx.release(h)
    n_ie, n_cells = int(ref["n_ie"]), int(np.prod(ref["dims"]))
    out = _outputs(n_ie + 5, n_cells + 5)
    xyz, nrm, lab, mat = _device_cloud(sc)
    info = ctx.voxelize_static(xyz, nrm, lab, out, material=mat, params=p)
    assert info["n_ie"] == n_ie and info["n_cells"] == n_cells
    np.testing.assert_array_equal(info["dims"], ref["dims"])
    np.testing.assert_array_equal(info["origin"], ref["origin"])
    g = {k: v.cpu().numpy() for k, v in out.items() if hasattr(v, "cpu")}
    np.testing.assert_array_equal(g["kind"][:n_ie], ref["kind"])
    np.testing.assert_array_equal(g["label"][:n_ie].astype(np.uint32), ref["label"])
    np.testing.assert_array_equal(g["gs"][:3 * n_ie].reshape(-1, 3), ref["gs"])
    np.testing.assert_array_equal(g["pcount"][:n_ie], ref["prange"][:, 1])
    np.testing.assert_array_equal(g["material"][:n_ie], ref["material"])
    np.testing.assert_allclose(g["rp"][:3 * n_ie].reshape(-1, 3), ref["rp"], atol=2e-6)
    np.testing.assert_allclose(g["normal"][:3 * n_ie].reshape(-1, 3), ref["normal"], atol=2e-6)
    np.testing.assert_allclose(g["bbc"][:3 * n_ie].reshape(-1, 3), ref["bbc"], atol=2e-6)
    np.testing.assert_array_equal(g["cell_count"][:n_cells], ref["cell_count"])
    occ = ref["cell_count"] > 0
    np.testing.assert_array_equal(g["cell_begin"][:n_cells][occ], ref["cell_begin"][occ])
    np.testing.assert_array_equal(g["march"][:n_cells], ref["march"])
    # slots beyond the outputs' sizes are untouched
    assert np.all(g["kind"][n_ie:] == -7) and np.all(g["march"][n_cells:] == 77)


def test_static_voxelize_matches_regular_twice_in_a_row(ctx):
    tiny = scenes.room_tiny()
    rng = np.random.default_rng(9)
    n = 50_000
    xyz = rng.uniform(0, 5, size=(n, 3)).astype(np.float32)
    nrm = rng.normal(size=(n, 3)).astype(np.float32)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    lab = rng.integers(0, 9, n).astype(np.uint32)
    rand = scenes.Scene("rand", xyz, nrm, lab, (lab % 4).astype(np.uint8))
    p = config.Params()
    _check_against_regular(ctx, tiny, p)
    _check_against_regular(ctx, rand, p)


def test_static_voxelize_rejects_oversized_clouds(ctx):
    import torch
    from paper_2402_13747_b300._abi import NimbusError, STATIC_MAX_POINTS
    n = STATIC_MAX_POINTS + 1
    d = torch.device("cuda", 0)
    xyz = torch.rand((n, 3), device=d)
    nrm = torch.zeros((n, 3), device=d)
    nrm[:, 2] = 1
    lab = torch.zeros(n, dtype=torch.int32, device=d)
    with pytest.raises(NimbusError) as ei:
        ctx.voxelize_static(xyz, nrm, lab, _outputs(16, 16), params=config.Params())
    assert "NIMBUS_STATIC_MAX_POINTS" in str(ei.value)


def _rand_scene(seed, n=50_000, extent=5.0, labels=9):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0, extent, size=(n, 3)).astype(np.float32)
    nrm = rng.normal(size=(n, 3)).astype(np.float32)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    lab = rng.integers(0, labels, n).astype(np.uint32)
    return scenes.Scene("rand", xyz, nrm, lab, (lab % 4).astype(np.uint8))


def test_static_voxelize_allocates_nothing(ctx):
    """After a first call (which resolves the fixed array's address and loads the
    kernels), a second call leaves the library's allocation counter, the context's
    memory accounting and the device's free memory exactly where they were."""
    import torch
    from paper_2402_13747_b300 import _abi
    sc = scenes.room_tiny()
    p = config.Params()
    xyz, nrm, lab, mat = _device_cloud(sc)
    out = _outputs(40_000, 40_000)
    first = ctx.voxelize_static(xyz, nrm, lab, out, material=mat, params=p)
    torch.cuda.synchronize()
    a0, m0, f0 = _abi.device_allocations(), ctx.memory_used(), torch.cuda.mem_get_info(0)[0]
    again = ctx.voxelize_static(xyz, nrm, lab, out, material=mat, params=p)
    torch.cuda.synchronize()
    a1, m1, f1 = _abi.device_allocations(), ctx.memory_used(), torch.cuda.mem_get_info(0)[0]
    assert (a1, m1, f1) == (a0, m0, f0)
    assert again["n_ie"] == first["n_ie"] > 0
    # the regular path does allocate, so the counter is live
    h = ctx.voxelize_scene(sc, p)
    assert _abi.device_allocations() > a1
    ctx.release(h)


def test_static_voxelize_rejects_oversized_grids(ctx):
    """A cloud within the point limit whose grid exceeds NIMBUS_STATIC_MAX_CELLS."""
    import torch
    from paper_2402_13747_b300._abi import NimbusError, STATIC_MAX_CELLS
    d = torch.device("cuda", 0)
    xyz = torch.tensor([[0.0, 0.0, 0.0], [60.0, 60.0, 60.0]], device=d)   # 123^3 voxels of 0.5 m
    nrm = torch.tensor([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]], device=d)
    lab = torch.zeros(2, dtype=torch.int32, device=d)
    assert 123 ** 3 > STATIC_MAX_CELLS
    with pytest.raises(NimbusError) as ei:
        ctx.voxelize_static(xyz, nrm, lab, _outputs(16, 16), params=config.Params())
    assert "NIMBUS_STATIC_MAX_CELLS" in str(ei.value) and ei.value.code == 1


def test_static_voxelize_rejects_negative_labels(ctx):
    """An int32 label array holding -1 reads as 2^32 - 1: refused by the 2^24 limit."""
    import torch
    from paper_2402_13747_b300._abi import NimbusError
    sc = _rand_scene(11, n=2000)
    xyz, nrm, lab, mat = _device_cloud(sc)
    lab[5] = -1
    with pytest.raises(NimbusError) as ei:
        ctx.voxelize_static(xyz, nrm, lab, _outputs(4096, 4096), material=mat, params=config.Params())
    assert "2^24" in str(ei.value) and ei.value.code == 1


def test_static_voxelize_reports_needed_sizes(ctx):
    """Capacities one short: NIMBUS_ERR_OVERFLOW with the regular path's sizes, and
    the outputs untouched.  An entity capacity one short is found after the count
    (both sizes known); a voxel capacity one short before it (n_ie = -1)."""
    import torch
    sc = _rand_scene(12, n=20_000)
    p = config.Params()
    h = ctx.voxelize_scene(sc, p)
    ref = ctx.scene_tables(h)
    ctx.release(h)
    n_ie, n_cells = int(ref["n_ie"]), int(np.prod(ref["dims"]))
    xyz, nrm, lab, mat = _device_cloud(sc)
    out = _outputs(n_ie - 1, n_cells)
    info = ctx.voxelize_static(xyz, nrm, lab, out, material=mat, params=p, allow_overflow=True)
    assert info["overflow"] and info["n_ie"] == n_ie and info["n_cells"] == n_cells
    np.testing.assert_array_equal(info["dims"], ref["dims"])
    torch.cuda.synchronize()
    assert bool((out["kind"] == -7).all()) and bool((out["march"] == 77).all())
    out = _outputs(n_ie, n_cells - 1)
    info = ctx.voxelize_static(xyz, nrm, lab, out, material=mat, params=p, allow_overflow=True)
    assert info["overflow"] and info["n_ie"] == -1 and info["n_cells"] == n_cells
    assert bool((out["kind"] == -7).all()) and bool((out["cell_count"] == -7).all())


@pytest.mark.parametrize("bad", ["null", "host"])
@pytest.mark.parametrize("field", ["kind", "material", "march"])
def test_static_voxelize_rejects_bad_outputs(ctx, bad, field):
    """A null or host output buffer with a non-zero capacity is an argument error,
    found before any device work."""
    from paper_2402_13747_b300._abi import NimbusError
    sc = _rand_scene(13, n=2000)
    xyz, nrm, lab, mat = _device_cloud(sc)
    out = _outputs(4096, 4096)
    out[field] = None if bad == "null" else out[field].cpu().numpy()
    with pytest.raises(NimbusError) as ei:
        ctx.voxelize_static(xyz, nrm, lab, out, material=mat, params=config.Params())
    assert "device pointers" in str(ei.value) and ei.value.code == 1
