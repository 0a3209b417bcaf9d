"""GPU parity of the projectors against the FP64 oracle (through the C ABI).

Bar: projections and backprojections within 1e-5 relative L2 of the oracle
(plus an element-wise bound), the GPU dot-product test within 1e-5.
Full-size configurations are checked on sampled rays / voxels, which the
oracle computes one by one.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import krylov

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


@pytest.fixture(scope="module")
def cbct():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_14212_gb300 import cbct as mod
    return mod


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(a, ref):
    return float(np.linalg.norm(np.asarray(a, np.float64).ravel() - ref.ravel()) / np.linalg.norm(ref))


def elementwise_tol(ref, rel=REL_L2):
    """Per-element bound: 4x the relative bar on the element, plus a floor of
    1e-5 of the largest value.  The floor is the FP32 geometry limit: the plane
    positions relative to each ray's origin are rounded to FP32 (~1e-5 mm of
    lateral shift at 100-250 mm), which a ray meeting a plane at a glancing
    angle turns into a crossing misplaced by ~1e-5..1e-4 mm along the ray; at a
    unit density jump that moves ~1e-5 of a full ray sum."""
    return 4 * rel * np.abs(ref) + 1e-5 * np.abs(ref).max()


def assert_elementwise(got, ref, rel=REL_L2, what="", idx=None):
    tol = elementwise_tol(ref, rel)
    bad = np.abs(got - ref) > tol
    if bad.any():
        w = int(np.argmax(np.abs(got - ref) - tol))
        where = int(idx[w]) if idx is not None else w
        raise AssertionError("%s: %d elements off; worst at %d: got %r ref %r tol %r"
                             % (what, int(bad.sum()), where, got.flat[w], ref.flat[w], tol.flat[w]))


def assert_close(got, ref, rel=REL_L2):
    got = np.asarray(got, np.float64).reshape(ref.shape)
    if not np.any(ref):
        assert not np.any(got)
        return
    assert rel_l2(got, ref) <= rel
    bad = np.abs(got - ref) > elementwise_tol(ref, rel)
    assert not bad.any(), "%d elements off, worst %g" % (bad.sum(), np.abs(got - ref)[bad].max())


GEOMS = {
    "tiny": synth.config("tiny"),
    "small": synth.config("small"),     # ragged: 40x36x28 volume, 77x45 detector, non-cubic voxels
    "c1": synth.config("c1"),
    # odd detector counts: the central row / column rays lie in voxel planes
    "odd": synth.Geometry(20, 22, 18, 1.0, 1.0, 1.0, 33, 25, 1.1, 1.0, 150.0, 240.0,
                          np.radians([0.0, 45.0, 90.0, 180.0, 271.0])),
    # single voxel, single pixel rows, one angle
    "one_voxel": synth.Geometry(1, 1, 1, 2.0, 2.0, 2.0, 9, 7, 0.5, 0.5, 50.0, 80.0, np.radians([12.0])),
    "one_pixel": synth.Geometry(16, 16, 16, 1.0, 1.0, 1.0, 1, 1, 1.0, 1.0, 100.0, 150.0, np.radians([0.0, 33.0])),
    # short scan, high magnification
    "short_scan": synth.Geometry(48, 48, 32, 0.25, 0.25, 0.25, 96, 64, 0.6, 0.6, 40.0, 240.0,
                                 synth.circular_angles(37, 200.0)),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_forward_matches_oracle(cbct, name):
    g = GEOMS[name]
    geom = cbct.Geometry(g)
    for x in (synth.ellipsoid_phantom(g, 6, seed=5), synth.random_volume(g, 6).astype(np.float32),
              np.ones(g.vol_shape, np.float32)):
        y = cbct.project(geom, dev(x)).cpu().numpy()
        assert_close(y, oracle.project(g, x.astype(np.float64)))


@pytest.mark.parametrize("name", list(GEOMS))
def test_backward_matches_oracle(cbct, name):
    g = GEOMS[name]
    geom = cbct.Geometry(g)
    y = synth.random_projections(g, 7).astype(np.float32)
    x = cbct.backproject(geom, dev(y)).cpu().numpy()
    assert_close(x, oracle.backproject(g, y.astype(np.float64), 8))


@pytest.mark.parametrize("name", ["small", "short_scan", "odd"])
def test_every_launch_shape_matches_oracle(cbct, name):
    """All forward / transpose launch shapes compute the same A and A^T."""
    g = GEOMS[name]
    geom = cbct.Geometry(g)
    x = synth.random_volume(g, 21).astype(np.float32)
    y = synth.random_projections(g, 22).astype(np.float32)
    y_ref = oracle.project(g, x.astype(np.float64))
    x_ref = oracle.backproject(g, y.astype(np.float64), 8)
    for fr in cbct.FWD_ROWS:
        for bc in range(len(cbct.BWD_CONFIGS)):
            cbct.set_launch(geom, fr, bc)
            assert cbct.get_launch(geom) == (fr, bc)
            assert_close(cbct.project(geom, dev(x)).cpu().numpy(), y_ref)
            assert_close(cbct.backproject(geom, dev(y)).cpu().numpy(), x_ref)
    with pytest.raises(cbct.CbctError):
        cbct.set_launch(geom, 3, 0)


@pytest.mark.parametrize("name", ["small", "short_scan"])
def test_transpose_in_angle_passes_matches_oracle(cbct, name):
    """The transpose summed in passes over blocks of angles (FP32 running sums
    between passes) computes the same A^T y, for every block size."""
    g = GEOMS[name]
    geom = cbct.Geometry(g)
    y = synth.random_projections(g, 31).astype(np.float32)
    x_ref = oracle.backproject(g, y.astype(np.float64), 8)
    for block in (1, 4, g.nangles - 1, g.nangles):
        cbct.set_angle_block(geom, block)
        assert cbct.get_angle_block(geom) == block
        for bc in range(len(cbct.BWD_CONFIGS)):
            cbct.set_launch(geom, 2, bc)
            assert_close(cbct.backproject(geom, dev(y)).cpu().numpy(), x_ref)
    cbct.set_angle_block(geom, 0)
    assert cbct.get_angle_block(geom) == g.nangles        # small scans fit in one pass
    with pytest.raises(cbct.CbctError):
        cbct.set_angle_block(geom, -1)


def test_autotune_picks_a_valid_shape(cbct, tmp_path):
    g = synth.config("c1")
    geom = cbct.Geometry(g)
    cache = tmp_path / "tune.json"
    res = cbct.autotune(geom, max_angles=8, cache=cache)
    assert res["fwd_rows"] in cbct.FWD_ROWS and res["bwd_shape"] in cbct.BWD_CONFIGS and not res["cached"]
    assert all(t > 0 for t in res["forward_ms"].values()) and all(t > 0 for t in res["backward_ms"].values())
    x = synth.random_volume(g, 23).astype(np.float32)
    assert_close(cbct.project(geom, dev(x)).cpu().numpy(), oracle.project(g, x.astype(np.float64)))
    # a second scan of the same class takes the cached shapes without timing
    geom2 = cbct.Geometry(g)
    res2 = cbct.autotune(geom2, max_angles=8, cache=cache)
    assert res2["cached"] and cbct.get_launch(geom2) == (res["fwd_rows"], res["bwd_config"])


@pytest.mark.parametrize("name", ["small", "c1", "short_scan"])
def test_gpu_dot_product(cbct, name):
    import torch
    g = GEOMS[name]
    geom = cbct.Geometry(g)
    x = dev(synth.random_volume(g, 8))
    y = dev(synth.random_projections(g, 9) - 0.5)
    ax = cbct.project(geom, x).double()
    aty = cbct.backproject(geom, y).double()
    lhs = torch.dot(ax.ravel(), y.double().ravel()).item()
    rhs = torch.dot(x.double().ravel(), aty.ravel()).item()
    assert abs(lhs - rhs) <= 1e-5 * ax.norm().item() * y.double().norm().item()


def test_nnz_count_matches_oracle(cbct):
    g = synth.config("c1")
    geom = cbct.Geometry(g)
    n_gpu = cbct.count_nnz(geom)
    n_ref = oracle.nnz(g)
    # both count positive-length segments; FP32 and FP64 disagree only on slivers
    # (rays passing within rounding distance of a voxel edge)
    assert abs(n_gpu - n_ref) <= 1e-3 * n_ref


def test_results_independent_of_stream_and_repeat(cbct):
    import torch
    g = synth.config("c1")
    geom = cbct.Geometry(g)
    x = dev(synth.ellipsoid_phantom(g, 10, seed=0))
    y1 = cbct.project(geom, x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y2 = cbct.project(geom, x, stream=s)
    s.synchronize()
    assert torch.equal(y1, y2)       # one thread per ray, fixed order: bit-identical


@pytest.mark.parametrize("dtype,bound", [("f16", 2e-3), ("bf16", 1.2e-2)])
def test_reduced_precision_storage_error(cbct, dtype, bound):
    """FP16/BF16 storage with compensated FP32 ray sums: error vs the FP64 oracle is
    set by rounding the stored values (unit roundoff 4.9e-4 / 3.9e-3)."""
    import torch
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    g = synth.config("c1")
    geom = cbct.Geometry(g)
    x = synth.ellipsoid_phantom(g, 10, seed=0)
    y = cbct.project(geom, dev(x).to(tdt)).float().cpu().numpy()
    ref = oracle.project(g, x.astype(np.float64))
    err_f = rel_l2(y, ref)
    yr = synth.random_projections(g, 3).astype(np.float32)
    xb = cbct.backproject(geom, dev(yr).to(tdt)).float().cpu().numpy()
    err_b = rel_l2(xb, oracle.backproject(g, yr.astype(np.float64), 8))
    print("%s storage: forward rel err %.3g, backward rel err %.3g" % (dtype, err_f, err_b))
    assert err_f <= bound and err_b <= bound


# --------------------------------------------------------------- full sizes
@pytest.fixture(scope="module")
def c2_inputs():
    g = synth.config("c2")
    x = synth.ellipsoid_phantom(g, 10, seed=1, scale=0.02)
    return g, x


@pytest.fixture(scope="module")
def c2_geom(cbct, c2_inputs):
    """The 256^3 geometry in the launch configuration the benchmark times (its
    autotuner run on 32 angles)."""
    g, _ = c2_inputs
    geom = cbct.Geometry(g)
    cbct.autotune(geom, max_angles=32)
    return geom


def test_c2_forward_sampled_rays(cbct, c2_inputs, c2_geom):
    g, x = c2_inputs
    geom = c2_geom
    y = cbct.project(geom, dev(x)).cpu().numpy().ravel()
    rng = np.random.default_rng(11)
    rays = rng.choice(g.num_rays, size=3000, replace=False)
    ref = oracle.project_rays(g, x.astype(np.float64), rays)
    got = y[rays].astype(np.float64)
    assert rel_l2(got, ref) <= REL_L2
    assert_elementwise(got, ref, what="sampled rays", idx=rays)


def test_c2_backward_sampled_voxels(cbct, c2_inputs, c2_geom):
    g, _ = c2_inputs
    geom = c2_geom
    yh = synth.random_projections(g, 12).astype(np.float32)
    x = cbct.backproject(geom, dev(yh)).cpu().numpy().ravel()
    rng = np.random.default_rng(13)
    vox = rng.choice(g.num_voxels, size=400, replace=False)
    ref = oracle.backproject_voxels(g, yh.astype(np.float64), vox)
    got = x[vox].astype(np.float64)
    assert rel_l2(got, ref) <= REL_L2
    assert_elementwise(got, ref, what="sampled voxels", idx=vox)


def test_c2_dot_product(cbct, c2_inputs, c2_geom):
    import torch
    g, x = c2_inputs
    geom = c2_geom
    xd = dev(x)
    gen = torch.Generator(device="cuda").manual_seed(5)
    y = torch.rand(g.proj_shape, device="cuda", generator=gen)
    ax = cbct.project(geom, xd).double()
    aty = cbct.backproject(geom, y).double()
    lhs = torch.dot(ax.ravel(), y.double().ravel()).item()
    rhs = torch.dot(xd.double().ravel(), aty.ravel()).item()
    assert abs(lhs - rhs) <= 1e-5 * ax.norm().item() * y.double().norm().item()


# the voxel-driven interpolating backprojector (an approximation of A^T, Sec. 2.1.4)
VD_GEOMS = dict(GEOMS, tall=synth.Geometry(20, 18, 100, 1.0, 1.0, 0.5, 40, 72, 1.0, 1.0, 120.0, 200.0,
                                           synth.circular_angles(11)))   # several 64-voxel z blocks, ragged


@pytest.mark.parametrize("name", list(VD_GEOMS))
def test_voxel_driven_backprojector_matches_oracle(cbct, name):
    """The kernel against the oracle's FP64 voxel-driven backprojector, on
    random projections and on projections of a phantom.  An FP32 emulation of
    the kernel's arithmetic stays below 4e-7 relative L2 on these cases, so the
    projectors' 1e-5 bar applies unchanged."""
    g = VD_GEOMS[name]
    geom = cbct.Geometry(g)
    bp = krylov.VoxelDrivenBackprojector(g)
    for y in (synth.random_projections(g, 7), oracle.project(g, synth.ellipsoid_phantom(g, 6, seed=5)
                                                             .astype(np.float64))):
        x = cbct.backproject_voxel_driven(geom, dev(y)).cpu().numpy()
        assert_close(x, bp(np.asarray(y, np.float64)).reshape(g.vol_shape))


def test_voxel_driven_backprojector_is_not_the_transpose(cbct):
    """It approximates A^T (B 1 / A^T 1 averages to within 10% of one inside
    the volume) but is not it: <A x, y> != <x, B y> beyond rounding."""
    g = synth.config("c1")
    geom = cbct.Geometry(g)
    ones = dev(np.ones(g.proj_shape, np.float32))
    bt = cbct.backproject(geom, ones).cpu().numpy().astype(np.float64)
    bv = cbct.backproject_voxel_driven(geom, ones).cpu().numpy().astype(np.float64)
    inner = (slice(2, -2),) * 3
    assert 0.9 < (bv[inner] / bt[inner]).mean() < 1.1
    x = (synth.random_volume(g, 3) - 0.5).astype(np.float32)        # zero-mean: no common bulk term
    y = (synth.random_projections(g, 4) - 0.5).astype(np.float32)
    ax = cbct.project(geom, dev(x)).cpu().numpy().astype(np.float64)
    by = cbct.backproject_voxel_driven(geom, dev(y)).cpu().numpy().astype(np.float64)
    lhs, rhs = float(np.vdot(ax, y)), float(np.vdot(x, by))
    assert abs(lhs - rhs) > 0.1 * abs(lhs)
