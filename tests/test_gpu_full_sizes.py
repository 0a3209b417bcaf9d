"""GPU parity at the two largest benchmark configurations, through the C ABI.

512^3 / 768 x 512 / 720 angles (the precision-study scan) and 1024^3 /
1536^2 / 1600 angles at magnification 6 (the micro-CT scan) are too large for
whole oracle products, so the oracle computes sampled rays and voxels one by
one; the GPU dot-product test covers every element.  At 512^3 the hybrid
LSQR precision variants (FP32 / FP16 / BF16 storage) are run at the full
iteration count and compared with each other.
"""
import numpy as np
import pytest

import oracle
import synth

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


def rel_l2(a, ref):
    a = np.asarray(a, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def elementwise_ok(got, ref, rel=REL_L2):
    """4x the relative bar per element plus 1e-5 of the largest value (the FP32
    plane-position floor, as in the smaller projector tests)."""
    return np.abs(got - ref) <= 4 * rel * np.abs(ref) + 1e-5 * np.abs(ref).max()


def ddot(a, b, chunk=1 << 26):
    """FP64 dot product of two FP32 device tensors, in chunks (bounded memory)."""
    a, b = a.reshape(-1), b.reshape(-1)
    return sum(float(a[i:i + chunk].double().dot(b[i:i + chunk].double())) for i in range(0, a.numel(), chunk))


def dot_test(cbct, geom, g, x_dev, seed):
    import torch
    gen = torch.Generator(device="cuda").manual_seed(seed)
    y = torch.rand(g.proj_shape, device="cuda", generator=gen)
    ax = cbct.project(geom, x_dev)
    aty = cbct.backproject(geom, y)
    lhs, rhs = ddot(ax, y), ddot(x_dev, aty)
    assert abs(lhs - rhs) <= 1e-5 * (ddot(ax, ax) * ddot(y, y)) ** 0.5


def forward_sampled(cbct, geom, g, x, seed, count):
    import torch
    rays = np.random.default_rng(seed).choice(g.num_rays, size=count, replace=False)
    y = cbct.project(geom, torch.from_numpy(x).cuda())
    got = y.view(-1)[torch.from_numpy(rays).cuda()].double().cpu().numpy()
    del y
    ref = oracle.project_rays(g, x, rays)
    assert rel_l2(got, ref) <= REL_L2
    assert elementwise_ok(got, ref).all()


# ----------------------------------------------------------- 512^3, 720 angles
@pytest.fixture(scope="module")
def c3():
    g = synth.config("c3")
    return g, synth.ellipsoid_phantom(g, 10, seed=2, scale=0.02)


def test_c3_forward_sampled_rays(cbct, c3):
    g, x = c3
    forward_sampled(cbct, cbct.Geometry(g), g, x, 21, 2000)


def test_c3_backward_sampled_voxels(cbct, c3):
    import torch
    g, _ = c3
    geom = cbct.Geometry(g)
    yh = synth.random_projections(g, 22).astype(np.float32)
    xb = cbct.backproject(geom, torch.from_numpy(yh).cuda()).cpu().numpy().ravel()
    vox = np.random.default_rng(23).choice(g.num_voxels, size=200, replace=False)
    ref = oracle.backproject_voxels(g, yh.astype(np.float64), vox)
    got = xb[vox].astype(np.float64)
    assert rel_l2(got, ref) <= REL_L2
    assert elementwise_ok(got, ref).all()


def test_c3_dot_product(cbct, c3):
    import torch
    g, x = c3
    dot_test(cbct, cbct.Geometry(g), g, torch.from_numpy(x).cuda(), 24)


def test_c3_hybrid_precision_variants(cbct, c3):
    """Hybrid LSQR, 50 iterations, GCV, on the noisy 512^3 scan: FP16 and BF16
    storage stay within their storage precision of the FP32 run (relative
    2-norm: FP16 <= 5e-3, BF16 <= 3e-2), and choose nearly the same lambda_k."""
    import torch
    g, x = c3
    geom = cbct.Geometry(g)
    b = cbct.project(geom, torch.from_numpy(x).cuda()).cpu().numpy()
    b = torch.from_numpy(synth.poisson_log_noise(b, 1e5, seed=25).astype(np.float32)).cuda()
    runs = {}
    for storage in ("f32", "f16", "bf16"):
        xs, rep = cbct.hybrid_lsqr(geom, b, 50, rule="gcv", storage=storage)
        assert rep.iters_done == 50 and np.isfinite(rep.lam).all()
        runs[storage] = (xs.float().cpu().numpy(), rep)
        del xs
    x32, r32 = runs["f32"]
    for storage, bound in (("f16", 5e-3), ("bf16", 3e-2)):
        xs, rep = runs[storage]
        err = rel_l2(xs, x32)
        print("%s vs f32 after 50 iterations: %.3g (lambda_50 %.4g vs %.4g)" % (storage, err, rep.lam[-1], r32.lam[-1]))
        assert err <= bound
        assert abs(rep.lam[-1] - r32.lam[-1]) <= 10 * bound * r32.lam[-1]


# ------------------------------------------------- 1024^3, 1600 angles (micro-CT)
@pytest.fixture(scope="module")
def c5():
    g = synth.config("c5")
    return g, synth.ellipsoid_phantom(g, 4, seed=4, scale=0.02, cylinder=True)


def test_c5_forward_sampled_rays(cbct, c5):
    g, x = c5
    forward_sampled(cbct, cbct.Geometry(g), g, x, 31, 1000)


def test_c5_dot_product(cbct, c5):
    import torch
    g, x = c5
    dot_test(cbct, cbct.Geometry(g), g, torch.from_numpy(x).cuda(), 32)
