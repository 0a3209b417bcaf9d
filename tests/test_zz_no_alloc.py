"""cbct_project_static (forward projection with its scratch in a fixed device
array instead of a per-call allocation) gives exactly what cbct_project gives,
on consecutive calls that leave the shared scratch dirty, allocates no device
memory from the stream-ordered pool the library otherwise uses, and rejects
volumes whose padded copy exceeds its 66 MiB scratch.  This file is collected
last, so it also runs after every other GPU test has used the library."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cbct():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_14212_gb300 import cbct as mod
    return mod


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return t if dtype is None else t.to(dtype)


@pytest.mark.parametrize("name", ["small", "c1"])
def test_consecutive_calls_equal_cbct_project(cbct, name):
    import torch
    g = synth.config(name)
    geom = cbct.Geometry(g)
    # two different volumes, one after the other: the second call finds the
    # first one's data in the scratch
    for seed in (1, 2):
        x = dev(synth.ellipsoid_phantom(g, 6, seed=seed))
        ref = cbct.project(geom, x)
        got = cbct.project_static(geom, x)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_largest_volume_and_reduced_storage(cbct):
    """A 256^3 FP32 volume (67.6 MB padded) nearly fills the scratch; FP16
    storage uses half of it."""
    import torch
    g = synth.Geometry(256, 256, 256, 1.0, 1.0, 1.0, 128, 96, 3.2, 3.2, 1000.0, 1536.0,
                       synth.circular_angles(12))
    geom = cbct.Geometry(g)
    for seed, dtype in ((3, None), (4, torch.float16), (5, None)):
        x = dev(synth.random_volume(g, seed), dtype)
        ref = cbct.project(geom, x)
        got = cbct.project_static(geom, x)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def _cudart():
    for name in ("libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.fail("libcudart.so not found")


# cudaMemPoolAttr values of the CUDA runtime API
USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8


def test_no_pool_allocation(cbct):
    """Device memory in use from the current device's default stream-ordered
    pool (where cbct_project takes its scratch) does not grow during calls of
    cbct_project_static: high-water mark reset after the reference calls,
    read after several static calls."""
    import torch
    rt = _cudart()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    g = synth.config("c1")
    geom = cbct.Geometry(g)
    x = dev(synth.ellipsoid_phantom(g, 6, seed=7))
    ref = cbct.project(geom, x)
    out = torch.empty_like(ref)
    cbct.project_static(geom, x, out=out)
    torch.cuda.synchronize()
    cur = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, USED_MEM_CURRENT, ctypes.byref(cur)) == 0
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0
    for _ in range(3):
        cbct.project_static(geom, x, out=out)
    torch.cuda.synchronize()
    high = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, USED_MEM_HIGH, ctypes.byref(high)) == 0
    assert high.value <= cur.value
    assert torch.equal(out, ref)


def test_oversized_volume_rejected(cbct):
    g = synth.Geometry(272, 256, 256, 1.0, 1.0, 1.0, 64, 64, 6.0, 6.0, 1000.0, 1536.0,
                       synth.circular_angles(4))
    geom = cbct.Geometry(g)
    x = dev(np.zeros(g.vol_shape, np.float32))
    with pytest.raises(cbct.CbctError) as e:
        cbct.project_static(geom, x)
    assert e.value.status == cbct.CBCT_EINVAL
    assert "66 MiB" in str(e.value)
