"""cbct_project_static (forward projection with its scratch in a fixed device
array instead of a per-call allocation) gives exactly what cbct_project gives,
on consecutive calls that leave the shared scratch dirty, and rejects volumes
larger than its 64 MiB scratch.  This file is collected last, so it also runs
after every other GPU test has used the library."""
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
    """A 256^3 FP32 volume fills the scratch exactly; FP16 storage uses half of it."""
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


def test_oversized_volume_rejected(cbct):
    g = synth.Geometry(257, 256, 256, 1.0, 1.0, 1.0, 64, 64, 6.0, 6.0, 1000.0, 1536.0,
                       synth.circular_angles(4))
    geom = cbct.Geometry(g)
    x = dev(np.zeros(g.vol_shape, np.float32))
    with pytest.raises(cbct.CbctError) as e:
        cbct.project_static(geom, x)
    assert e.value.status == cbct.CBCT_EINVAL
    assert "64 MiB" in str(e.value)
