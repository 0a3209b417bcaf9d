"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/cbct.h declares; argument validation rejects bad
input before any CUDA call."""
import ctypes

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_14212_gb300 import cbct
    return cbct.load()


def test_exports_every_declared_function(lib):
    from paper_2211_14212_gb300 import cbct
    names = cbct.declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _desc(**over):
    from paper_2211_14212_gb300 import cbct
    g = synth.config("small")
    kw = {f: getattr(g, f) for f in cbct.Geometry.FIELDS}
    kw.update(over)
    ang = np.ascontiguousarray(over.get("angles", g.angles), dtype=np.float64)
    d = cbct._Desc(int(kw["nx"]), int(kw["ny"]), int(kw["nz"]), float(kw["dx"]), float(kw["dy"]), float(kw["dz"]),
                   int(kw["nu"]), int(kw["nv"]), float(kw["du"]), float(kw["dv"]), float(kw["dso"]),
                   float(kw["dsd"]), int(over.get("nangles", ang.shape[0])),
                   ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return d, ang


@pytest.mark.parametrize("over", [
    {"nx": 0}, {"nv": -3}, {"dx": 0.0}, {"du": -1.0}, {"dsd": 100.0, "dso": 300.0},
    {"dso": 10.0, "dsd": 480.0},               # source inside the volume's cylinder
    {"dso": 300.0, "dsd": 310.0},              # detector inside the cylinder
    {"angles": np.array([0.0, np.nan])},
    {"nangles": 0},
])
def test_geometry_create_rejects_bad_descriptions(lib, over):
    from paper_2211_14212_gb300 import cbct
    d, keep = _desc(**over)
    h = ctypes.c_void_p()
    st = lib.cbct_geometry_create(ctypes.byref(d), ctypes.byref(h))
    assert st == cbct.CBCT_EINVAL
    assert not h.value
    assert len(lib.cbct_last_error()) > 0


def test_null_arguments(lib):
    from paper_2211_14212_gb300 import cbct
    assert lib.cbct_geometry_create(None, None) == cbct.CBCT_EINVAL
    assert lib.cbct_project(None, None, None, 0, None) == cbct.CBCT_EINVAL
    assert lib.cbct_backproject(None, None, None, 0, None) == cbct.CBCT_EINVAL
    assert lib.cbct_project_static(None, None, None, 0, None) == cbct.CBCT_EINVAL
    assert lib.cbct_backproject_voxel_driven(None, None, None, None) == cbct.CBCT_EINVAL
    assert lib.cbct_geometry_num_rays(None) == -1
    lib.cbct_geometry_destroy(None)          # no-op


def test_solver_argument_checks(lib):
    from paper_2211_14212_gb300 import cbct
    opts = cbct._Opts(0, 0.0, 0, 0, 0, 0)
    rep = cbct._Report()
    for fn in ("cbct_cgls_solve", "cbct_lsqr_solve", "cbct_lsmr_solve", "cbct_hybrid_lsqr_solve",
               "cbct_hybrid_lsmr_solve", "cbct_ab_gmres_solve", "cbct_ba_gmres_solve", "cbct_cgls_tv_solve"):
        assert getattr(lib, fn)(None, None, None, ctypes.byref(opts), ctypes.byref(rep), None) == cbct.CBCT_EINVAL


def test_launch_shape_calls_reject_null(lib):
    from paper_2211_14212_gb300 import cbct
    assert lib.cbct_geometry_set_launch(None, 2, 0) == cbct.CBCT_EINVAL
    assert lib.cbct_geometry_get_launch(None, None, None) == cbct.CBCT_EINVAL
    assert lib.cbct_geometry_autotune(None, 8, None, None) == cbct.CBCT_EINVAL
    assert lib.cbct_geometry_set_angle_block(None, 4) == cbct.CBCT_EINVAL
    assert lib.cbct_geometry_get_angle_block(None, None) == cbct.CBCT_EINVAL


def test_server_argument_checks(lib):
    from paper_2211_14212_gb300 import cbct
    h = ctypes.c_void_p()
    assert lib.cbct_server_create(None, ctypes.byref(h)) == cbct.CBCT_EINVAL
    for budget, slots, sched in ((0, 4, 0), (1 << 30, 0, 0), (1 << 30, 65, 0), (1 << 30, 4, 4), (1 << 30, 4, -1)):
        o = cbct._ServerOpts(budget, slots, 1, sched)
        assert lib.cbct_server_create(ctypes.byref(o), ctypes.byref(h)) == cbct.CBCT_EINVAL
    rid = ctypes.c_uint64()
    assert lib.cbct_server_submit(None, None, None, 0, None, ctypes.byref(rid)) == cbct.CBCT_EINVAL
    done = ctypes.c_int()
    assert lib.cbct_server_poll(None, 1, ctypes.byref(done)) == cbct.CBCT_EINVAL
    assert lib.cbct_server_wait(None, 1, 0.0, None, None, None) == cbct.CBCT_EINVAL
    lib.cbct_server_destroy(None)


def test_server_request_bytes(lib):
    """The budget charge of a server request, computed on the host: it
    counts the Krylov vectors (LSMR keeps one more volume than LSQR, each
    iteration adds two FP64 history entries) and grows with the scan."""
    from paper_2211_14212_gb300 import cbct
    g = synth.config("c1")
    lsqr = cbct.server_request_bytes(g, "lsqr", 10)
    lsmr = cbct.server_request_bytes(g, "lsmr", 10)
    padded_volume = g.nx * g.ny * (g.nz + 2) + 4
    assert lsqr >= 4 * (3 * g.num_rays + 3 * padded_volume)
    assert lsmr - lsqr >= 4 * padded_volume
    # buffers are rounded up to 1 KiB each
    assert cbct.server_request_bytes(g, "lsqr", 1000) - lsqr >= 2 * 990 * 8 - 1024
    more_angles = g.with_angles(synth.circular_angles(2 * g.nangles))
    assert cbct.server_request_bytes(more_angles, "lsqr", 10) - lsqr >= 4 * 3 * g.num_rays
    d, _angles = cbct._desc_of(g)
    out = ctypes.c_size_t()
    assert lib.cbct_server_request_bytes(None, 0, 10, ctypes.byref(out)) == cbct.CBCT_EINVAL
    assert lib.cbct_server_request_bytes(ctypes.byref(d), 0, 10, None) == cbct.CBCT_EINVAL
    assert lib.cbct_server_request_bytes(ctypes.byref(d), 2, 10, ctypes.byref(out)) == cbct.CBCT_EINVAL
    assert lib.cbct_server_request_bytes(ctypes.byref(d), 0, 0, ctypes.byref(out)) == cbct.CBCT_EINVAL
    bad = cbct._desc_of(g)[0]
    bad.nx = 0
    assert lib.cbct_server_request_bytes(ctypes.byref(bad), 0, 10, ctypes.byref(out)) == cbct.CBCT_EINVAL


def test_geometry_device_of_null(lib):
    assert lib.cbct_geometry_device(None) == -1


def test_binding_rejects_tensors_on_another_device():
    """The binding refuses a buffer on another CUDA device than the
    geometry's before calling the library (the library itself refuses a call
    made while another device is current)."""
    from paper_2211_14212_gb300 import cbct

    class Device:
        index = 1

    class Tensor:
        is_cuda = True
        device = Device()

        def is_contiguous(self):
            return True

        def numel(self):
            return 10

    with pytest.raises(ValueError, match="geometry lives on cuda:0"):
        cbct._require_cuda(Tensor(), "x", 10, 0)
    cbct._require_cuda(Tensor(), "x", 10, 1)
    cbct._require_cuda(Tensor(), "x", 10)
