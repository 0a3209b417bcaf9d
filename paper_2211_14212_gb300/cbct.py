"""Python binding of libcbct.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/cbct.h; all
computation happens in the library's CUDA kernels.  PyTorch provides device
memory and the current stream.  There is no CPU fallback: if libcbct.so cannot
be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcbct.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "cbct.h")

CBCT_OK, CBCT_EINVAL, CBCT_ENOMEM, CBCT_ECUDA, CBCT_EBREAKDOWN, CBCT_ETIMEOUT, CBCT_EBUDGET, CBCT_ENOTFOUND = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EBREAKDOWN", 5: "ETIMEOUT",
                6: "EBUDGET", 7: "ENOTFOUND"}
F32, F16, BF16 = 0, 1, 2
LAMBDA_FIXED, LAMBDA_GCV, LAMBDA_DP = 0, 1, 2


class CbctError(RuntimeError):
    def __init__(self, func, status, message):
        super().__init__("%s failed: %s (%s)" % (func, STATUS_NAMES.get(status, status), message))
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int),
        ("du", ctypes.c_double), ("dv", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double),
        ("nangles", ctypes.c_int), ("angles_rad", ctypes.POINTER(ctypes.c_double)),
    ]


class _Opts(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("lam", ctypes.c_double), ("rule", ctypes.c_int),
                ("storage", ctypes.c_int), ("use_graph", ctypes.c_int), ("profile", ctypes.c_int),
                ("noise_level", ctypes.c_double), ("explicit_residual", ctypes.c_int),
                ("stop_tol", ctypes.c_double), ("gmres_backprojector", ctypes.c_int),
                ("tv_outer", ctypes.c_int), ("tv_tau", ctypes.c_double), ("reorth", ctypes.c_int)]


class _Report(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int),
                ("resid_norm", ctypes.POINTER(ctypes.c_double)),
                ("normal_resid_norm", ctypes.POINTER(ctypes.c_double)),
                ("lambda_k", ctypes.POINTER(ctypes.c_double)),
                ("kernel_launches", ctypes.c_int64),
                ("forward_launches", ctypes.c_int64),
                ("backward_launches", ctypes.c_int64),
                ("forward_ms", ctypes.c_double),
                ("backward_ms", ctypes.c_double),
                ("explicit_resid_norm", ctypes.POINTER(ctypes.c_double)),
                ("explicit_count", ctypes.c_int),
                ("stopped_on_residual", ctypes.c_int)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("schedule", ctypes.c_int)]


class _Times(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("graph_replays", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t),
                ("active", ctypes.c_int), ("pending", ctypes.c_int)]


_lib = None


def declared_functions() -> list:
    """Names of the functions include/cbct.h declares."""
    text = open(HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cbct_[a-z0-9_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load libcbct.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libcbct.so is not built (%s); run paper_2211_14212_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    G = ctypes.c_void_p
    lib.cbct_geometry_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_void_p)]
    lib.cbct_geometry_destroy.argtypes = [G]
    lib.cbct_geometry_destroy.restype = None
    lib.cbct_geometry_num_voxels.argtypes = [G]
    lib.cbct_geometry_num_voxels.restype = i64
    lib.cbct_geometry_num_rays.argtypes = [G]
    lib.cbct_geometry_num_rays.restype = i64
    lib.cbct_geometry_device.argtypes = [G]
    lib.cbct_geometry_device.restype = ctypes.c_int
    for fn in ("cbct_project", "cbct_backproject", "cbct_project_static"):
        getattr(lib, fn).argtypes = [G, vp, vp, ctypes.c_int, vp]
    lib.cbct_count_nnz.argtypes = [G, ctypes.POINTER(i64), vp]
    lib.cbct_backproject_voxel_driven.argtypes = [G, vp, vp, vp]
    lib.cbct_geometry_set_launch.argtypes = [G, ctypes.c_int, ctypes.c_int]
    lib.cbct_geometry_get_launch.argtypes = [G, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.cbct_geometry_autotune.argtypes = [G, ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
    lib.cbct_geometry_set_angle_block.argtypes = [G, ctypes.c_int]
    lib.cbct_geometry_get_angle_block.argtypes = [G, ctypes.POINTER(ctypes.c_int)]
    for fn in ("cbct_cgls_solve", "cbct_lsqr_solve", "cbct_lsmr_solve", "cbct_hybrid_lsqr_solve",
               "cbct_hybrid_lsmr_solve", "cbct_ab_gmres_solve", "cbct_ba_gmres_solve", "cbct_cgls_tv_solve"):
        getattr(lib, fn).argtypes = [G, vp, vp, ctypes.POINTER(_Opts), ctypes.POINTER(_Report), vp]
    lib.cbct_server_create.argtypes = [ctypes.POINTER(_ServerOpts), ctypes.POINTER(ctypes.c_void_p)]
    lib.cbct_server_submit.argtypes = [vp, ctypes.POINTER(_Desc), vp, ctypes.c_int, ctypes.POINTER(_Opts),
                                       ctypes.POINTER(ctypes.c_uint64)]
    lib.cbct_server_request_bytes.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_size_t)]
    lib.cbct_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
    lib.cbct_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, vp, ctypes.POINTER(_Report),
                                     ctypes.POINTER(_Times)]
    lib.cbct_server_get_stats.argtypes = [vp, ctypes.POINTER(_ServerStats)]
    lib.cbct_server_destroy.argtypes = [vp]
    lib.cbct_server_destroy.restype = None
    lib.cbct_last_error.restype = ctypes.c_char_p
    lib.cbct_last_error.argtypes = []
    _lib = lib
    return lib


def _check(func, status):
    if status != CBCT_OK:
        raise CbctError(func, status, load().cbct_last_error().decode(errors="replace"))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t):
    import torch
    codes = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}
    if t not in codes:
        raise TypeError("unsupported dtype %s" % t)
    return codes[t]


STORAGE = {"f32": F32, "f16": F16, "bf16": BF16, F32: F32, F16: F16, BF16: BF16}


def _desc_of(spec):
    """A cbct_geometry_desc for any object carrying the scan parameters; returns
    (desc, angles array that must outlive it)."""
    angles = np.ascontiguousarray(np.asarray(spec.angles, dtype=np.float64))
    d = _Desc(int(spec.nx), int(spec.ny), int(spec.nz), float(spec.dx), float(spec.dy), float(spec.dz),
              int(spec.nu), int(spec.nv), float(spec.du), float(spec.dv), float(spec.dso), float(spec.dsd),
              int(angles.shape[0]), angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return d, angles


class Geometry:
    """Device-side scan geometry (cbct_geometry_create / _destroy).

    Accepts the scan parameters as keywords or any object carrying them as
    attributes (nx, ny, nz, dx, dy, dz, nu, nv, du, dv, dso, dsd, angles).
    """

    FIELDS = ("nx", "ny", "nz", "dx", "dy", "dz", "nu", "nv", "du", "dv", "dso", "dsd")

    def __init__(self, spec=None, **kw):
        if spec is not None:
            kw = {f: getattr(spec, f) for f in self.FIELDS + ("angles",)}
        self.params = kw
        self.angles = np.ascontiguousarray(np.asarray(kw["angles"], dtype=np.float64))
        lib = load()
        d = _Desc(int(kw["nx"]), int(kw["ny"]), int(kw["nz"]), float(kw["dx"]), float(kw["dy"]), float(kw["dz"]),
                  int(kw["nu"]), int(kw["nv"]), float(kw["du"]), float(kw["dv"]), float(kw["dso"]), float(kw["dsd"]),
                  int(self.angles.shape[0]), self.angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        h = ctypes.c_void_p()
        _check("cbct_geometry_create", lib.cbct_geometry_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.num_voxels = int(lib.cbct_geometry_num_voxels(h))
        self.num_rays = int(lib.cbct_geometry_num_rays(h))
        self.device = int(lib.cbct_geometry_device(h))
        self.vol_shape = (int(kw["nz"]), int(kw["ny"]), int(kw["nx"]))
        self.proj_shape = (int(self.angles.shape[0]), int(kw["nv"]), int(kw["nu"]))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().cbct_geometry_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _require_cuda(t, name, numel, device=None):
    """A contiguous CUDA tensor of `numel` elements, on CUDA device `device`
    (the geometry's) when given."""
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if device is not None and t.device.index != device:
        raise ValueError("%s is on cuda:%s but the geometry lives on cuda:%d" % (name, t.device.index, device))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))


def project(geom: Geometry, x, out=None, stream=None):
    """y = A x on the GPU (cbct_project); x and y share one dtype (f32/f16/bf16)."""
    import torch
    _require_cuda(x, "x", geom.num_voxels, geom.device)
    if out is None:
        out = torch.empty(geom.proj_shape, dtype=x.dtype, device=x.device)
    _require_cuda(out, "out", geom.num_rays, geom.device)
    if out.dtype != x.dtype:
        raise TypeError("x and out must share a dtype")
    _check("cbct_project", load().cbct_project(geom.handle, ctypes.c_void_p(x.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), _dtype_code(x.dtype),
                                               _stream_handle(stream)))
    return out


def backproject_voxel_driven(geom: Geometry, y, out=None, stream=None):
    """The voxel-driven interpolating approximation of A^T (not its transpose),
    FP32 (cbct_backproject_voxel_driven)."""
    import torch
    _require_cuda(y, "y", geom.num_rays, geom.device)
    if y.dtype != torch.float32:
        raise TypeError("y must be float32")
    if out is None:
        out = torch.empty(geom.vol_shape, dtype=torch.float32, device=y.device)
    _require_cuda(out, "out", geom.num_voxels, geom.device)
    _check("cbct_backproject_voxel_driven",
           load().cbct_backproject_voxel_driven(geom.handle, ctypes.c_void_p(y.data_ptr()),
                                                ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def project_static(geom: Geometry, x, out=None, stream=None):
    """y = A x like project(), through cbct_project_static, which allocates no
    device memory (padded volume copy of at most 66 MiB, e.g. 256^3 FP32;
    calls must not overlap on the GPU)."""
    import torch
    _require_cuda(x, "x", geom.num_voxels, geom.device)
    if out is None:
        out = torch.empty(geom.proj_shape, dtype=x.dtype, device=x.device)
    _require_cuda(out, "out", geom.num_rays, geom.device)
    if out.dtype != x.dtype:
        raise TypeError("x and out must share a dtype")
    _check("cbct_project_static", load().cbct_project_static(geom.handle, ctypes.c_void_p(x.data_ptr()),
                                                             ctypes.c_void_p(out.data_ptr()), _dtype_code(x.dtype),
                                                             _stream_handle(stream)))
    return out


def backproject(geom: Geometry, y, out=None, stream=None):
    """x = A^T y on the GPU (cbct_backproject), the exact transpose of project()."""
    import torch
    _require_cuda(y, "y", geom.num_rays, geom.device)
    if out is None:
        out = torch.empty(geom.vol_shape, dtype=y.dtype, device=y.device)
    _require_cuda(out, "out", geom.num_voxels, geom.device)
    if out.dtype != y.dtype:
        raise TypeError("y and out must share a dtype")
    _check("cbct_backproject", load().cbct_backproject(geom.handle, ctypes.c_void_p(y.data_ptr()),
                                                       ctypes.c_void_p(out.data_ptr()), _dtype_code(y.dtype),
                                                       _stream_handle(stream)))
    return out


def count_nnz(geom: Geometry, stream=None) -> int:
    n = ctypes.c_int64()
    _check("cbct_count_nnz", load().cbct_count_nnz(geom.handle, ctypes.byref(n), _stream_handle(stream)))
    return int(n.value)


TUNE_TIMES = 13
FWD_ROWS = (1, 2, 4)
BWD_CONFIGS = ("4x2 columns x 32", "4x2 columns x 64", "8x1 columns x 32", "2x4 columns x 64",
               "4x2 columns x 128", "2x4 columns x 128", "4x2 columns x 256", "2x4 columns x 256",
               "2x4 columns x 128, rows held", "4x2 columns x 128, rows held")


def set_launch(geom: Geometry, fwd_rows: int, bwd_config: int):
    """Set the projector launch shapes of a geometry (cbct_geometry_set_launch)."""
    _check("cbct_geometry_set_launch", load().cbct_geometry_set_launch(geom.handle, int(fwd_rows), int(bwd_config)))


def get_launch(geom: Geometry):
    """(fwd_rows, bwd_config) of a geometry."""
    f, b = ctypes.c_int(), ctypes.c_int()
    _check("cbct_geometry_get_launch", load().cbct_geometry_get_launch(geom.handle, ctypes.byref(f), ctypes.byref(b)))
    return int(f.value), int(b.value)


def set_angle_block(geom: Geometry, angles: int):
    """Angles per pass of the transpose (cbct_geometry_set_angle_block; 0 = default)."""
    _check("cbct_geometry_set_angle_block", load().cbct_geometry_set_angle_block(geom.handle, int(angles)))


def get_angle_block(geom: Geometry) -> int:
    a = ctypes.c_int()
    _check("cbct_geometry_get_angle_block", load().cbct_geometry_get_angle_block(geom.handle, ctypes.byref(a)))
    return int(a.value)


TUNE_CACHE_VERSION = 1


def tune_key(params: dict, nangles: int, device: str) -> str:
    """The geometry class a launch-shape choice is cached under: volume and
    detector sizes and spacings, source distances, angle count, the device's
    name and the library's shape tables (a cache written for other shapes
    does not match)."""
    p = params
    return "|".join((
        "vol %dx%dx%d @ %.6g,%.6g,%.6g" % (int(p["nx"]), int(p["ny"]), int(p["nz"]),
                                           float(p["dx"]), float(p["dy"]), float(p["dz"])),
        "det %dx%d @ %.6g,%.6g" % (int(p["nu"]), int(p["nv"]), float(p["du"]), float(p["dv"])),
        "dso %.6g dsd %.6g" % (float(p["dso"]), float(p["dsd"])),
        "angles %d" % int(nangles),
        device,
        "rows %s" % ",".join(str(r) for r in FWD_ROWS),
        "tiles %s" % ";".join(BWD_CONFIGS)))


class TuneCache:
    """Launch shapes chosen by `autotune`, per geometry class, in a JSON file
    {"version": 1, "entries": {key: {"fwd_rows", "bwd_config", ...}}}.  A
    missing, unreadable or other-version file reads as empty; `put` merges
    with what is on disk and replaces the file atomically."""

    def __init__(self, path):
        self.path = os.fspath(path)

    def _read(self) -> dict:
        import json
        try:
            with open(self.path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            return {}
        if not isinstance(data, dict) or data.get("version") != TUNE_CACHE_VERSION:
            return {}
        entries = data.get("entries")
        return entries if isinstance(entries, dict) else {}

    def get(self, key: str):
        e = self._read().get(key)
        if not isinstance(e, dict):
            return None
        f, b = e.get("fwd_rows"), e.get("bwd_config")
        if f not in FWD_ROWS or not isinstance(b, int) or not 0 <= b < len(BWD_CONFIGS):
            return None
        return e

    def put(self, key: str, entry: dict):
        import json
        import tempfile
        entries = self._read()
        entries[key] = entry
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".tune-", suffix=".json", dir=d)
        try:
            with os.fdopen(fd, "w") as f:
                json.dump({"version": TUNE_CACHE_VERSION, "entries": entries}, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def _device_name() -> str:
    import torch
    if torch.cuda.is_available():
        return torch.cuda.get_device_name(torch.cuda.current_device())
    return "no device"


def autotune(geom: Geometry, max_angles: int = 32, stream=None, cache=None) -> dict:
    """Time every launch shape on <= max_angles angles and keep the fastest
    (cbct_geometry_autotune).  Returns the chosen shapes and all timings.

    With `cache` (a JSON file path; default: the CBCT_TUNE_CACHE environment
    variable, if set) a geometry class tuned before takes its cached shapes
    without timing (`"cached": True`), and a new choice is added to the file."""
    cache = cache if cache is not None else os.environ.get("CBCT_TUNE_CACHE")
    key = store = None
    if cache:
        store = TuneCache(cache)
        key = tune_key(geom.params, len(geom.angles), _device_name())
        e = store.get(key)
        if e is not None:
            set_launch(geom, e["fwd_rows"], e["bwd_config"])
            return dict(e, bwd_shape=BWD_CONFIGS[e["bwd_config"]], cached=True)
    t = (ctypes.c_double * TUNE_TIMES)()
    _check("cbct_geometry_autotune", load().cbct_geometry_autotune(geom.handle, int(max_angles), t,
                                                                     _stream_handle(stream)))
    f, b = get_launch(geom)
    out = {"fwd_rows": f, "bwd_config": b, "bwd_shape": BWD_CONFIGS[b],
           "forward_ms": {str(r): t[i] for i, r in enumerate(FWD_ROWS)},
           "backward_ms": {BWD_CONFIGS[c]: t[len(FWD_ROWS) + c] for c in range(len(BWD_CONFIGS))}}
    if store is not None:
        store.put(key, dict(out, max_angles=int(max_angles)))
    return dict(out, cached=False)


@dataclass
class SolveReport:
    iters_done: int
    resid: np.ndarray
    normal_resid: np.ndarray
    lam: np.ndarray = field(default=None)
    kernel_launches: int = 0
    forward_launches: int = 0
    backward_launches: int = 0
    forward_ms: float = 0.0
    backward_ms: float = 0.0
    explicit_resid: np.ndarray = field(default=None)
    stopped_on_residual: bool = False


def _solve(fn, geom, b, iters, lam=0.0, storage="f32", rule="gcv", use_graph=True, x=None, stream=None,
           profile=False, noise_level=0.0, explicit_residual=False, stop_tol=0.0, backprojector="transpose",
           tv_outer=1, tv_tau=1e-3, reorth=False):
    """Run one of the C-ABI solvers.  b/x may be CUDA tensors or host (numpy or
    CPU torch, FP32) buffers; host buffers are staged by the library."""
    import torch
    lib = load()
    on_device = isinstance(b, torch.Tensor) and b.is_cuda
    if on_device:
        _require_cuda(b, "b", geom.num_rays, geom.device)
        if b.dtype != torch.float32:
            raise TypeError("b must be float32")
        if x is None:
            x = torch.empty(geom.vol_shape, dtype=torch.float32, device=b.device)
        _require_cuda(x, "x", geom.num_voxels, geom.device)
        bptr, xptr = b.data_ptr(), x.data_ptr()
    else:
        bh = b.numpy() if isinstance(b, torch.Tensor) else np.asarray(b)
        if bh.dtype != np.float32 or not bh.flags.c_contiguous or bh.size != geom.num_rays:
            raise TypeError("host b must be a contiguous float32 array of %d elements" % geom.num_rays)
        if x is None:
            x = np.empty(geom.vol_shape, dtype=np.float32)
        xh = x.numpy() if isinstance(x, torch.Tensor) else x
        if xh.dtype != np.float32 or not xh.flags.c_contiguous or xh.size != geom.num_voxels:
            raise TypeError("host x must be a contiguous float32 array of %d elements" % geom.num_voxels)
        bptr, xptr = bh.ctypes.data, xh.ctypes.data
    rule_code = ({"fixed": LAMBDA_FIXED, "gcv": LAMBDA_GCV, "dp": LAMBDA_DP}[rule] if isinstance(rule, str)
                 else int(rule))
    opts = _Opts(int(iters), float(lam), rule_code, STORAGE[storage], 1 if use_graph else 0, 1 if profile else 0,
                 float(noise_level), 1 if explicit_residual else 0, float(stop_tol),
                 {"transpose": 0, "sirt": 1, "voxel": 2}[backprojector], int(tv_outer), float(tv_tau),
                 1 if reorth else 0)
    hr = np.zeros(iters, dtype=np.float64)
    hn = np.zeros(iters, dtype=np.float64)
    hl = np.zeros(iters, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    he = np.zeros(iters, dtype=np.float64)
    rep = _Report(0, hr.ctypes.data_as(dp), hn.ctypes.data_as(dp), hl.ctypes.data_as(dp))
    rep.explicit_resid_norm = he.ctypes.data_as(dp)
    st = getattr(lib, fn)(geom.handle, ctypes.c_void_p(bptr), ctypes.c_void_p(xptr), ctypes.byref(opts),
                          ctypes.byref(rep), _stream_handle(stream))
    _check(fn, st)
    k = rep.iters_done
    return x, SolveReport(k, hr[:k].copy(), hn[:k].copy(), hl[:k].copy(), int(rep.kernel_launches),
                          int(rep.forward_launches), int(rep.backward_launches), float(rep.forward_ms),
                          float(rep.backward_ms), he[:rep.explicit_count].copy(), bool(rep.stopped_on_residual))


def cgls(geom, b, iters, lam=0.0, **kw):
    """CGLS (Sec. 2.1.1), optionally damped (Eq. 7)."""
    return _solve("cbct_cgls_solve", geom, b, iters, lam=lam, **kw)


def lsqr(geom, b, iters, lam=0.0, **kw):
    """LSQR (Sec. 2.1.2), optionally damped (Eq. 7)."""
    return _solve("cbct_lsqr_solve", geom, b, iters, lam=lam, **kw)


def lsmr(geom, b, iters, lam=0.0, **kw):
    """LSMR (Sec. 2.1.3), optionally damped (Eq. 7)."""
    return _solve("cbct_lsmr_solve", geom, b, iters, lam=lam, **kw)


def hybrid_lsqr(geom, b, iters, rule="gcv", lam=0.0, noise_level=0.0, **kw):
    """Hybrid LSQR (Sec. 2.2.1, Eq. 8) with lambda_k fixed, by GCV or by the
    discrepancy principle with relative noise level `noise_level` (Sec. 2.2.2)."""
    return _solve("cbct_hybrid_lsqr_solve", geom, b, iters, lam=lam, rule=rule, noise_level=noise_level, **kw)


def cgls_tv(geom, b, iters, lam, outer, tau=1e-3, **kw):
    """CGLS-TV (Sec. 2.3.1): `outer` reweighting steps sharing `iters` CGLS
    iterations on min ||A x - b||^2 + lam^2 ||W D x||^2."""
    return _solve("cbct_cgls_tv_solve", geom, b, iters, lam=lam, tv_outer=outer, tv_tau=tau, **kw)


def ab_gmres(geom, b, iters, backprojector="transpose", **kw):
    """AB-GMRES (Sec. 2.1.4); backprojector "transpose" (B = A^T), "sirt"
    (B = C A^T R with the SIRT weights) or "voxel" (voxel-driven, interpolating)."""
    return _solve("cbct_ab_gmres_solve", geom, b, iters, backprojector=backprojector, **kw)


def ba_gmres(geom, b, iters, backprojector="transpose", **kw):
    """BA-GMRES (Sec. 2.1.4); backprojector as for ab_gmres."""
    return _solve("cbct_ba_gmres_solve", geom, b, iters, backprojector=backprojector, **kw)


def hybrid_lsmr(geom, b, iters, rule="gcv", lam=0.0, **kw):
    """Hybrid LSMR: Tikhonov on LSMR's projected problem, lambda_k fixed or by
    GCV (the generalisation mentioned in Sec. 2.2.2)."""
    return _solve("cbct_hybrid_lsmr_solve", geom, b, iters, lam=lam, rule=rule, **kw)


# ------------------------------------------------------------------ serving
@dataclass
class ServedResult:
    x: np.ndarray
    report: SolveReport
    submit_s: float
    admit_s: float
    finish_s: float


def server_request_bytes(spec, solver="lsqr", iters=30) -> int:
    """Device memory a server request of this scan holds at its peak, the
    amount cbct_server_submit charges against the budget
    (cbct_server_request_bytes; host arithmetic, no device needed)."""
    d, _angles = _desc_of(spec)
    out = ctypes.c_size_t()
    _check("cbct_server_request_bytes", load().cbct_server_request_bytes(ctypes.byref(d), Server.SOLVERS[solver],
                                                                         int(iters), ctypes.byref(out)))
    return int(out.value)


class Server:
    """Continuous-batching server (cbct_server_*): requests of different scans
    are admitted by device-memory budget and advanced in steps of one Krylov
    iteration; schedule "fifo" (default) advances the oldest requests until a
    step fills the GPU, "srpt" the ones with the least remaining work,
    "ratio" orders them by response ratio (age + remaining) / remaining,
    "share" advances all of them."""

    SOLVERS = {"lsqr": 0, "lsmr": 1}
    SCHEDULES = {"srpt": 0, "share": 1, "ratio": 2, "fifo": 3}

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 16, use_graph: bool = True, schedule: str = "fifo"):
        lib = load()
        o = _ServerOpts(int(hbm_budget_bytes), int(max_slots), 1 if use_graph else 0, self.SCHEDULES[schedule])
        h = ctypes.c_void_p()
        _check("cbct_server_create", lib.cbct_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._shapes = {}

    def submit(self, spec, b, solver="lsqr", iters=30, lam=0.0) -> int:
        """Queue one reconstruction; b is copied (host FP32, N values)."""
        d, angles = _desc_of(spec)
        bh = np.ascontiguousarray(np.asarray(b, dtype=np.float32))
        n = int(d.nangles) * d.nv * d.nu
        if bh.size != n:
            raise ValueError("b has %d values, expected %d" % (bh.size, n))
        o = _Opts(int(iters), float(lam), 0, F32, 0, 0)
        rid = ctypes.c_uint64()
        _check("cbct_server_submit", load().cbct_server_submit(self._h, ctypes.byref(d), bh.ctypes.data,
                                                                 self.SOLVERS[solver], ctypes.byref(o),
                                                                 ctypes.byref(rid)))
        self._shapes[rid.value] = ((spec.nz, spec.ny, spec.nx), int(iters))
        return int(rid.value)

    def poll(self, rid: int) -> bool:
        done = ctypes.c_int()
        _check("cbct_server_poll", load().cbct_server_poll(self._h, rid, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, rid: int, timeout: float = -1.0) -> ServedResult:
        """Block until the request is done (CbctError with status ETIMEOUT on time-out)."""
        shape, iters = self._shapes[rid]
        x = np.empty(shape, dtype=np.float32)
        hr = np.zeros(iters)
        hn = np.zeros(iters)
        dp = ctypes.POINTER(ctypes.c_double)
        rep = _Report(0, hr.ctypes.data_as(dp), hn.ctypes.data_as(dp), None)
        t = _Times()
        _check("cbct_server_wait", load().cbct_server_wait(self._h, rid, float(timeout), x.ctypes.data,
                                                             ctypes.byref(rep), ctypes.byref(t)))
        del self._shapes[rid]
        k = rep.iters_done
        return ServedResult(x, SolveReport(k, hr[:k].copy(), hn[:k].copy()), t.submit_s, t.admit_s, t.finish_s)

    def stats(self) -> dict:
        st = _ServerStats()
        _check("cbct_server_get_stats", load().cbct_server_get_stats(self._h, ctypes.byref(st)))
        return {"steps": st.steps, "graph_replays": st.graph_replays, "bytes_in_use": st.bytes_in_use,
                "active": st.active, "pending": st.pending}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().cbct_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
