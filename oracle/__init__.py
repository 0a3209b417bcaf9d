"""FP64 CPU oracle for Krylov cone-beam CT reconstruction.

TEST INFRASTRUCTURE.  Only the tests, the smoke check of ``__graft_entry__``
and the CPU-baseline leg of ``bench.py`` import this package.  The GPU library
never does, and this package imports nothing from it: the two share no code.

* ``oracle/siddon.c``  -- the system matrix A (Sec. 1, Eq. 1) by definition:
  ray/voxel intersection lengths of source -> pixel-centre segments, merged-alpha
  form, FP64; A x with OpenMP over rays; A^T y as an explicit sequential
  scatter, and voxel by voxel from ray/box clipping.
* ``oracle/krylov.py`` -- textbook CGLS, LSQR, LSMR (with Tikhonov damping),
  hybrid LSQR with GCV, in FP64 numpy (Sec. 2.1-2.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int),
        ("du", ctypes.c_double), ("dv", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double),
        ("nangles", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile oracle/siddon.c into oracle/liboracle.so (gcc, OpenMP, IEEE FP64)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    G = ctypes.POINTER(_Geom)
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_num_rays.argtypes = [G]
    lib.oracle_num_rays.restype = ctypes.c_int64
    lib.oracle_max_segments.argtypes = [G]
    lib.oracle_max_segments.restype = ctypes.c_int64
    lib.oracle_ray_segments.argtypes = [G, ctypes.c_int64, lp, dp, ctypes.c_int]
    lib.oracle_ray_segments.restype = ctypes.c_int
    lib.oracle_project_rays.argtypes = [G, dp, lp, ctypes.c_int64, dp, ctypes.c_int]
    lib.oracle_project_rays.restype = None
    lib.oracle_project.argtypes = [G, dp, dp, ctypes.c_int]
    lib.oracle_project.restype = None
    lib.oracle_backproject.argtypes = [G, dp, dp, ctypes.c_int]
    lib.oracle_backproject.restype = None
    lib.oracle_nnz.argtypes = [G, ctypes.c_int]
    lib.oracle_nnz.restype = ctypes.c_int64
    lib.oracle_backproject_voxels.argtypes = [G, dp, lp, ctypes.c_int64, dp, ctypes.c_int]
    lib.oracle_backproject_voxels.restype = None
    _lib = lib
    return lib


def _geom(g):
    angles = np.ascontiguousarray(g.angles, dtype=np.float64)
    s = _Geom(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.nu, g.nv, g.du, g.dv, g.dso, g.dsd,
              int(angles.shape[0]), angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return s, angles          # keep `angles` alive alongside the struct


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def project(g, x, nthreads: int = 0) -> np.ndarray:
    """y = A x, y of shape (nangles, nv, nu)."""
    lib = _load()
    s, keep = _geom(g)
    x = _f64(x).reshape(-1)
    assert x.size == g.num_voxels
    y = np.empty(g.proj_shape, dtype=np.float64)
    lib.oracle_project(ctypes.byref(s), _dptr(x), _dptr(y), int(nthreads))
    return y


def project_rays(g, x, rays, nthreads: int = 0) -> np.ndarray:
    """(A x)_r for the flat ray indices r = (a*nv + iv)*nu + iu in `rays`."""
    lib = _load()
    s, keep = _geom(g)
    x = _f64(x).reshape(-1)
    rays = np.ascontiguousarray(np.asarray(rays, dtype=np.int64))
    out = np.empty(rays.shape[0], dtype=np.float64)
    lib.oracle_project_rays(ctypes.byref(s), _dptr(x), _lptr(rays), int(rays.shape[0]),
                            _dptr(out), int(nthreads))
    return out


def backproject(g, y, nthreads: int = 1) -> np.ndarray:
    """x = A^T y (explicit scatter; sequential, or over `nthreads` ray chunks), shape (nz, ny, nx)."""
    lib = _load()
    s, keep = _geom(g)
    y = _f64(y).reshape(-1)
    assert y.size == g.num_rays
    x = np.empty(g.vol_shape, dtype=np.float64)
    lib.oracle_backproject(ctypes.byref(s), _dptr(y), _dptr(x), int(nthreads))
    return x


def backproject_voxels(g, y, voxels, nthreads: int = 0) -> np.ndarray:
    """(A^T y)_j for the flat voxel indices j = (k*ny + j)*nx + i in `voxels`."""
    lib = _load()
    s, keep = _geom(g)
    y = _f64(y).reshape(-1)
    vox = np.ascontiguousarray(np.asarray(voxels, dtype=np.int64))
    out = np.empty(vox.shape[0], dtype=np.float64)
    lib.oracle_backproject_voxels(ctypes.byref(s), _dptr(y), _lptr(vox), int(vox.shape[0]),
                                  _dptr(out), int(nthreads))
    return out


def nnz(g, nthreads: int = 0) -> int:
    """Number of positive-length ray/voxel pairs, i.e. nonzeros of A."""
    lib = _load()
    s, keep = _geom(g)
    return int(lib.oracle_nnz(ctypes.byref(s), int(nthreads)))


def ray_segments(g, ray: int):
    """(voxel indices, lengths) of one ray, in order from the source."""
    lib = _load()
    s, keep = _geom(g)
    cap = int(lib.oracle_max_segments(ctypes.byref(s)))
    idx = np.empty(cap, dtype=np.int64)
    ln = np.empty(cap, dtype=np.float64)
    c = lib.oracle_ray_segments(ctypes.byref(s), int(ray), _lptr(idx), _dptr(ln), cap)
    if c < 0:
        raise RuntimeError("segment buffer too small")
    return idx[:c].copy(), ln[:c].copy()


def dense_matrix(g) -> np.ndarray:
    """A as a dense (N, M) FP64 array (tiny geometries only)."""
    n, m = g.num_rays, g.num_voxels
    if n * m > 5e7:
        raise ValueError("geometry too large for a dense matrix")
    a = np.zeros((n, m), dtype=np.float64)
    for r in range(n):
        idx, ln = ray_segments(g, r)
        a[r, idx] += ln
    return a


class Operator:
    """A and A^T of a geometry as flat-vector callables (what the solvers take)."""

    def __init__(self, g, nthreads: int = 0):
        self.g = g
        self.nthreads = nthreads
        self.shape = (g.num_rays, g.num_voxels)

    def matvec(self, x):
        return project(self.g, x, self.nthreads).reshape(-1)

    def rmatvec(self, y):
        return backproject(self.g, y, self.nthreads or (os.cpu_count() or 1)).reshape(-1)


class DenseOperator:
    """A dense matrix exposed with the same interface as `Operator`."""

    def __init__(self, a):
        self.a = np.asarray(a, dtype=np.float64)
        self.shape = self.a.shape

    def matvec(self, x):
        return self.a @ np.asarray(x, dtype=np.float64).reshape(-1)

    def rmatvec(self, y):
        return self.a.T @ np.asarray(y, dtype=np.float64).reshape(-1)
