"""Seeded synthetic inputs for cone-beam CT reconstruction.

This module is shared by the FP64 oracle (``oracle/``) and the GPU library
(``paper_2211_14212_gb300``).  It holds *inputs only*: scan geometries (plain
numbers), voxelised ellipsoid phantoms, random test vectors and the photon-count
noise model.  It contains none of the reconstruction arithmetic (no ray
tracing, no projector, no solver), so sharing it does not couple the two
implementations.

The paper reconstructs a synthetic head phantom, an Alderson head scan and a
micro-CT bumblebee scan (Sec. 3).  None of them is available, so the generators
below produce seeded random-ellipsoid phantoms with the sizes and magnification
of those workloads instead.  The noise model follows Sec. 3.1.1: Poisson photon
counts with air count I0 applied to exp(-b), then log-transformed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Geometry",
    "circular_angles",
    "config",
    "CONFIG_NAMES",
    "ellipsoid_phantom",
    "random_volume",
    "random_projections",
    "poisson_log_noise",
]


def circular_angles(nangles: int, arc_deg: float = 360.0) -> np.ndarray:
    """Equally spaced source angles a*arc/nangles, a = 0..nangles-1 (end point excluded)."""
    return np.arange(nangles, dtype=np.float64) * (math.radians(arc_deg) / nangles)


@dataclass
class Geometry:
    """Circular cone-beam scan description (all lengths in mm, angles in rad).

    Conventions (the paper leaves geometry to its toolbox; these are the ones
    used throughout this repository):

    * rotation axis = z; origin = rotation centre = volume centre;
    * source at (dso cos t, dso sin t, 0); detector centre at
      -(dsd - dso) (cos t, sin t, 0); detector axes e_u = (-sin t, cos t, 0),
      e_v = (0, 0, 1);
    * pixel (iu, iv) centre = detector centre + (iu-(nu-1)/2) du e_u
      + (iv-(nv-1)/2) dv e_v; one ray per pixel, source -> pixel centre;
    * voxel (i, j, k) is the half-open box [x0+i dx, x0+(i+1) dx) x ... with
      x0 = -nx dx / 2; volume stored x[k][j][i]; projections y[a][iv][iu].
    """

    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    nu: int
    nv: int
    du: float
    dv: float
    dso: float
    dsd: float
    angles: np.ndarray = field(repr=False)

    def __post_init__(self):
        self.angles = np.ascontiguousarray(np.asarray(self.angles, dtype=np.float64))

    @property
    def nangles(self) -> int:
        return int(self.angles.shape[0])

    @property
    def vol_shape(self) -> tuple:
        return (self.nz, self.ny, self.nx)

    @property
    def proj_shape(self) -> tuple:
        return (self.nangles, self.nv, self.nu)

    @property
    def num_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def num_rays(self) -> int:
        return self.nangles * self.nv * self.nu

    def with_angles(self, angles) -> "Geometry":
        """Same scanner and volume, another list of source angles."""
        return Geometry(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz,
                        self.nu, self.nv, self.du, self.dv, self.dso, self.dsd,
                        np.asarray(angles, dtype=np.float64))

    def angle_subset(self, count: int) -> "Geometry":
        """`count` angles taken with a fixed stride from this geometry's list."""
        stride = max(1, self.nangles // count)
        return self.with_angles(self.angles[::stride][:count])

    def describe(self) -> dict:
        return {
            "volume": [self.nx, self.ny, self.nz],
            "voxel_mm": [self.dx, self.dy, self.dz],
            "detector": [self.nu, self.nv],
            "pixel_mm": [self.du, self.dv],
            "angles": self.nangles,
            "dso_mm": self.dso,
            "dsd_mm": self.dsd,
        }


def _cube(n, voxel, nu, nv, pix, nangles, dso, dsd, arc=360.0, nvox_z=None, pix_v=None):
    nz = n if nvox_z is None else nvox_z
    return Geometry(n, n, nz, voxel, voxel, voxel, nu, nv, pix,
                    pix if pix_v is None else pix_v, dso, dsd,
                    circular_angles(nangles, arc))


# Workload shapes.  "tiny"/"small" are test cases; c1..c5 are the five
# benchmark configurations (medical CBCT at 32^3..512^3 and a high-magnification
# micro-CT at 1024^3).  Sizes the paper does not state (voxel and pixel pitch,
# distances of the smaller cases) are chosen so the detector covers the volume.
def config(name: str) -> Geometry:
    if name == "tiny":        # 8^3, 16x16 detector, 20 angles: dense A is 5120 x 512
        return _cube(8, 1.0, 16, 16, 1.2, 20, 100.0, 150.0)
    if name == "small":       # several CTA tiles and ragged edges
        return Geometry(40, 36, 28, 1.0, 1.1, 0.9, 77, 45, 1.3, 1.1, 300.0, 480.0,
                        circular_angles(23))
    if name == "c1":          # 32^3 x 1 mm, 64^2 x 1.2 mm, 60 angles / 360, DSO 1000, DSD 1500
        return _cube(32, 1.0, 64, 64, 1.2, 60, 1000.0, 1500.0)
    if name == "c2":          # 256^3 x 1 mm, 512^2 x 0.8 mm, 360 angles, DSO 1000, DSD 1536
        return _cube(256, 1.0, 512, 512, 0.8, 360, 1000.0, 1536.0)
    if name == "c3":          # 512^3 x 0.5 mm, 768 x 512 x 0.8 mm, 720 angles
        return Geometry(512, 512, 512, 0.5, 0.5, 0.5, 768, 512, 0.8, 0.8, 1000.0, 1536.0,
                        circular_angles(720))
    if name == "c5":          # micro-CT: 1024^3 x 0.1 mm, 1536^2 x 0.6 mm, 1600 angles, DSO 200, DSD 1200
        return _cube(1024, 0.1, 1536, 1536, 0.6, 1600, 200.0, 1200.0)
    raise KeyError(name)


CONFIG_NAMES = ("tiny", "small", "c1", "c2", "c3", "c5")


def serving_request_geometry(n: int, nu: int, nangles: int, short_scan: bool) -> Geometry:
    """One request of the serving stream: n^3 voxels over a 256 mm field of view,
    nu x nu detector of 409.6 mm width, `nangles` over 360 deg or a 200 deg short scan."""
    arc = 200.0 if short_scan else 360.0
    return Geometry(n, n, n, 256.0 / n, 256.0 / n, 256.0 / n, nu, nu, 409.6 / nu, 409.6 / nu,
                    1000.0, 1536.0, circular_angles(nangles, arc))


def _voxel_centres(g: Geometry, axis: int, xp=np):
    n, d = [(g.nx, g.dx), (g.ny, g.dy), (g.nz, g.dz)][axis]
    return (xp.arange(n, dtype=xp.float64) + 0.5) * d - n * d / 2.0


def ellipsoid_phantom(g: Geometry, n_ellipsoids: int = 10, seed: int = 0, scale: float = 1.0,
                      cylinder: bool = False, dtype=np.float32) -> np.ndarray:
    """Seeded random-ellipsoid phantom sampled at voxel centres.

    Ellipsoid e has centre uniform in +-0.35 x extent, semi-axes uniform in
    [0.05, 0.35] x extent, rotation about z uniform in [0, pi) and density
    uniform in [0, 1]; later ellipsoids overwrite earlier ones, so values stay in
    [0, 1] before `scale` (e.g. 0.02 mm^-1 for water-like attenuation).  With
    `cylinder` a coaxial cylinder of density 0.3 (radius 0.45 x extent, height
    0.8 x extent) is drawn first, as a sample holder in micro-CT.
    Returns an array of shape (nz, ny, nx).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ext = np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz])
    cz, cy, cx = _voxel_centres(g, 2), _voxel_centres(g, 1), _voxel_centres(g, 0)
    vol = np.zeros(g.vol_shape, dtype=np.float64)
    if cylinder:
        r = 0.45 * min(ext[0], ext[1])
        inside = ((cx[None, None, :] ** 2 + cy[None, :, None] ** 2 <= r * r)
                  & (np.abs(cz)[:, None, None] <= 0.4 * ext[2]))
        vol[np.broadcast_to(inside, vol.shape)] = 0.3
    for _ in range(n_ellipsoids):
        c = rng.uniform(-0.35, 0.35, 3) * ext
        a = rng.uniform(0.05, 0.35, 3) * ext
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        cp, sp = math.cos(phi), math.sin(phi)
        # only voxel centres inside the ellipsoid's bounding sphere can be inside it
        rmax = float(a.max())
        sl = []
        for centres, cc in ((cz, c[2]), (cy, c[1]), (cx, c[0])):
            idx = np.nonzero(np.abs(centres - cc) <= rmax)[0]
            sl.append(slice(idx[0], idx[-1] + 1) if idx.size else slice(0, 0))
        oz = (cz[sl[0]] - c[2])[:, None, None]
        oy = (cy[sl[1]] - c[1])[None, :, None]
        ox = (cx[sl[2]] - c[0])[None, None, :]
        # rotate voxel-centre offsets into the ellipsoid frame (rotation about z)
        ex = (cp * ox + sp * oy) / a[0]
        ey = (-sp * ox + cp * oy) / a[1]
        ez = oz / a[2]
        inside = ex * ex + ey * ey + ez * ez <= 1.0
        sub = vol[sl[0], sl[1], sl[2]]
        sub[np.broadcast_to(inside, sub.shape)] = rho
    return (vol * scale).astype(dtype)


def random_volume(g: Geometry, seed: int, dtype=np.float64) -> np.ndarray:
    """Uniform [0, 1) volume of shape (nz, ny, nx) (for adjoint and parity tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random(g.vol_shape).astype(dtype)


def random_projections(g: Geometry, seed: int, dtype=np.float64) -> np.ndarray:
    """Uniform [0, 1) projection stack of shape (nangles, nv, nu)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random(g.proj_shape).astype(dtype)


def poisson_log_noise(b_clean: np.ndarray, i0: float, seed: int, dtype=np.float32) -> np.ndarray:
    """Photon-count noise: c ~ Poisson(i0 exp(-b)), b_noisy = -ln(max(c, 1) / i0).

    Clamping at one count keeps the logarithm finite (the paper does not say how
    it treats zero counts).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = i0 * np.exp(-np.asarray(b_clean, dtype=np.float64))
    counts = rng.poisson(lam).astype(np.float64)
    return (-np.log(np.maximum(counts, 1.0) / i0)).astype(dtype)
