"""Pins of the oracle's system matrix A against closed forms and brute force.

A[i][j] is the length of ray i inside voxel j (Sec. 1, Eq. 1).  Each check
below fixes a different part of the oracle: the total chord (no length lost or
double counted), whole-voxel cuboids (index <-> position map and storage
order), brute-force quadrature (every entry), a lone voxel seen from known
directions (rotation sense, detector axes, magnification), the half-open voxel
rule, and convergence to the analytic chord of an ellipsoid.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def ray_points(g, ray):
    """Source and pixel centre of a flat ray index, from the geometry convention."""
    per = g.nu * g.nv
    a, rem = divmod(int(ray), per)
    iv, iu = divmod(rem, g.nu)
    t = g.angles[a]
    u = (iu - (g.nu - 1) / 2) * g.du
    v = (iv - (g.nv - 1) / 2) * g.dv
    src = np.array([g.dso * math.cos(t), g.dso * math.sin(t), 0.0])
    det_c = -(g.dsd - g.dso) * np.array([math.cos(t), math.sin(t), 0.0])
    e_u = np.array([-math.sin(t), math.cos(t), 0.0])
    e_v = np.array([0.0, 0.0, 1.0])
    return src, det_c + u * e_u + v * e_v


def chord_through_box(src, pix, lo, hi):
    """Length of the segment src->pix inside the box [lo, hi] (slab clipping)."""
    d = pix - src
    t0, t1 = 0.0, 1.0
    for c in range(3):
        if d[c] == 0.0:
            if not (lo[c] <= src[c] <= hi[c]):
                return 0.0
            continue
        a, b = (lo[c] - src[c]) / d[c], (hi[c] - src[c]) / d[c]
        t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
    return max(0.0, t1 - t0) * float(np.linalg.norm(d))


def volume_box(g):
    half = np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz]) / 2
    return -half, half


def sample_rays(g, count, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(g.num_rays, size=min(count, g.num_rays), replace=False)


@pytest.mark.parametrize("name", ["tiny", "small", "c1"])
def test_sum_rule_equals_chord(name):
    """Sum of a ray's segment lengths = its chord through the whole volume box."""
    g = synth.config(name)
    lo, hi = volume_box(g)
    for r in sample_rays(g, 400, 1):
        _, ln = oracle.ray_segments(g, r)
        s, p = ray_points(g, r)
        assert abs(ln.sum() - chord_through_box(s, p, lo, hi)) <= 1e-11 * max(1.0, ln.sum())


@pytest.mark.parametrize("name,box", [("small", (3, 29, 5, 17, 2, 11)), ("c1", (1, 9, 20, 31, 4, 30))])
def test_cuboid_of_whole_voxels(name, box):
    """A x for x = 1 on an off-centre block of voxels = chord through that block."""
    g = synth.config(name)
    i0, i1, j0, j1, k0, k1 = box
    x = np.zeros(g.vol_shape)
    x[k0:k1, j0:j1, i0:i1] = 1.0
    y = oracle.project(g, x).reshape(-1)
    vlo, _ = volume_box(g)
    lo = vlo + np.array([i0 * g.dx, j0 * g.dy, k0 * g.dz])
    hi = vlo + np.array([i1 * g.dx, j1 * g.dy, k1 * g.dz])
    for r in sample_rays(g, 600, 2):
        s, p = ray_points(g, r)
        assert abs(y[r] - chord_through_box(s, p, lo, hi)) <= 1e-10


def test_brute_force_quadrature():
    """Every entry: midpoint quadrature of the piecewise-constant field along the ray."""
    g = synth.config("tiny")
    x = synth.random_volume(g, 7)
    y = oracle.project(g, x).reshape(-1)
    lo, hi = volume_box(g)
    nsamp = 400_000
    for r in sample_rays(g, 40, 3):
        s, p = ray_points(g, r)
        d = p - s
        length = float(np.linalg.norm(d))
        t = (np.arange(nsamp) + 0.5) / nsamp
        pts = s[None, :] + t[:, None] * d[None, :]
        ijk = np.floor((pts - lo) / np.array([g.dx, g.dy, g.dz])).astype(np.int64)
        inside = np.all((ijk >= 0) & (ijk < np.array([g.nx, g.ny, g.nz])), axis=1)
        vals = np.zeros(nsamp)
        q = ijk[inside]
        vals[inside] = x[q[:, 2], q[:, 1], q[:, 0]]
        approx = vals.sum() * length / nsamp
        # each boundary crossing can misplace at most one quadrature step of weight <= max|x|
        bound = (g.nx + g.ny + g.nz + 3) * (length / nsamp) * 1.0
        assert abs(y[r] - approx) <= bound


def test_lone_voxel_seen_from_known_directions():
    """One bright voxel: its projection lands where perspective projection puts it."""
    g = synth.Geometry(24, 20, 16, 1.0, 1.0, 1.0, 64, 48, 0.75, 0.75, 200.0, 330.0,
                       np.radians([0.0, 30.0, 90.0, 145.0, 200.0, 290.0]))
    i, j, k = 17, 4, 11
    x = np.zeros(g.vol_shape)
    x[k, j, i] = 1.0
    y = oracle.project(g, x)
    centre = np.array([(i + 0.5) - g.nx / 2, (j + 0.5) - g.ny / 2, (k + 0.5) - g.nz / 2])
    for a, t in enumerate(g.angles):
        along = g.dso - (centre[0] * math.cos(t) + centre[1] * math.sin(t))
        across = -centre[0] * math.sin(t) + centre[1] * math.cos(t)
        u = across * g.dsd / along
        v = centre[2] * g.dsd / along
        iu = u / g.du + (g.nu - 1) / 2
        iv = v / g.dv + (g.nv - 1) / 2
        img = y[a]
        nz_iv, nz_iu = np.nonzero(img)
        assert img[int(round(iv)), int(round(iu))] > 0.5     # ray through the centre: chord ~1 mm
        # the footprint is compact around the projected centre
        mag = g.dsd / along
        assert np.all(np.abs(nz_iu - iu) <= mag * 1.8 / g.du + 1)
        assert np.all(np.abs(nz_iv - iv) <= mag * 1.8 / g.dv + 1)


def test_half_open_voxels_ray_in_a_plane():
    """A ray lying in the plane z = 0 (a voxel face) belongs to the voxel above it."""
    g = synth.Geometry(10, 10, 6, 1.0, 1.0, 1.0, 21, 5, 1.0, 1.0, 100.0, 160.0,
                       np.radians([0.0, 37.0]))
    # nv = 5 -> the central detector row has v = 0, so its rays stay in z = 0
    for a in range(g.nangles):
        for iu in range(g.nu):
            r = (a * g.nv + 2) * g.nu + iu
            idx, ln = oracle.ray_segments(g, r)
            if len(idx):
                k = idx // (g.nx * g.ny)
                assert np.all(k == g.nz // 2)
                assert abs(ln.sum() - chord_through_box(*ray_points(g, r), *volume_box(g))) < 1e-11


def test_single_ellipsoid_converges_to_analytic_chord():
    """Voxelised unit-density ellipsoid -> analytic ray/quadric chord at first order in h."""
    centre = np.array([6.0, -9.0, 4.0])
    axes = np.array([30.0, 22.0, 26.0])
    fov = 96.0
    errs = []
    for n in (16, 32, 64):
        h = fov / n
        g = synth.Geometry(n, n, n, h, h, h, 48, 48, 4.0, 4.0, 400.0, 600.0, np.radians([0.0, 50.0, 120.0]))
        zc = (np.arange(n) + 0.5) * h - fov / 2
        z, yy, xx = np.meshgrid(zc, zc, zc, indexing="ij")
        inside = (((xx - centre[0]) / axes[0]) ** 2 + ((yy - centre[1]) / axes[1]) ** 2
                  + ((z - centre[2]) / axes[2]) ** 2) <= 1.0
        y = oracle.project(g, inside.astype(np.float64)).reshape(-1)
        exact = np.empty_like(y)
        for r in range(g.num_rays):
            s, p = ray_points(g, r)
            d = p - s
            # |(s + t d - c)/axes|^2 = 1  ->  A t^2 + B t + C = 0
            ds, dd = (s - centre) / axes, d / axes
            qa, qb, qc = dd @ dd, 2 * ds @ dd, ds @ ds - 1.0
            disc = qb * qb - 4 * qa * qc
            exact[r] = 0.0 if disc <= 0 else math.sqrt(disc) / qa * float(np.linalg.norm(d))
        errs.append(np.abs(y - exact).mean())
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 1.5 and errs[1] / errs[2] > 1.5


def test_nnz_matches_dense_count():
    g = synth.config("tiny")
    a = oracle.dense_matrix(g)
    count = oracle.nnz(g)
    # count includes rounding-level slivers where a ray grazes a voxel edge
    assert abs(count - int((a > 0).sum())) <= 1e-3 * count
    assert int((a > 1e-9).sum()) <= count
