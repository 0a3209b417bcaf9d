"""Pins of the oracle's A^T (Sec. 2: every Krylov step needs an exact transpose).

The explicit scatter, the voxel-by-voxel clipping route and the dense matrix
transpose are three independent computations of A^T y; the dot-product test
<A x, y> = <x, A^T y> fixes A^T against the separately pinned A.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("name", ["tiny", "small", "c1"])
def test_dot_product_identity(name):
    g = synth.config(name)
    x = synth.random_volume(g, 11)
    y = synth.random_projections(g, 12) - 0.5
    ax = oracle.project(g, x)
    aty = oracle.backproject(g, y)
    lhs = float(np.dot(ax.ravel(), y.ravel()))
    rhs = float(np.dot(x.ravel(), aty.ravel()))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(ax) * np.linalg.norm(y)


def test_scatter_equals_dense_transpose():
    g = synth.config("tiny")
    a = oracle.dense_matrix(g)
    y = synth.random_projections(g, 13)
    np.testing.assert_allclose(oracle.backproject(g, y).ravel(), a.T @ y.ravel(), rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("name", ["small", "c1"])
def test_voxel_by_voxel_route_equals_scatter(name):
    """(A^T y)_j from ray/box clipping over the voxel's footprint = the ray-driven scatter."""
    g = synth.config(name)
    y = synth.random_projections(g, 14)
    full = oracle.backproject(g, y).ravel()
    rng = np.random.default_rng(5)
    vox = rng.choice(g.num_voxels, size=300, replace=False)
    part = oracle.backproject_voxels(g, y, vox)
    np.testing.assert_allclose(part, full[vox], rtol=1e-11, atol=1e-11)


def test_project_rays_subset_equals_full():
    g = synth.config("small")
    x = synth.random_volume(g, 15)
    full = oracle.project(g, x).ravel()
    rays = np.array([0, 5, g.num_rays // 3, g.num_rays - 1], dtype=np.int64)
    np.testing.assert_array_equal(oracle.project_rays(g, x, rays), full[rays])
