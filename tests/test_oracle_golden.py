"""The FP64 oracle against its stored regression values (tests/golden/, written
by tests/golden/make_golden.py from the oracle alone; the paper prints no
worked example with numbers).  Any change of the oracle's arithmetic shows up
here and must name the passage of the paper that justifies it."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import krylov

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")
RTOL = 1e-10          # FP64 sums whose grouping may depend on the thread count


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_tiny_projector_values(golden):
    t = golden["tiny"]
    g = synth.config("tiny")
    x = synth.ellipsoid_phantom(g, 4, seed=3).astype(np.float64)
    np.testing.assert_allclose(oracle.project_rays(g, x, np.array(t["rays"])), t["project_rays"], rtol=RTOL)
    y = synth.random_projections(g, 8)
    np.testing.assert_allclose(oracle.backproject_voxels(g, y, np.array(t["voxels"])), t["backproject_voxels"],
                               rtol=RTOL)
    assert oracle.nnz(g) == t["nnz"]


def test_c1_solver_histories(golden):
    c = golden["c1"]
    g = synth.config("c1")
    xt = synth.ellipsoid_phantom(g, 10, seed=0).astype(np.float64)
    b = oracle.project(g, xt).ravel()
    op = oracle.Operator(g)
    for m in ("cgls", "lsqr", "lsmr"):
        _, h = getattr(krylov, m)(op, b, 6)
        np.testing.assert_allclose(h["resid"], c[m]["resid"], rtol=RTOL)
        np.testing.assert_allclose(h["normal_resid"], c[m]["normal_resid"], rtol=RTOL)
    bn = synth.poisson_log_noise(b, 1e3, seed=5).astype(np.float64)
    _, h = krylov.hybrid_lsqr(op, bn, 6, rule="gcv")
    np.testing.assert_allclose(h["lambda"], c["hybrid_gcv_lambda"], rtol=1e-8)
    _, h = krylov.hybrid_lsqr(op, bn, 6, rule="dp", noise_level=c["dp_noise_level"])
    np.testing.assert_allclose(h["lambda"], c["hybrid_dp_lambda"], rtol=1e-8)


def test_voxel_driven_backprojector_values(golden):
    t = golden["tiny"]
    g = synth.config("tiny")
    y = synth.random_projections(g, 8)
    got = krylov.VoxelDrivenBackprojector(g)(y)[np.array(t["voxels"])]
    np.testing.assert_allclose(got, t["voxel_driven_voxels"], rtol=RTOL)


def test_c1_extended_solver_histories(golden):
    """Hybrid LSMR (GCV), re-orthogonalised LSQR, AB-/BA-GMRES with each
    backprojector and CGLS-TV on the c1 problem."""
    c = golden["c1"]
    g = synth.config("c1")
    xt = synth.ellipsoid_phantom(g, 10, seed=0).astype(np.float64)
    b = oracle.project(g, xt).ravel()
    bn = synth.poisson_log_noise(b, 1e3, seed=5).astype(np.float64)
    op = oracle.Operator(g)
    _, h = krylov.hybrid_lsmr(op, bn, 6, rule="gcv")
    np.testing.assert_allclose(h["lambda"], c["hybrid_lsmr_gcv_lambda"], rtol=1e-8)
    _, h = krylov.lsqr(op, bn, 6, reorth=True)
    np.testing.assert_allclose(h["resid"], c["lsqr_reorth_resid"], rtol=RTOL)
    bps = {"transpose": None, "sirt": krylov.WeightedBackprojector(op), "voxel": krylov.VoxelDrivenBackprojector(g)}
    for name, bp in bps.items():
        for variant in ("ab", "ba"):
            _, h = getattr(krylov, variant + "_gmres")(op, b, 5, backprojector=bp)
            np.testing.assert_allclose(h["resid"], c["%s_gmres_%s_resid" % (variant, name)], rtol=RTOL)
    _, h = krylov.cgls_tv(op, g.vol_shape, bn, 2, 3, 2.0, 1e-2)
    np.testing.assert_allclose(h["resid"], c["cgls_tv_resid"], rtol=RTOL)


def test_precision_reference_values():
    """The stored FP64 values of the storage-precision study (written by
    tests/golden/make_golden_precision.py from the oracle) are the oracle's:
    20 of the 512^3 scan's sampled rays and 5 of its sampled voxels recomputed."""
    with open(os.path.join(os.path.dirname(GOLDEN), "precision_reference.json")) as f:
        ref = json.load(f)["c3"]
    g = synth.config("c3")
    x = synth.ellipsoid_phantom(g, 10, seed=ref["phantom_seed"], scale=0.02).astype(np.float64)
    rays = np.asarray(ref["rays"][::100])
    np.testing.assert_allclose(oracle.project_rays(g, x, rays), ref["project_rays"][::100], rtol=RTOL)
    sub = np.asarray(ref["voxels"][::40])
    y = synth.random_projections(g, ref["y_seed"]).astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(oracle.backproject_voxels(g, y, sub), ref["backproject_voxels"][::40], rtol=RTOL)


def test_c2_anchor_first_iterate_is_along_the_backprojected_data():
    """The stored 256^3 anchor (tests/golden/make_golden_c2_solvers.py) against
    a property of its first iterates: LSQR's and LSMR's x_1 are multiples of
    A^T b (Sec. 2.1.2-2.1.3: x_1 lies in span{A^T b}).  A^T b is recomputed at
    60 of the stored voxels by the oracle's voxel-by-voxel route, independent
    of the scatter the stored run used."""
    path = os.path.join(os.path.dirname(GOLDEN), "c2_solver_anchor.json")
    with open(path) as f:
        anchor = json.load(f)
    g = synth.config(anchor["geometry"])
    b = synth.random_projections(g, anchor["b"]["seed"]).astype(np.float32).astype(np.float64)
    pick = np.arange(0, len(anchor["voxels"]), len(anchor["voxels"]) // 60)[:60]
    vox = np.asarray(anchor["voxels"])[pick]
    atb = oracle.backproject_voxels(g, b, vox)
    for method in ("lsqr", "lsmr"):
        x1 = np.asarray(anchor[method]["iterates"][0])[pick]
        ratio = x1 / atb
        np.testing.assert_allclose(ratio, ratio[0], rtol=1e-9)
        assert ratio[0] > 0
