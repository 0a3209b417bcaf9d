"""Writes oracle_regression.json: regression values of the FP64 oracle.

The paper prints no worked example with numerical values (its results are
figures of reconstructions and residual histories), so there is no printed
number to pin against.  These fixtures are written by this script from the
oracle alone (oracle/ and the synthetic inputs of synth/, nothing else) and
pin the oracle against unintended change; its correctness is pinned by the
closed-form, brute-force and definition tests in tests/test_oracle_*.py.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import krylov  # noqa: E402

THREADS = 4


def fixtures():
    out = {}
    g = synth.config("tiny")
    x = synth.ellipsoid_phantom(g, 4, seed=3).astype(np.float64)
    rays = np.random.default_rng(7).choice(g.num_rays, size=16, replace=False)
    y = synth.random_projections(g, 8)
    vox = np.random.default_rng(9).choice(g.num_voxels, size=16, replace=False)
    out["tiny"] = {
        "rays": rays.tolist(),
        "project_rays": oracle.project_rays(g, x, rays, THREADS).tolist(),
        "voxels": vox.tolist(),
        "backproject_voxels": oracle.backproject_voxels(g, y, vox, THREADS).tolist(),
        "nnz": int(oracle.nnz(g)),
        "voxel_driven_voxels": krylov.VoxelDrivenBackprojector(g)(y)[vox].tolist(),
    }
    g = synth.config("c1")
    xt = synth.ellipsoid_phantom(g, 10, seed=0).astype(np.float64)
    b = oracle.project(g, xt, THREADS).ravel()
    op = oracle.Operator(g)
    res = {}
    for m in ("cgls", "lsqr", "lsmr"):
        _, h = getattr(krylov, m)(op, b, 6)
        res[m] = {"resid": h["resid"], "normal_resid": h["normal_resid"]}
    bn = synth.poisson_log_noise(b, 1e3, seed=5).astype(np.float64)
    _, h = krylov.hybrid_lsqr(op, bn, 6, rule="gcv")
    res["hybrid_gcv_lambda"] = h["lambda"]
    nl = 1.5 * float(np.linalg.norm(bn - b) / np.linalg.norm(bn))
    _, h = krylov.hybrid_lsqr(op, bn, 6, rule="dp", noise_level=nl)
    res["hybrid_dp_lambda"] = h["lambda"]
    res["dp_noise_level"] = nl
    _, h = krylov.hybrid_lsmr(op, bn, 6, rule="gcv")
    res["hybrid_lsmr_gcv_lambda"] = h["lambda"]
    _, h = krylov.lsqr(op, bn, 6, reorth=True)
    res["lsqr_reorth_resid"] = h["resid"]
    bps = {"transpose": None, "sirt": krylov.WeightedBackprojector(op), "voxel": krylov.VoxelDrivenBackprojector(g)}
    for name, bp in bps.items():
        for variant in ("ab", "ba"):
            _, h = getattr(krylov, variant + "_gmres")(op, b, 5, backprojector=bp)
            res["%s_gmres_%s_resid" % (variant, name)] = h["resid"]
    _, h = krylov.cgls_tv(op, g.vol_shape, bn, 2, 3, 2.0, 1e-2)
    res["cgls_tv_resid"] = h["resid"]
    out["c1"] = res
    return out


if __name__ == "__main__":
    oracle.build()
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(fixtures(), f, indent=1)
    print("wrote", os.path.join(HERE, "oracle_regression.json"))
