"""Writes precision_reference.json: FP64 oracle values that the storage-
precision study (FP32 / FP16 / BF16 storage of volumes and projections, FP32
ray sums, FP64 Krylov scalars) measures its error against.

* "c3": the 512^3 scan (512^3 x 0.5 mm, 768 x 512 x 0.8 mm detector, 720
  angles, DSO 1000 / DSD 1536): (A x)_r of the seeded ellipsoid phantom at
  2000 sampled rays and (A^T y)_j of a seeded uniform projection stack
  (rounded to FP32) at 200 sampled voxels (Sec. 1, Eq. 1).
* "medium": the 64^3 reduction of the 256^3 medical scan (64^3 x 4 mm,
  128^2 x 3.2 mm, 90 angles) with a seeded uniform b (rounded to FP32): the
  FP64 iterates of LSQR, LSMR and hybrid LSQR with GCV after 20 iterations
  (Sec. 2.1.2, 2.1.3, 2.2.1-2.2.2) at 4000 sampled voxels, and the norms of
  the whole iterates.

Written from the oracle alone (oracle/ and synth/):

    python tests/golden/make_golden_precision.py
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

OUT = os.path.join(HERE, "precision_reference.json")


def medium_geometry():
    return synth.Geometry(64, 64, 64, 4.0, 4.0, 4.0, 128, 128, 3.2, 3.2, 1000.0, 1536.0,
                          synth.circular_angles(90))


def c3_fixtures():
    g = synth.config("c3")
    x = synth.ellipsoid_phantom(g, 10, seed=2, scale=0.02).astype(np.float64)
    rays = np.sort(np.random.default_rng(71).choice(g.num_rays, size=2000, replace=False))
    y = synth.random_projections(g, 72).astype(np.float32).astype(np.float64)
    vox = np.sort(np.random.default_rng(73).choice(g.num_voxels, size=200, replace=False))
    return {"phantom_seed": 2, "y_seed": 72,
            "rays": rays.tolist(), "project_rays": oracle.project_rays(g, x, rays).tolist(),
            "voxels": vox.tolist(), "backproject_voxels": oracle.backproject_voxels(g, y, vox).tolist()}


def medium_fixtures(iters=20):
    g = medium_geometry()
    b = synth.random_projections(g, 74).astype(np.float32).astype(np.float64).ravel()
    vox = np.sort(np.random.default_rng(75).choice(g.num_voxels, size=4000, replace=False))
    op = oracle.Operator(g)
    out = {"b_seed": 74, "iters": iters, "voxels": vox.tolist()}
    for name, fn in (("lsqr", lambda: krylov.lsqr(op, b, iters)),
                     ("lsmr", lambda: krylov.lsmr(op, b, iters)),
                     ("hybrid_lsqr", lambda: krylov.hybrid_lsqr(op, b, iters, rule="gcv"))):
        x, _ = fn()
        out[name] = {"sampled": x[vox].tolist(), "norm": float(np.linalg.norm(x))}
    return out


if __name__ == "__main__":
    oracle.build()
    data = {"c3": c3_fixtures(), "medium": medium_fixtures()}
    with open(OUT, "w") as f:
        json.dump(data, f)
    print("wrote", OUT)
