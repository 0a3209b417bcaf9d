"""Writes c2_solver_anchor.json: the FP64 oracle's LSQR and LSMR iterates on
the full 256^3 medical scan (256^3 x 1 mm, 512^2 x 0.8 mm detector, 360
angles, DSO 1000 / DSD 1536), sampled at fixed voxels.

The GPU solvers are compared with the oracle element by element only on
reduced copies of this scan (the oracle needs about 8 minutes per product
here); this anchor checks the full-size solver, in the launch configuration
the benchmark uses, at the sampled voxels after k = 1, 2, 3 iterations
(Sec. 2.1.2 LSQR, Sec. 2.1.3 LSMR).

Input: b = a seeded uniform [0, 1) projection stack (synth.random_projections),
rounded to FP32 so that the GPU and the oracle read the same numbers.
LSQR and LSMR run the same Golub-Kahan process on the same b; the operator
below remembers each product by the bytes of its input vector, so the two
solvers share their 7 products instead of computing 14.  Written from the
oracle alone (oracle/ and synth/):

    nice -n 19 python tests/golden/make_golden_c2_solvers.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import krylov  # noqa: E402

B_SEED = 61
VOXEL_SEED = 62
SAMPLES = 2000
ITERS = 3
OUT = os.path.join(HERE, "c2_solver_anchor.json")


class RememberingOperator:
    """oracle.Operator whose products are kept, keyed by the input's bytes."""

    def __init__(self, g):
        self.op = oracle.Operator(g)
        self.shape = self.op.shape
        self.memo = {}
        self.computed = 0

    def _get(self, kind, v, fn):
        v = np.ascontiguousarray(v, dtype=np.float64)
        key = (kind, hashlib.sha256(v.tobytes()).hexdigest())
        if key not in self.memo:
            t0 = time.time()
            self.memo[key] = fn(v)
            self.computed += 1
            print("  %s product %d: %.0f s" % (kind, self.computed, time.time() - t0), flush=True)
        return self.memo[key].copy()

    def matvec(self, x):
        return self._get("A", x, self.op.matvec)

    def rmatvec(self, y):
        return self._get("AT", y, self.op.rmatvec)


def sample_voxels(g):
    """SAMPLES seeded voxels plus the 8 corners and the centres of the 6 faces
    (ABI flat index (k * ny + j) * nx + i)."""
    rng = np.random.default_rng(VOXEL_SEED)
    vox = set(rng.choice(g.num_voxels, size=SAMPLES, replace=False).tolist())
    last = (g.nx - 1, g.ny - 1, g.nz - 1)
    for k in (0, last[2]):
        for j in (0, last[1]):
            for i in (0, last[0]):
                vox.add((k * g.ny + j) * g.nx + i)
    c = (g.nx // 2, g.ny // 2, g.nz // 2)
    for axis in range(3):
        for end in (0, last[axis]):
            p = list(c)
            p[axis] = end
            vox.add((p[2] * g.ny + p[1]) * g.nx + p[0])
    return np.array(sorted(vox), dtype=np.int64)


def main():
    oracle.build()
    g = synth.config("c2")
    b = synth.random_projections(g, B_SEED).astype(np.float32).astype(np.float64).ravel()
    vox = sample_voxels(g)
    op = RememberingOperator(g)
    out = {"geometry": "c2", "b": {"generator": "synth.random_projections", "seed": B_SEED,
                                   "rounded_to": "float32"},
           "iters": ITERS, "voxels": vox.tolist()}
    for method in ("lsqr", "lsmr"):
        t0 = time.time()
        _, h = getattr(krylov, method)(op, b, ITERS, keep_iterates=True)
        out[method] = {
            "iterates": [xk[vox].tolist() for xk in h["iterates"]],
            "norms": [float(np.linalg.norm(xk)) for xk in h["iterates"]],
            "resid": h["resid"], "normal_resid": h["normal_resid"]}
        print("%s: %.0f s, %d products computed so far" % (method, time.time() - t0, op.computed), flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
