"""Full-size solver anchor: LSQR and LSMR on the 256^3 medical scan (256^3 x
1 mm volume, 512^2 x 0.8 mm detector, 360 angles, DSO 1000 / DSD 1536) in the
launch configuration the benchmark uses (autotuned shapes, graph replay),
against the FP64 oracle's iterates after k = 1, 2, 3 (Sec. 2.1.2 LSQR,
Sec. 2.1.3 LSMR).

The oracle's iterates were computed once, offline, by
tests/golden/make_golden_c2_solvers.py (oracle and synth only) and stored at
2000+ sampled voxels together with the norms of the whole iterates and the
residual estimates.  Bars: 1e-4 relative on the sampled voxels (2-norm), on
||x_k|| and on the residual estimates, at every k.
"""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_solver_anchor.json")
TOL = 1e-4


@pytest.fixture(scope="module")
def cbct():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_14212_gb300 import cbct as mod
    return mod


@pytest.fixture(scope="module")
def anchor():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def problem(cbct, anchor):
    import torch
    g = synth.config(anchor["geometry"])
    b = synth.random_projections(g, anchor["b"]["seed"]).astype(np.float32)
    geom = cbct.Geometry(g)
    cbct.autotune(geom, max_angles=32)           # the benchmark's launch shapes
    return g, geom, torch.from_numpy(b).cuda()


@pytest.mark.parametrize("method", ["lsqr", "lsmr"])
def test_full_size_iterates(cbct, anchor, problem, method):
    import torch
    g, geom, b = problem
    ref = anchor[method]
    vox = torch.from_numpy(np.asarray(anchor["voxels"], dtype=np.int64)).cuda()
    lines = []
    for k in range(1, anchor["iters"] + 1):
        x, rep = getattr(cbct, method)(geom, b, k)
        assert rep.iters_done == k
        got = x.view(-1)[vox].double().cpu().numpy()
        want = np.asarray(ref["iterates"][k - 1])
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        nrm = float(torch.linalg.vector_norm(x.double()))
        nerr = abs(nrm - ref["norms"][k - 1]) / ref["norms"][k - 1]
        rerr = abs(rep.resid[-1] - ref["resid"][k - 1]) / ref["resid"][k - 1]
        nrerr = abs(rep.normal_resid[-1] - ref["normal_resid"][k - 1]) / ref["normal_resid"][k - 1]
        lines.append("k=%d sampled %.2e  norm %.2e  resid %.2e  normal resid %.2e" % (k, err, nerr, rerr, nrerr))
        assert err <= TOL and nerr <= TOL and rerr <= TOL and nrerr <= TOL, "\n".join(lines)
        del x
    print("%s at 256^3:\n  %s" % (method, "\n  ".join(lines)))
