"""Continuous-batching server (cbct_server_*): every result is the same alone
and in a mix of other scans (within FP32 rounding), equals the single-request
solver's and the FP64 oracle's iterate, and admission follows the device
memory budget."""
import time

import numpy as np
import pytest

import oracle
import synth
from oracle import krylov

pytestmark = pytest.mark.gpu

MIX_TOL = 1e-5          # alone vs in a mix: only the transpose's accumulation order differs
ITER_TOL = 1e-4         # vs the FP64 oracle at a k where FP32 meets it (k = 10 here)


@pytest.fixture(scope="module")
def cbct():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_14212_gb300 import cbct as mod
    return mod


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(g, seed, noisy):
    x = synth.ellipsoid_phantom(g, 8, seed=seed, scale=0.02 if noisy else 1.0)
    b = oracle.project(g, x.astype(np.float64))
    if noisy:
        b = synth.poisson_log_noise(b, 1e5, seed=seed + 100)
    return b.astype(np.float64).ravel()


@pytest.fixture(scope="module")
def scans():
    ga = synth.config("c1")
    gb = synth.config("small")
    gc = synth.Geometry(48, 48, 40, 5.0, 5.0, 5.0, 96, 80, 4.0, 4.0, 1000.0, 1536.0, synth.circular_angles(64, 200.0))
    return [(ga, problem(ga, 1, False), "lsqr", 0.0),
            (gb, problem(gb, 2, False), "lsmr", 0.0),
            (gc, problem(gc, 3, True), "lsmr", 0.01)]


def test_alone_equals_mix_equals_solver(cbct, scans):
    iters = 10
    alone = []
    for g, b, solver, lam_frac in scans:
        lam = lam_frac * float(np.linalg.norm(b))
        with cbct.Server(8 << 30, max_slots=8) as srv:
            rid = srv.submit(g, b, solver, iters, lam)
            alone.append(srv.wait(rid, timeout=300).x)
    with cbct.Server(8 << 30, max_slots=8) as srv:
        ids = [srv.submit(g, b, solver, iters, lam_frac * float(np.linalg.norm(b)))
               for g, b, solver, lam_frac in scans]
        mixed = [srv.wait(i, timeout=300) for i in ids]
        st = srv.stats()
    assert st["graph_replays"] > 0
    for (g, b, solver, lam_frac), xa, res in zip(scans, alone, mixed):
        lam = lam_frac * float(np.linalg.norm(b))
        assert res.report.iters_done == iters
        assert rel(res.x, xa) <= MIX_TOL
        geom = cbct.Geometry(g)
        xs, _ = getattr(cbct, solver)(geom, b.astype(np.float32), iters, lam=lam)
        assert rel(res.x, xs) <= MIX_TOL
        x_ref, _ = getattr(krylov, solver)(oracle.Operator(g), b, iters, damp=lam)
        assert rel(res.x, x_ref) <= ITER_TOL
        assert res.submit_s <= res.admit_s <= res.finish_s


def test_budget_admission_one_at_a_time(cbct, scans):
    """A budget that fits one request and not two (slots to spare): the others
    wait and are admitted once its memory is back, after its result."""
    g, b, solver, _ = scans[2]
    need = cbct.server_request_bytes(g, solver, 6)
    with cbct.Server(need + need // 2, max_slots=4) as srv:
        ids = [srv.submit(g, b, solver, 6) for _ in range(3)]
        res = [srv.wait(i, timeout=300) for i in ids]
    for r0, r1 in zip(res, res[1:]):
        assert r1.admit_s >= r0.finish_s
    for r in res[1:]:
        assert rel(r.x, res[0].x) <= MIX_TOL


def test_over_budget_request_rejected(cbct, scans):
    g, b, _, _ = scans[0]
    with cbct.Server(1 << 20, max_slots=4) as srv:
        with pytest.raises(cbct.CbctError) as e:
            srv.submit(g, b, "lsqr", 5)
        assert e.value.status == cbct.CBCT_EBUDGET


def test_wait_timeout_keeps_request(cbct, scans):
    g, b, _, _ = scans[2]
    with cbct.Server(4 << 30, max_slots=2) as srv:
        rid = srv.submit(g, b, "lsqr", 40)
        with pytest.raises(cbct.CbctError) as e:
            srv.wait(rid, timeout=0.0)
        assert e.value.status == cbct.CBCT_ETIMEOUT
        res = srv.wait(rid, timeout=300)
        assert res.report.iters_done == 40
        with pytest.raises(cbct.CbctError):
            srv.poll(rid)                 # forgotten after a successful wait


def test_many_requests_continuous(cbct):
    """Requests submitted while others run are admitted between steps; all finish."""
    rng = np.random.default_rng(9)
    with cbct.Server(2 << 30, max_slots=4) as srv:
        ids, shapes = [], []
        for i in range(10):
            n = int(rng.choice([16, 24, 32]))
            g = synth.Geometry(n, n, n, 64.0 / n, 64.0 / n, 64.0 / n, 48, 40, 2.0, 2.0, 400.0, 640.0,
                               synth.circular_angles(int(rng.integers(12, 40))))
            b = np.abs(rng.standard_normal(g.num_rays)).astype(np.float32)
            ids.append(srv.submit(g, b, ["lsqr", "lsmr"][i % 2], int(rng.integers(3, 12))))
            shapes.append(g.vol_shape)
        res = [srv.wait(i, timeout=300) for i in ids]
        # a result is returned once on the host; its memory is freed right after
        deadline = time.monotonic() + 10.0
        st = srv.stats()
        while st["bytes_in_use"] and time.monotonic() < deadline:
            time.sleep(0.01)
            st = srv.stats()
    assert all(np.isfinite(r.x).all() and r.x.shape == s for r, s in zip(res, shapes))
    assert st["bytes_in_use"] == 0 and st["active"] == 0 and st["pending"] == 0


@pytest.mark.parametrize("schedule", ["fifo", "srpt", "ratio", "share"])
def test_schedule(cbct, schedule):
    """A large request (more forward tiles than one step needs to fill the GPU)
    and a short one submitted right after it: FIFO runs the large one to the
    end first and SRPT the short one, each alone, so the steps add up; SHARE
    advances both in the same steps."""
    big = synth.Geometry(128, 128, 128, 2.0, 2.0, 2.0, 256, 256, 1.6, 1.6, 1000.0, 1536.0,
                         synth.circular_angles(180))
    small = synth.config("c1")
    rng = np.random.default_rng(4)
    b_big = np.abs(rng.standard_normal(big.num_rays)).astype(np.float32)
    b_small = np.abs(rng.standard_normal(small.num_rays)).astype(np.float32)
    with cbct.Server(8 << 30, max_slots=4, schedule=schedule) as srv:
        i_big = srv.submit(big, b_big, "lsqr", 30)
        i_small = srv.submit(small, b_small, "lsqr", 4)
        r_big, r_small = srv.wait(i_big, timeout=300), srv.wait(i_small, timeout=300)
        st = srv.stats()
    assert r_big.report.iters_done == 30 and r_small.report.iters_done == 4
    if schedule == "srpt":
        assert st["steps"] == 34
        assert r_small.finish_s <= r_big.finish_s
    elif schedule == "fifo":
        assert st["steps"] == 34
        assert r_small.finish_s >= r_big.finish_s
    elif schedule == "share":
        assert st["steps"] < 34
    else:                       # the young short request has the higher response ratio
        assert r_small.finish_s <= r_big.finish_s
    alone, _ = cbct.lsqr(cbct.Geometry(small), b_small, 4)
    assert rel(r_small.x, alone) <= MIX_TOL


def test_srpt_does_not_starve_a_long_request(cbct):
    """SRPT with a sustained stream of short requests behind a long one: the
    long request (more forward tiles than a step takes) is passed over while
    shorter work is available, but after 64 consecutive steps without it it
    goes first, so it finishes well before the stream ends."""
    big = synth.Geometry(128, 128, 128, 2.0, 2.0, 2.0, 256, 256, 1.6, 1.6, 1000.0, 1536.0,
                         synth.circular_angles(180))
    small = synth.config("c1")
    rng = np.random.default_rng(6)
    b_big = np.abs(rng.standard_normal(big.num_rays)).astype(np.float32)
    b_small = np.abs(rng.standard_normal(small.num_rays)).astype(np.float32)
    with cbct.Server(16 << 30, max_slots=16, schedule="srpt") as srv:
        i_big = srv.submit(big, b_big, "lsqr", 30)
        ids = [srv.submit(small, b_small, "lsqr", 10) for _ in range(100)]
        r_big = srv.wait(i_big, timeout=600)
        smalls = [srv.wait(i, timeout=600) for i in ids]
    assert r_big.report.iters_done == 30
    last_small = max(r.finish_s for r in smalls)
    assert r_big.finish_s < last_small
    # and the short ones did go first while it waited
    assert sum(r.finish_s < r_big.finish_s for r in smalls) >= 10
