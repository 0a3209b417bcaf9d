"""Pins of the oracle's Krylov solvers against definitions that do not use their recurrences.

* Each iterate is the minimiser over K_k(A^T A, A^T b) of the method's own
  criterion (Eqs. 3-5): compared with a dense Krylov basis + lstsq.
* CGLS and LSQR are mathematically equivalent (Sec. 2.1.2).
* LSQR/LSMR converge to the least-squares solution (Sec. 2.1.3); with damping
  lam, to the solution of the augmented system (Eq. 7).
* ||r_k|| is monotone for CGLS/LSQR and ||A^T r_k|| for LSMR.
* Hybrid LSQR with a fixed lam equals projecting the augmented system (Sec. 2.2.1).
* The GCV function equals its definition with an explicit H^+_lam (Sec. 2.2.2),
  and its minimiser agrees with a brute-force grid.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import krylov


@pytest.fixture(scope="module")
def tiny_system():
    g = synth.config("tiny")
    a = oracle.dense_matrix(g)
    x_true = synth.ellipsoid_phantom(g, 4, seed=3).astype(np.float64).ravel()
    rng = np.random.default_rng(4)
    b = a @ x_true + 0.05 * rng.standard_normal(a.shape[0])
    return a, b


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("method", ["cgls", "lsqr", "lsmr"])
@pytest.mark.parametrize("damp", [0.0, 1.5])
def test_iterates_minimise_over_krylov_space(tiny_system, method, damp):
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    solver = getattr(krylov, method)
    _, hist = solver(op, b, 8, damp=damp, keep_iterates=True)
    for k, xk in enumerate(hist["iterates"], start=1):
        ref = krylov.krylov_reference(a, b, k, method, damp)
        assert rel(xk, ref) < 1e-8, (method, damp, k)


def test_cgls_equals_lsqr(tiny_system):
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    _, hc = krylov.cgls(op, b, 12, keep_iterates=True)
    _, hl = krylov.lsqr(op, b, 12, keep_iterates=True)
    for xc, xl in zip(hc["iterates"], hl["iterates"]):
        assert rel(xc, xl) < 1e-9


def test_lsqr_lsmr_reach_least_squares_solution():
    rng = np.random.default_rng(8)
    a = rng.standard_normal((60, 20))
    b = rng.standard_normal(60)
    ref = np.linalg.lstsq(a, b, rcond=None)[0]
    op = oracle.DenseOperator(a)
    for solver in (krylov.lsqr, krylov.lsmr, krylov.cgls):
        x, _ = solver(op, b, 60)
        assert rel(x, ref) < 1e-10


@pytest.mark.parametrize("solver", [krylov.lsmr, krylov.lsqr, krylov.cgls])
def test_damped_limit_is_augmented_lstsq(tiny_system, solver):
    a, b = tiny_system
    lam = 2.0
    aug = np.vstack([a, lam * np.eye(a.shape[1])])
    rhs = np.concatenate([b, np.zeros(a.shape[1])])
    ref = np.linalg.lstsq(aug, rhs, rcond=None)[0]
    x, _ = solver(oracle.DenseOperator(a), b, 150, damp=lam)
    assert rel(x, ref) < 1e-8


def test_residual_histories_monotone_and_match_explicit(tiny_system):
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    for name in ("cgls", "lsqr"):
        _, h = getattr(krylov, name)(op, b, 25, keep_iterates=True)
        r = np.array(h["resid"])
        assert np.all(np.diff(r) <= 1e-12 * r[0])
        explicit = [np.linalg.norm(b - a @ x) for x in h["iterates"]]
        np.testing.assert_allclose(r, explicit, rtol=1e-9)
        explicit_n = [np.linalg.norm(a.T @ (b - a @ x)) for x in h["iterates"]]
        np.testing.assert_allclose(h["normal_resid"], explicit_n, rtol=1e-6)
    _, h = krylov.lsmr(op, b, 25, keep_iterates=True)
    nr = np.array(h["normal_resid"])
    assert np.all(np.diff(nr) <= 1e-12 * nr[0])
    explicit_n = [np.linalg.norm(a.T @ (b - a @ x)) for x in h["iterates"]]
    np.testing.assert_allclose(nr, explicit_n, rtol=1e-6)
    explicit = [np.linalg.norm(b - a @ x) for x in h["iterates"]]
    np.testing.assert_allclose(h["resid"], explicit, rtol=1e-9)


def test_damped_residual_estimates(tiny_system):
    a, b = tiny_system
    lam = 1.5
    op = oracle.DenseOperator(a)
    _, h = krylov.lsqr(op, b, 15, damp=lam, keep_iterates=True)
    aug = [math.sqrt(np.linalg.norm(b - a @ x) ** 2 + lam * lam * np.linalg.norm(x) ** 2) for x in h["iterates"]]
    np.testing.assert_allclose(h["resid"], aug, rtol=1e-9)
    _, h = krylov.lsmr(op, b, 15, damp=lam, keep_iterates=True)
    normal = [np.linalg.norm(a.T @ (b - a @ x) - lam * lam * x) for x in h["iterates"]]
    np.testing.assert_allclose(h["normal_resid"], normal, rtol=1e-6)


def test_hybrid_fixed_lambda_equals_damped_lsqr(tiny_system):
    a, b = tiny_system
    lam = 3.0
    op = oracle.DenseOperator(a)
    _, hh = krylov.hybrid_lsqr(op, b, 10, rule="fixed", lam=lam, keep_iterates=True)
    _, hl = krylov.lsqr(op, b, 10, damp=lam, keep_iterates=True)
    for k, (xh, xl) in enumerate(zip(hh["iterates"], hl["iterates"]), start=1):
        assert rel(xh, xl) < 1e-9
        assert rel(xh, krylov.krylov_reference(a, b, k, "lsqr", lam)) < 1e-8


def test_projected_tikhonov_matches_normal_equations():
    rng = np.random.default_rng(21)
    k = 7
    h = np.zeros((k + 1, k))
    for i in range(k):
        h[i, i] = rng.uniform(0.5, 2)
        h[i + 1, i] = rng.uniform(0.1, 1)
    beta1, lam = 3.7, 0.4
    y = krylov.projected_tikhonov(h, beta1, lam)
    e1 = np.zeros(k + 1)
    e1[0] = beta1
    ref = np.linalg.solve(h.T @ h + lam * lam * np.eye(k), h.T @ e1)
    np.testing.assert_allclose(y, ref, rtol=1e-12)


def test_gcv_function_equals_definition():
    rng = np.random.default_rng(22)
    k = 9
    h = np.zeros((k + 1, k))
    for i in range(k):
        h[i, i] = rng.uniform(0.01, 2)
        h[i + 1, i] = rng.uniform(0.01, 1)
    beta1 = 2.3
    p, sigma, _ = np.linalg.svd(h, full_matrices=True)
    e1 = np.zeros(k + 1)
    e1[0] = beta1
    for lam in (1e-3, 0.05, 0.7, 4.0):
        hdag = np.linalg.solve(h.T @ h + lam * lam * np.eye(k), h.T)
        m = np.eye(k + 1) - h @ hdag
        direct = np.linalg.norm(m @ e1) ** 2 / np.trace(m) ** 2
        assert abs(krylov.gcv_function(sigma, p[0], beta1, lam) - direct) <= 1e-12 * direct


def test_gcv_minimiser_matches_brute_force_grid(tiny_system):
    a, b = tiny_system
    _, h = krylov.lsqr(oracle.DenseOperator(a), b, 12)
    k = 12
    hk = np.zeros((k + 1, k))
    for i in range(k):
        hk[i, i] = h["alpha"][i]
        hk[i + 1, i] = h["beta"][i + 1]
    beta1 = h["beta"][0]
    p, sigma, _ = np.linalg.svd(hk, full_matrices=True)
    lam = krylov.gcv_lambda(sigma, p[0], beta1)
    grid = np.exp(np.linspace(math.log(sigma.max()) - 8 * math.log(10), math.log(sigma.max()), 10_000))
    vals = np.array([krylov.gcv_function(sigma, p[0], beta1, t) for t in grid])
    best = grid[np.argmin(vals)]
    step = grid[1] / grid[0]
    assert best / step <= lam <= best * step
    assert krylov.gcv_function(sigma, p[0], beta1, lam) <= vals.min() * (1 + 1e-9)


def test_hybrid_gcv_runs_and_lambda_positive(tiny_system):
    a, b = tiny_system
    x, h = krylov.hybrid_lsqr(oracle.DenseOperator(a), b, 10, rule="gcv")
    assert all(l > 0 for l in h["lambda"])
    # projected residual equals the explicit one (A V_k = U_{k+1} H_k)
    assert abs(h["resid"][-1] - np.linalg.norm(b - a @ x)) <= 1e-8 * np.linalg.norm(b)


# ------------------------------------------------- discrepancy principle (Sec. 2.2.2)
def test_dp_residual_meets_noise_level_explicitly(tiny_system):
    """Where the projected problem can reach it, the DP lam_k makes the explicit
    residual ||b - A x_k|| (dense product, not the projected formula) equal
    nl ||b||; before that (residual of the unregularised iterate still above
    the target) lam_k = 0 and x_k is the LSQR iterate."""
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    nb = np.linalg.norm(b)
    _, h_lsqr = krylov.lsqr(op, b, 12, keep_iterates=True)
    nl = 0.999 * h_lsqr["resid"][5] / nb            # reachable once r_k of LSQR drops below r_6
    _, h = krylov.hybrid_lsqr(op, b, 12, rule="dp", noise_level=nl, keep_iterates=True)
    reached = 0
    for k in range(1, 13):
        xk = h["iterates"][k - 1]
        explicit = np.linalg.norm(b - a @ xk)
        if h["lambda"][k - 1] == 0.0:
            assert rel(xk, h_lsqr["iterates"][k - 1]) <= 1e-8
            assert explicit >= nl * nb * (1 - 1e-9)
        else:
            reached += 1
            assert abs(explicit - nl * nb) <= 1e-8 * nb
    assert reached >= 3


def test_dp_lambda_grows_with_noise_level(tiny_system):
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    nb = np.linalg.norm(b)
    _, h_lsqr = krylov.lsqr(op, b, 10)
    lams = []
    for f in (0.1, 0.3, 0.6, 0.9):
        nl = h_lsqr["resid"][-1] / nb + f * (1 - h_lsqr["resid"][-1] / nb)
        _, h = krylov.hybrid_lsqr(op, b, 10, rule="dp", noise_level=nl)
        lams.append(h["lambda"][-1])
    assert all(l1 < l2 for l1, l2 in zip(lams, lams[1:]))
    assert lams[0] > 0


def test_dp_bisection_brackets_the_root():
    """dp_lambda against a brute-force scan of the projected residual on a
    random bidiagonal H (the root lies between neighbouring scan points)."""
    rng = np.random.default_rng(31)
    k = 8
    h = np.zeros((k + 1, k))
    for i in range(k):
        h[i, i] = rng.uniform(0.05, 2)
        h[i + 1, i] = rng.uniform(0.05, 1)
    beta1 = 1.7
    p, sigma, _ = np.linalg.svd(h, full_matrices=True)
    r0 = krylov.projected_residual(sigma, p[0], beta1, 0.0)
    target = 0.5 * (r0 + beta1)
    lam = krylov.dp_lambda(sigma, p[0], beta1, target)
    # independent check of the residual at lam: solve the regularised problem directly
    y = np.linalg.solve(h.T @ h + lam * lam * np.eye(k), h.T @ (beta1 * np.eye(k + 1)[0]))
    assert abs(np.linalg.norm(beta1 * np.eye(k + 1)[0] - h @ y) - target) <= 1e-8 * beta1
    assert krylov.dp_lambda(sigma, p[0], beta1, 0.5 * r0) == 0.0


# ------------------------------- explicit residuals and the stopping rule (Sec. 3.1.1)
class _UnmatchedOperator:
    """A with a mismatched 'transpose' B = D A^T (D a fixed positive diagonal on
    the voxel side), the situation the paper's toolbox meets with its
    approximately matched backprojector."""

    def __init__(self, a, seed):
        self.a = a
        self.shape = a.shape
        self.d = np.random.default_rng(seed).uniform(0.3, 1.7, a.shape[1])

    def matvec(self, x):
        return self.a @ x

    def rmatvec(self, y):
        return self.d * (self.a.T @ y)


def test_explicit_residuals_equal_lsqr_estimates(tiny_system):
    """With the exact transpose in FP64 the explicit ||b - A x_k|| equals LSQR's
    recurrence estimate, decreases, and never triggers the stop."""
    a, b = tiny_system
    x, h = krylov.explicit_residual_stop(oracle.DenseOperator(a), b, "lsqr", 12)
    assert not h["stopped"] and len(h["iterates"]) == 12
    np.testing.assert_allclose(h["explicit_resid"], h["resid"], rtol=1e-9)
    assert np.all(np.diff(h["explicit_resid"]) < 0)


def test_stop_on_increase_with_unmatched_backprojector(tiny_system):
    """An unmatched B makes the explicit residual of LSQR increase at some k;
    the rule returns x_{k-1} (the unstopped run's iterate), and all residuals
    before the stop decrease."""
    a, b = tiny_system
    op = _UnmatchedOperator(a, 5)
    _, full = krylov.lsqr(op, b, 40, keep_iterates=True)
    res = [np.linalg.norm(b - a @ xk) for xk in full["iterates"]]
    first_up = next(k for k in range(1, len(res)) if res[k] > res[k - 1])      # 0-based index of iterate k+1
    x, h = krylov.explicit_residual_stop(op, b, "lsqr", 40)
    assert h["stopped"]
    assert len(h["iterates"]) == first_up
    np.testing.assert_array_equal(x, full["iterates"][first_up - 1])
    np.testing.assert_allclose(h["explicit_resid"], res[:first_up + 1], rtol=1e-12)
    assert np.all(np.diff(h["explicit_resid"][:-1]) < 0)


def test_stop_on_stalled_decrease(tiny_system):
    """stop_tol = 0.1: stop at the first iteration that reduces the explicit
    residual by less than 10 %."""
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    _, full = krylov.cgls(op, b, 30, keep_iterates=True)
    res = [np.linalg.norm(b - a @ xk) for xk in full["iterates"]]
    k_stall = next(k for k in range(1, len(res)) if res[k] > 0.9 * res[k - 1])
    x, h = krylov.explicit_residual_stop(op, b, "cgls", 30, stop_tol=0.1)
    assert h["stopped"] and len(h["iterates"]) == k_stall
    np.testing.assert_array_equal(x, full["iterates"][k_stall - 1])


# ------------------------------------------------ hybrid LSMR (Sec. 2.2.2 generalisation)
def test_hybrid_lsmr_without_regularisation_is_lsmr(tiny_system):
    """lam = 0: the projected problem is LSMR's own, so x_k is the LSMR iterate."""
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    _, h = krylov.hybrid_lsmr(op, b, 10, rule="fixed", lam=0.0, keep_iterates=True)
    _, h_ref = krylov.lsmr(op, b, 10, keep_iterates=True)
    for k in range(10):
        assert rel(h["iterates"][k], h_ref["iterates"][k]) <= 1e-9
    np.testing.assert_allclose(h["normal_resid"], h_ref["normal_resid"], rtol=1e-7)


@pytest.mark.parametrize("lam", [0.3, 3.0])
def test_hybrid_lsmr_minimises_tikhonov_normal_residual_over_krylov_space(tiny_system, lam):
    """Fixed lam: x_k = argmin over K_k of ||A^T (b - A x)||^2 + lam^2 ||x||^2,
    computed directly on a dense orthonormal basis of K_k."""
    a, b = tiny_system
    k = 8
    x, _ = krylov.hybrid_lsmr(oracle.DenseOperator(a), b, k, rule="fixed", lam=lam)
    v = krylov.krylov_basis(a, b, k)
    aug = np.vstack([a.T @ (a @ v), lam * np.eye(k)])
    rhs = np.concatenate([a.T @ b, np.zeros(k)])
    z = np.linalg.lstsq(aug, rhs, rcond=None)[0]
    assert rel(x, v @ z) <= 1e-8


def test_lsmr_projection_identity(tiny_system):
    """A^T A V_k = V_{k+1} Hbar_k on the Golub-Kahan basis."""
    a, b = tiny_system
    k = 6
    beta = np.linalg.norm(b)
    u = b / beta
    v = a.T @ u
    alpha = np.linalg.norm(v)
    v /= alpha
    alphas, betas, vs = [alpha], [beta], [v]
    for _ in range(k):
        u = a @ v - alpha * u
        beta = np.linalg.norm(u)
        u /= beta
        v = a.T @ u - beta * v
        alpha = np.linalg.norm(v)
        v /= alpha
        alphas.append(alpha)
        betas.append(beta)
        vs.append(v)
    vk, vk1 = np.stack(vs[:k], axis=1), np.stack(vs[:k + 1], axis=1)
    hb = krylov.lsmr_projection(alphas, betas, k)
    assert np.linalg.norm(a.T @ (a @ vk) - vk1 @ hb) <= 1e-9 * np.linalg.norm(a) ** 2


def test_hybrid_lsmr_gcv_runs(tiny_system):
    a, b = tiny_system
    x, h = krylov.hybrid_lsmr(oracle.DenseOperator(a), b, 10, rule="gcv")
    assert all(l > 0 for l in h["lambda"]) and np.isfinite(x).all()


# ------------------------------------------------------ AB-/BA-GMRES (Sec. 2.1.4)
def test_ab_gmres_with_the_transpose_is_lsqr(tiny_system):
    """B = A^T: min ||b - A A^T z|| over K_k(A A^T, b) is LSQR's problem."""
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    _, h = krylov.ab_gmres(op, b, 10, keep_iterates=True)
    _, h_ref = krylov.lsqr(op, b, 10, keep_iterates=True)
    for k in range(10):
        assert rel(h["iterates"][k], h_ref["iterates"][k]) <= 1e-8
    np.testing.assert_allclose(h["resid"], h_ref["resid"], rtol=1e-8)


def test_ba_gmres_with_the_transpose_is_lsmr(tiny_system):
    """B = A^T: min ||A^T (b - A x)|| over K_k(A^T A, A^T b) is LSMR's problem."""
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    _, h = krylov.ba_gmres(op, b, 10, keep_iterates=True)
    _, h_ref = krylov.lsmr(op, b, 10, keep_iterates=True)
    for k in range(10):
        assert rel(h["iterates"][k], h_ref["iterates"][k]) <= 1e-8
    np.testing.assert_allclose(h["resid"], h_ref["normal_resid"], rtol=1e-7)


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_gmres_with_unmatched_backprojector_minimises_over_krylov_space(tiny_system, variant):
    """B = C A^T R (SIRT weights, B != A^T): the iterate is the minimiser of the
    GMRES objective over the Krylov space, computed on a dense basis; the
    residual never increases."""
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    bw = krylov.WeightedBackprojector(op)
    bm = np.diag(bw.c) @ a.T @ np.diag(bw.r)
    assert np.linalg.norm(bm - a.T) > 0.1 * np.linalg.norm(a)
    k = 7
    if variant == "ab":
        x, h = krylov.ab_gmres(op, b, k, backprojector=bw)
        m_op, r0 = a @ bm, b
    else:
        x, h = krylov.ba_gmres(op, b, k, backprojector=bw)
        m_op, r0 = bm @ a, bm @ b
    # dense orthonormal basis of K_k(M, r0)
    q = np.zeros((r0.size, k))
    v = r0 / np.linalg.norm(r0)
    for j in range(k):
        q[:, j] = v
        v = m_op @ v
        for _ in range(2):
            v = v - q[:, :j + 1] @ (q[:, :j + 1].T @ v)
        v = v / np.linalg.norm(v)
    z = np.linalg.lstsq(m_op @ q, r0, rcond=None)[0]
    ref = bm @ (q @ z) if variant == "ab" else q @ z
    assert rel(x, ref) <= 1e-7
    assert np.all(np.diff(h["resid"]) <= 1e-12 * h["resid"][0])


# ------------------------------------------------------------ CGLS-TV (Sec. 2.3)
def test_gradient_adjoint_and_tv_closed_form():
    rng = np.random.default_rng(41)
    x = rng.standard_normal((5, 6, 7))
    u = rng.standard_normal((3, 5, 6, 7))
    lhs = float(np.sum(krylov.grad3(x) * u))
    rhs = float(np.sum(x * krylov.grad3_adjoint(u)))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(u)
    # a unit cube of ones inside zeros: TV counts the jumps across its faces;
    # a voxel next to the cube on its + side along one axis sees one jump of 1,
    # a voxel inside on the - faces sees jumps toward the outside
    c = np.zeros((6, 6, 6))
    c[2:4, 2:4, 2:4] = 1.0
    d = krylov.grad3(c)
    mag = np.sqrt(np.sum(d * d, axis=0))
    assert abs(krylov.total_variation(c) - float(mag.sum())) <= 1e-12
    # brute force by the definition, voxel by voxel
    tv = 0.0
    for k in range(6):
        for j in range(6):
            for i in range(6):
                gi = c[k, j, i + 1] - c[k, j, i] if i < 5 else 0.0
                gj = c[k, j + 1, i] - c[k, j, i] if j < 5 else 0.0
                gk = c[k + 1, j, i] - c[k, j, i] if k < 5 else 0.0
                tv += np.sqrt(gi * gi + gj * gj + gk * gk)
    assert abs(krylov.total_variation(c) - tv) <= 1e-12


def test_irn_weights_give_the_tv_majorant():
    """IRN (Sec. 2.3) works because, per voxel, sqrt(t) <= t / (2 sqrt(c)) +
    sqrt(c) / 2 (equality at t = c): with w = W(D x_k) the quadratic
        Q(x) = sum (|D x|^2 + tau^2) w^2 / 2 + 1 / (2 w^2)
    majorises the smoothed TV, sum sqrt(|D x|^2 + tau^2), and touches it at
    x_k.  Only the exponent -1/4 in w gives both; and as tau -> 0,
    ||W(Dx) D x||^2 tends to TV(x)."""
    rng = np.random.default_rng(43)
    tau = 0.1
    xk = rng.standard_normal((5, 6, 7))
    w2 = krylov.irn_weights(xk, tau) ** 2

    def smoothed_tv(x):
        return float(np.sum(np.sqrt(np.sum(krylov.grad3(x) ** 2, axis=0) + tau * tau)))

    def q(x):
        t = np.sum(krylov.grad3(x) ** 2, axis=0) + tau * tau
        return float(np.sum(t * w2 / 2 + 1 / (2 * w2)))

    assert abs(q(xk) - smoothed_tv(xk)) <= 1e-12 * smoothed_tv(xk)
    for _ in range(20):
        x = xk + rng.standard_normal(xk.shape) * rng.uniform(0.01, 3.0)
        assert q(x) >= smoothed_tv(x) * (1 - 1e-12)
    c = np.zeros((6, 6, 6))
    c[2:4, 2:4, 2:4] = 1.0
    wc = krylov.irn_weights(c, 1e-9)
    weighted = float(np.sum(wc ** 2 * np.sum(krylov.grad3(c) ** 2, axis=0)))
    assert abs(weighted - krylov.total_variation(c)) <= 1e-8 * krylov.total_variation(c)


def test_cgls_tv_inner_solve_is_the_weighted_tikhonov_solution(tiny_system):
    """One outer step with enough inner iterations reaches the solution of the
    normal equations (A^T A + lam^2 D^T W^2 D) x = A^T b (dense solve)."""
    a, b = tiny_system
    g = synth.config("tiny")
    shape = g.vol_shape
    lam, tau = 0.5, 1e-2
    x, _ = krylov.cgls_tv(oracle.DenseOperator(a), shape, b, 1, 1000, lam, tau)
    m = a.shape[1]
    eye = np.eye(m)
    dmat = np.stack([krylov.grad3(eye[:, c].reshape(shape)).ravel() for c in range(m)], axis=1)   # (3M, M)
    w = krylov.irn_weights(np.zeros(shape), tau).ravel()
    w3 = np.concatenate([w, w, w])
    lhs = a.T @ a + lam * lam * dmat.T @ (w3[:, None] ** 2 * dmat)
    x_ref = np.linalg.solve(lhs, a.T @ b)
    assert rel(x.ravel(), x_ref) <= 1e-6


def test_cgls_tv_objective_decreases(tiny_system):
    """IRN is a majorise-minimise scheme: with (nearly) exact inner solves the
    TV objective ||A x - b||^2 + lam^2 TV(x) does not increase."""
    a, b = tiny_system
    shape = synth.config("tiny").vol_shape
    _, h = krylov.cgls_tv(oracle.DenseOperator(a), shape, b, 6, 150, 0.5, 1e-3)
    obj = h["objective"]
    assert all(o2 <= o1 * (1 + 1e-6) for o1, o2 in zip(obj, obj[1:]))


# --------------------------------------- re-orthogonalised Golub-Kahan (Sec. 3.1.1, Sec. 4)
@pytest.mark.parametrize("method", ["lsqr", "lsmr", "hybrid_lsqr"])
def test_reorthogonalised_iterates_equal_plain_ones(tiny_system, method):
    """In FP64 on a well-conditioned range the re-orthogonalised process gives
    the same iterates (re-orthogonalisation only removes rounding)."""
    a, b = tiny_system
    op = oracle.DenseOperator(a)
    kw = {"rule": "fixed", "lam": 0.5} if method == "hybrid_lsqr" else {}
    _, h0 = getattr(krylov, method)(op, b, 10, keep_iterates=True, **kw)
    _, h1 = getattr(krylov, method)(op, b, 10, keep_iterates=True, reorth=True, **kw)
    for k in range(10):
        assert rel(h1["iterates"][k], h0["iterates"][k]) <= 1e-8


def test_reorthogonalisation_keeps_the_basis_orthonormal(tiny_system):
    """Run long enough that plain Golub-Kahan loses orthogonality, and compare
    ||V_k^T V_k - I|| of both processes (v_k recovered from the LSQR
    directions is awkward, so the hybrid solver's stored basis is used)."""
    a, b = tiny_system
    k = 60

    def basis(reorth):
        u = b / np.linalg.norm(b)
        v = a.T @ u
        alpha = np.linalg.norm(v)
        v /= alpha
        us, vs = [u], [v]
        for _ in range(k):
            u = a @ v - alpha * u
            if reorth:
                u = krylov._reorthogonalise(u, us)
            beta = np.linalg.norm(u)
            u /= beta
            us.append(u)
            v = a.T @ u - beta * v
            if reorth:
                v = krylov._reorthogonalise(v, vs)
            alpha = np.linalg.norm(v)
            v /= alpha
            vs.append(v)
        vm = np.stack(vs, axis=1)
        return np.linalg.norm(vm.T @ vm - np.eye(vm.shape[1]))

    plain, re = basis(False), basis(True)
    assert re <= 1e-12
    assert plain > 1e3 * re


def test_voxel_driven_backprojector_interpolates_exactly_and_approximates_the_transpose():
    """A projection that is linear in the detector coordinates is sampled
    exactly at every voxel's projected centre (bilinear interpolation), and the
    weights make B 1 match A^T 1 on average inside the volume (B is an
    approximation of A^T, not the transpose)."""
    g = synth.Geometry(12, 12, 12, 1.0, 1.0, 1.0, 40, 40, 1.0, 1.0, 200.0, 300.0, np.radians([0.0, 37.0]))
    bp = krylov.VoxelDrivenBackprojector(g)
    iu = np.arange(g.nu, dtype=np.float64)
    iv = np.arange(g.nv, dtype=np.float64)
    lin = 0.3 * iu[None, :] + 0.7 * iv[:, None] + 2.0
    one_angle = synth.Geometry(12, 12, 12, 1.0, 1.0, 1.0, 40, 40, 1.0, 1.0, 200.0, 300.0, np.radians([37.0]))
    b1 = krylov.VoxelDrivenBackprojector(one_angle)
    out = b1(lin[None]).reshape(one_angle.vol_shape)
    weight = b1(np.ones((1, g.nv, g.nu))).reshape(one_angle.vol_shape)
    # expected: the linear function at the projected centre of every voxel
    t = np.radians(37.0)
    zz, yy, xx = np.meshgrid(bp.zc, bp.yc, bp.xc, indexing="ij")
    mag = g.dsd / (g.dso - (xx * np.cos(t) + yy * np.sin(t)))
    fu = (-xx * np.sin(t) + yy * np.cos(t)) * mag / g.du + 0.5 * (g.nu - 1)
    fv = zz * mag / g.dv + 0.5 * (g.nv - 1)
    np.testing.assert_allclose(out / weight, 0.3 * fu + 0.7 * fv + 2.0, rtol=1e-12)
    full = synth.Geometry(12, 12, 12, 1.0, 1.0, 1.0, 40, 40, 1.0, 1.0, 200.0, 300.0, synth.circular_angles(90))
    op = oracle.Operator(full)
    bp = krylov.VoxelDrivenBackprojector(full)
    r = bp(np.ones(full.num_rays)).reshape(full.vol_shape) / op.rmatvec(np.ones(full.num_rays)).reshape(full.vol_shape)
    inner = r[2:-2, 2:-2, 2:-2]
    assert 0.9 < inner.mean() < 1.1


def test_voxel_driven_weight_is_the_ray_density():
    """With pixels much finer than the voxels (20 rays per voxel width at the
    rotation centre) A^T 1 at a voxel is its volume times the density of rays
    through it, which the voxel-driven weight dx dy dz mag^2 |d'| / (du dv DSD)
    states in closed form: B 1 = A^T 1 per voxel within 0.5 %, on a wide cone
    (|d'| / DSD up to 1.03 averaged over the angles, so a dropped |d'| factor,
    a wrong power of mag or a missing pixel area fails)."""
    g = synth.Geometry(8, 8, 8, 1.0, 1.0, 1.0, 300, 300, 0.1, 0.1, 20.0, 40.0, synth.circular_angles(8))
    ones = np.ones(g.proj_shape)
    ratio = krylov.VoxelDrivenBackprojector(g)(ones) / oracle.backproject(g, ones).ravel()
    assert np.abs(ratio - 1.0).max() < 5e-3


def test_sirt_weighted_backprojector_inverts_a_on_constants():
    """With R = 1 / (A 1) and C = 1 / (A^T 1), B = C A^T R maps A 1 back to 1
    on every voxel some ray meets (R A 1 = 1 on every ray that meets the
    volume, then C A^T 1 = 1), and B y is zero where no ray meets the voxel;
    swapping R and C, or dropping either, breaks it.  B is not A^T: <A x, y> and
    <x, B y> differ."""
    g = synth.Geometry(10, 9, 8, 1.0, 1.0, 1.0, 4, 10, 1.3, 1.3, 60.0, 100.0, np.radians([0.0, 90.0]))
    op = oracle.Operator(g)
    bw = krylov.WeightedBackprojector(op)
    one = np.ones(op.shape[1])
    met = op.rmatvec(np.ones(op.shape[0])) > 0
    assert 0 < met.sum() < met.size                          # the narrow detector misses the corners
    out = bw(op.matvec(one))
    np.testing.assert_allclose(out[met], 1.0, rtol=1e-12)
    assert np.all(out[~met] == 0.0)
    rng = np.random.default_rng(44)
    x, y = rng.standard_normal(op.shape[1]), rng.standard_normal(op.shape[0])
    assert abs(np.dot(op.matvec(x), y) - np.dot(x, bw(y))) > 1e-3 * abs(np.dot(op.matvec(x), y))
