"""Textbook Krylov least-squares solvers in FP64 numpy (test infrastructure).

TEST INFRASTRUCTURE: used by the tests, the smoke check and the CPU baseline
only; the GPU library never imports it.

Every solver starts from x_0 = 0, runs a fixed number of iterations and takes an
operator with ``matvec`` (A x) and ``rmatvec`` (A^T y) on flat vectors.  Each
follows the recurrences of the method's original publication, step by step, in
that publication's notation:

* ``cgls``  -- conjugate gradients on the normal equations A^T A x = A^T b
  (Sec. 2.1.1, Eq. 3; Hestenes-Stiefel), optionally on the damped system
  [A; lam I] x ~ [b; 0] of Sec. 2.2, Eq. 7.
* ``lsqr``  -- Golub-Kahan bidiagonalisation A V_k = U_{k+1} H_k with the
  Paige-Saunders short recurrences (Sec. 2.1.2, Eq. 4), optional damping.
* ``lsmr``  -- Golub-Kahan with the Fong-Saunders recurrences minimising
  ||A^T r_k|| (Sec. 2.1.3, Eq. 5), optional damping lam (Sec. 2.2, Eq. 7).
* ``hybrid_lsqr`` -- Tikhonov on the projected LSQR problem with lam_k per
  iteration (Sec. 2.2.1, Eq. 8), lam_k fixed or chosen by GCV (Sec. 2.2.2).
* ``krylov_reference`` -- the dense definition used to pin the recurrences:
  an orthonormal basis of K_k(A^T A, A^T b) (Sec. 2, Eq. 2 of the Methods
  introduction) and the small least-squares problem each method minimises.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["cgls", "lsqr", "lsmr", "hybrid_lsqr", "gcv_lambda", "gcv_function",
           "projected_tikhonov", "krylov_basis", "krylov_reference"]


def _norm(v):
    return float(np.sqrt(np.dot(v, v)))


def _reorthogonalise(vec, basis):
    """Classical Gram-Schmidt against the stored orthonormal vectors, applied
    twice ("twice is enough"): removes the components along earlier Krylov
    vectors that rounding reintroduces (the re-orthogonalisation the paper
    discusses for LSQR-type methods, Sec. 3.1.1 and Sec. 4)."""
    if not basis:
        return vec
    q = np.stack(basis, axis=1)
    for _ in range(2):
        vec = vec - q @ (q.T @ vec)
    return vec


def _rotation(a, b):
    """Givens rotation (c, s, r) with [c s; -s c] [a; b] = [r; 0], r = hypot(a, b) >= 0."""
    r = math.hypot(a, b)
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


# --------------------------------------------------------------------------- CGLS
def cgls(op, b, iters, damp=0.0, keep_iterates=False):
    """CGLS (Sec. 2.1.1): x_k minimises ||A x - b|| over K_k(A^T A, A^T b).

    With damp = lam the same recurrence runs on [A; lam I] x ~ [b; 0] (Eq. 7).
    History: ``resid`` = ||b - A x_k|| (carried explicitly as r_k),
    ``normal_resid`` = ||A^T r_k - lam^2 x_k||.
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    lam2 = float(damp) ** 2
    x = np.zeros(op.shape[1])
    r = b.copy()
    s = op.rmatvec(r)                      # s_0 = A^T r_0 - lam^2 x_0
    p = s.copy()
    gamma = float(np.dot(s, s))
    hist = {"resid": [], "normal_resid": [], "iterates": []}
    for _ in range(iters):
        q = op.matvec(p)
        delta = float(np.dot(q, q)) + lam2 * float(np.dot(p, p))
        if delta == 0.0 or gamma == 0.0:
            break
        alpha = gamma / delta
        x = x + alpha * p
        r = r - alpha * q
        s = op.rmatvec(r) - lam2 * x
        gamma_new = float(np.dot(s, s))
        beta = gamma_new / gamma
        p = s + beta * p
        gamma = gamma_new
        hist["resid"].append(_norm(r))
        hist["normal_resid"].append(math.sqrt(gamma))
        if keep_iterates:
            hist["iterates"].append(x.copy())
    return x, hist


# --------------------------------------------------------------------------- LSQR
def lsqr(op, b, iters, damp=0.0, keep_iterates=False, reorth=False):
    """LSQR (Sec. 2.1.2): Golub-Kahan bidiagonalisation + Paige-Saunders recurrences.

    Bidiagonalisation: beta_1 u_1 = b, alpha_1 v_1 = A^T u_1,
    beta_{i+1} u_{i+1} = A v_i - alpha_i u_i,
    alpha_{i+1} v_{i+1} = A^T u_{i+1} - beta_{i+1} v_i.
    With damp = lam > 0 a first rotation eliminates lam from the augmented
    bidiagonal (Eq. 7 projected).  History: ``resid`` = phibar estimate of
    ||r_k|| (augmented residual when damped), ``normal_resid`` =
    phibar alpha |c| estimate of ||A^T r_k||, ``alpha``/``beta`` = the
    bidiagonal entries.
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    lam = float(damp)
    x = np.zeros(op.shape[1])
    beta = _norm(b)
    hist = {"resid": [], "normal_resid": [], "alpha": [], "beta": [beta], "iterates": []}
    if beta == 0.0:
        return x, hist
    u = b / beta
    ub = [u] if reorth else []
    v = op.rmatvec(u)
    alpha = _norm(v)
    hist["alpha"].append(alpha)
    if alpha == 0.0:
        return x, hist
    v = v / alpha
    vb = [v] if reorth else []
    w = v.copy()
    phibar = beta
    rhobar = alpha
    psi_sq = 0.0
    for _ in range(iters):
        u = op.matvec(v) - alpha * u
        if reorth:
            u = _reorthogonalise(u, ub)
        beta = _norm(u)
        if beta > 0.0:
            u = u / beta
        if reorth:
            ub.append(u)
        v = op.rmatvec(u) - beta * v
        if reorth:
            v = _reorthogonalise(v, vb)
        alpha_next = _norm(v)
        if alpha_next > 0.0:
            v = v / alpha_next
        if reorth:
            vb.append(v)
        hist["beta"].append(beta)
        hist["alpha"].append(alpha_next)
        # rotation that eliminates the damping term
        c1, s1, rhobar1 = _rotation(rhobar, lam)
        psi = s1 * phibar
        phibar = c1 * phibar
        psi_sq += psi * psi
        # rotation that eliminates beta_{i+1}
        c, s, rho = _rotation(rhobar1, beta)
        theta = s * alpha_next
        rhobar = -c * alpha_next
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        alpha = alpha_next
        hist["resid"].append(math.sqrt(phibar * phibar + psi_sq))
        hist["normal_resid"].append(abs(phibar * alpha_next * c))
        if keep_iterates:
            hist["iterates"].append(x.copy())
        if beta == 0.0 or alpha_next == 0.0:
            break
    return x, hist


# --------------------------------------------------------------------------- LSMR
def lsmr(op, b, iters, damp=0.0, keep_iterates=False, reorth=False):
    """LSMR (Sec. 2.1.3): Golub-Kahan + Fong-Saunders recurrences.

    x_k minimises ||A^T r_k|| (of the damped system when damp = lam) over
    K_k(A^T A, A^T b).  Three rotations per step: P-hat eliminates the damping,
    P turns the bidiagonal into upper-triangular R_k, P-bar turns R_k^T into
    upper-bidiagonal R-bar_k.  History: ``normal_resid`` = |zeta-bar_{k+1}|
    estimate of ||A^T r_k - lam^2 x_k||, ``resid`` = the ||r_k|| estimate from
    the same publication's extra rotations (Q-hat, Q, Q-tilde).
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    lam = float(damp)
    x = np.zeros(op.shape[1])
    beta = _norm(b)
    hist = {"resid": [], "normal_resid": [], "iterates": []}
    if beta == 0.0:
        return x, hist
    u = b / beta
    ub = [u] if reorth else []
    v = op.rmatvec(u)
    alpha = _norm(v)
    if alpha == 0.0:
        return x, hist
    v = v / alpha
    vb = [v] if reorth else []

    alphabar = alpha
    zetabar = alpha * beta
    rho = 1.0
    rhobar = 1.0
    cbar, sbar = 1.0, 0.0
    h = v.copy()
    hbar = np.zeros_like(x)
    # state of the ||r_k|| estimate
    betadd = beta          # beta-double-dot
    betad = 0.0            # beta-dot
    rhod = 1.0             # rho-dot of the previous step
    tautilde = 0.0
    thetatilde = 0.0
    zeta = 0.0
    dsum = 0.0

    for _ in range(iters):
        u = op.matvec(v) - alpha * u
        if reorth:
            u = _reorthogonalise(u, ub)
        beta = _norm(u)
        if beta > 0.0:
            u = u / beta
        if reorth:
            ub.append(u)
        v = op.rmatvec(u) - beta * v
        if reorth:
            v = _reorthogonalise(v, vb)
        alpha = _norm(v)
        if alpha > 0.0:
            v = v / alpha
        if reorth:
            vb.append(v)

        chat, shat, alphahat = _rotation(alphabar, lam)          # P-hat_k
        rho_prev = rho
        c, s, rho = _rotation(alphahat, beta)                   # P_k
        theta_next = s * alpha
        alphabar = c * alpha

        rhobar_prev = rhobar                                     # P-bar_k
        zeta_prev = zeta
        thetabar = sbar * rho
        cbar, sbar, rhobar = _rotation(cbar * rho, theta_next)
        zeta = cbar * zetabar
        zetabar = -sbar * zetabar

        hbar = h - (thetabar * rho / (rho_prev * rhobar_prev)) * hbar
        x = x + (zeta / (rho * rhobar)) * hbar
        h = v - (theta_next / rho) * h

        # ||r_k||: apply Q-hat_k and Q_k to (beta-double-dot, 0), then Q-tilde_{k-1}
        betaacute = chat * betadd
        betacheck = -shat * betadd
        betahat = c * betaacute
        betadd = -s * betaacute
        thetatilde_prev = thetatilde
        ctilde, stilde, rhotilde_prev = _rotation(rhod, thetabar)
        thetatilde = stilde * rhobar
        rhod = ctilde * rhobar
        betad = -stilde * betad + ctilde * betahat
        tautilde = (zeta_prev - thetatilde_prev * tautilde) / rhotilde_prev
        taud = (zeta - thetatilde * tautilde) / rhod
        dsum += betacheck * betacheck
        hist["resid"].append(math.sqrt(dsum + (betad - taud) ** 2 + betadd * betadd))
        hist["normal_resid"].append(abs(zetabar))
        if keep_iterates:
            hist["iterates"].append(x.copy())
        if beta == 0.0 or alpha == 0.0:
            break
    return x, hist


# ------------------------------------------------------------------ hybrid LSQR + GCV
def _bidiagonal(alphas, betas, k):
    """H_k ((k+1) x k lower bidiagonal): H[i,i] = alpha_{i+1}, H[i+1,i] = beta_{i+2}."""
    h = np.zeros((k + 1, k))
    for i in range(k):
        h[i, i] = alphas[i]
        h[i + 1, i] = betas[i + 1]
    return h


def gcv_function(sigma, p1, beta1, lam):
    """GCV of the projected problem (Sec. 2.2.2) at lam, from H_k = P Sigma Q^T.

    G(lam) = ||(I - H H^+_lam) beta1 e1||^2 / (trace(I - H H^+_lam))^2 with
    H^+_lam = (H^T H + lam^2 I)^{-1} H^T; p1 = first row of P (length k+1).
    """
    k = sigma.shape[0]
    s2 = sigma * sigma
    l2 = lam * lam
    f = l2 / (s2 + l2)                               # 1 - filter factor
    num = float(np.sum((f * beta1 * p1[:k]) ** 2) + (beta1 * p1[k]) ** 2)
    den = float((k + 1) - np.sum(s2 / (s2 + l2)))
    return num / (den * den)


GCV_GRID_POINTS = 200
GCV_GRID_DECADES = 8.0
GCV_REL_TOL = 1e-10


def gcv_lambda(sigma, p1, beta1):
    """Minimiser of the GCV function.

    The paper gives no minimisation procedure.  Reading used here: evaluate G on
    200 log-spaced points over [sigma_max 1e-8, sigma_max]; take the smallest
    value (ties to the larger lam); refine by golden-section search in log lam on
    the neighbouring grid bracket until the bracket is narrower than 1e-10
    relative.
    """
    smax = float(np.max(sigma))
    if smax == 0.0:
        return 0.0
    lo_exp = math.log(smax) - GCV_GRID_DECADES * math.log(10.0)
    hi_exp = math.log(smax)
    n = GCV_GRID_POINTS
    grid = [lo_exp + (hi_exp - lo_exp) * i / (n - 1) for i in range(n)]
    vals = [gcv_function(sigma, p1, beta1, math.exp(t)) for t in grid]
    best = 0
    for i in range(1, n):
        if vals[i] <= vals[best]:
            best = i
    a = grid[max(best - 1, 0)]
    c = grid[min(best + 1, n - 1)]
    invphi = (math.sqrt(5.0) - 1.0) / 2.0
    x1 = c - invphi * (c - a)
    x2 = a + invphi * (c - a)
    f1 = gcv_function(sigma, p1, beta1, math.exp(x1))
    f2 = gcv_function(sigma, p1, beta1, math.exp(x2))
    while c - a > GCV_REL_TOL:
        if f1 < f2:
            c, x2, f2 = x2, x1, f1
            x1 = c - invphi * (c - a)
            f1 = gcv_function(sigma, p1, beta1, math.exp(x1))
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + invphi * (c - a)
            f2 = gcv_function(sigma, p1, beta1, math.exp(x2))
    t = 0.5 * (a + c)
    # keep the grid point if the refinement did not improve on it
    if gcv_function(sigma, p1, beta1, math.exp(t)) > vals[best]:
        t = grid[best]
    return math.exp(t)


def projected_residual(sigma, p1, beta1, lam):
    """||beta1 e1 - H_k y_lam|| of the projected Tikhonov solution (Eq. 8), from
    H_k = P Sigma Q^T: the component of beta1 e1 outside range(H_k) plus the
    filtered part inside it (the numerator of the GCV function, square-rooted)."""
    k = sigma.shape[0]
    s2 = sigma * sigma
    l2 = lam * lam
    f = l2 / (s2 + l2)
    return math.sqrt(float(np.sum((f * beta1 * p1[:k]) ** 2) + (beta1 * p1[k]) ** 2))


DP_DECADES = 8.0
DP_REL_TOL = 1e-10


def dp_lambda(sigma, p1, beta1, target):
    """Discrepancy principle (Sec. 2.2.2): lam with ||b - A x_lam|| = target
    (= nl ||b||), on the projected problem, where ||b - A V_k y|| equals
    ||beta1 e1 - H_k y||.

    The paper prints an argmin of ||A x_lam - b||^2 - nl^2 ||b||^2, unbounded
    below as written; the reading here is the root of the equality.  The
    projected residual grows monotonically with lam, so the root is bracketed
    in log lam over [sigma_max 1e-8, sigma_max 1e8] and found by bisection to a
    bracket narrower than 1e-10 (relative); if even the smallest lam leaves a
    residual above the target (too few iterations yet), lam = 0, and if the
    largest one stays below it, lam = the upper end.
    """
    smax = float(np.max(sigma))
    if smax == 0.0:
        return 0.0
    lo = math.log(smax) - DP_DECADES * math.log(10.0)
    hi = math.log(smax) + DP_DECADES * math.log(10.0)
    if projected_residual(sigma, p1, beta1, math.exp(lo)) >= target:
        return 0.0
    if projected_residual(sigma, p1, beta1, math.exp(hi)) <= target:
        return math.exp(hi)
    while hi - lo > DP_REL_TOL:
        mid = 0.5 * (lo + hi)
        if projected_residual(sigma, p1, beta1, math.exp(mid)) < target:
            lo = mid
        else:
            hi = mid
    return math.exp(0.5 * (lo + hi))


def projected_tikhonov(h, beta1, lam, svd=None):
    """y = argmin ||beta1 e1 - H y||^2 + lam^2 ||y||^2 (Eq. 8) via the SVD H = P Sigma Q^T."""
    p, sigma, qt = np.linalg.svd(h, full_matrices=True) if svd is None else svd
    k = h.shape[1]
    denom = sigma * sigma + lam * lam
    coef = np.where(denom > 0.0, sigma * beta1 * p[0, :k] / np.where(denom > 0.0, denom, 1.0), 0.0)
    return qt.T @ coef


def hybrid_lsqr(op, b, iters, rule="gcv", lam=0.0, keep_iterates=False, noise_level=0.0, reorth=False):
    """Hybrid LSQR (Sec. 2.2.1, Eq. 8) with lam_k fixed, chosen by GCV or by the
    discrepancy principle with relative noise level nl = noise_level (Sec. 2.2.2).

    Stores the basis V_k; at every iteration k solves the projected Tikhonov
    problem for y_k and forms x_k = V_k y_k.  History: ``resid`` = projected
    residual ||beta1 e1 - H_k y_k|| (equal to ||b - A x_k|| in exact arithmetic),
    ``lambda`` = lam_k, ``alpha``/``beta`` = bidiagonal entries.
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros(op.shape[1])
    beta1 = _norm(b)
    hist = {"resid": [], "lambda": [], "alpha": [], "beta": [beta1], "iterates": []}
    if beta1 == 0.0:
        return x, hist
    u = b / beta1
    ub = [u] if reorth else []
    v = op.rmatvec(u)
    alpha = _norm(v)
    hist["alpha"].append(alpha)
    if alpha == 0.0:
        return x, hist
    v = v / alpha
    vb = [v] if reorth else []
    basis = [v]
    for k in range(1, iters + 1):
        u = op.matvec(v) - alpha * u
        if reorth:
            u = _reorthogonalise(u, ub)
        beta = _norm(u)
        if beta > 0.0:
            u = u / beta
        if reorth:
            ub.append(u)
        v = op.rmatvec(u) - beta * v
        if reorth:
            v = _reorthogonalise(v, vb)
        alpha = _norm(v)
        if alpha > 0.0:
            v = v / alpha
        if reorth:
            vb.append(v)
        hist["beta"].append(beta)
        hist["alpha"].append(alpha)
        h = _bidiagonal(hist["alpha"], hist["beta"], k)
        svd = np.linalg.svd(h, full_matrices=True)
        if rule == "gcv":
            lam_k = gcv_lambda(svd[1], svd[0][0, :], beta1)
        elif rule == "dp":
            lam_k = dp_lambda(svd[1], svd[0][0, :], beta1, noise_level * beta1)
        elif rule == "fixed":
            lam_k = float(lam)
        else:
            raise ValueError(rule)
        y = projected_tikhonov(h, beta1, lam_k, svd)
        x = np.stack(basis, axis=1) @ y
        rhs = np.zeros(k + 1)
        rhs[0] = beta1
        hist["resid"].append(_norm(rhs - h @ y))
        hist["lambda"].append(lam_k)
        if keep_iterates:
            hist["iterates"].append(x.copy())
        basis.append(v)
        if beta == 0.0 or alpha == 0.0:
            break
    return x, hist


# ------------------------------------------------------------- hybrid LSMR
def lsmr_projection(alphas, betas, k):
    """LSMR's projected matrix after k Golub-Kahan steps (Fong-Saunders):
    A^T A V_k = V_{k+1} Hbar_k with Hbar_k = [H_k^T H_k ; alpha_{k+1} beta_{k+1} e_k^T]
    ((k+1) x k), and A^T b = alpha_1 beta_1 v_1, so that
    A^T (b - A V_k y) = V_{k+1} (alpha_1 beta_1 e_1 - Hbar_k y)."""
    h = _bidiagonal(alphas, betas, k)
    hb = np.zeros((k + 1, k))
    hb[:k, :] = h.T @ h
    hb[k, k - 1] = alphas[k] * betas[k]
    return hb


def hybrid_lsmr(op, b, iters, rule="gcv", lam=0.0, keep_iterates=False):
    """Hybrid LSMR: Tikhonov regularisation of LSMR's projected problem,
        y_k = argmin ||alpha_1 beta_1 e_1 - Hbar_k y||^2 + lam_k^2 ||y||^2,
    x_k = V_k y_k, i.e. x_k minimises ||A^T (b - A x)||^2 + lam_k^2 ||x||^2 over
    K_k(A^T A, A^T b); lam_k fixed or by GCV on the projected problem.  The
    paper (Sec. 2.2.2) remarks that GCV carries over to LSMR with LSMR's own
    small projected system in place of LSQR's; this is that system.  History: ``normal_resid`` = ||alpha_1 beta_1 e_1 - Hbar_k y_k||
    (= ||A^T r_k|| in exact arithmetic), ``lambda``, ``alpha``/``beta``."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros(op.shape[1])
    beta1 = _norm(b)
    hist = {"normal_resid": [], "lambda": [], "alpha": [], "beta": [beta1], "iterates": []}
    if beta1 == 0.0:
        return x, hist
    u = b / beta1
    v = op.rmatvec(u)
    alpha = _norm(v)
    hist["alpha"].append(alpha)
    if alpha == 0.0:
        return x, hist
    v = v / alpha
    rhs1 = alpha * beta1
    basis = [v]
    for k in range(1, iters + 1):
        u = op.matvec(v) - alpha * u
        beta = _norm(u)
        if beta > 0.0:
            u = u / beta
        v = op.rmatvec(u) - beta * v
        alpha = _norm(v)
        if alpha > 0.0:
            v = v / alpha
        hist["beta"].append(beta)
        hist["alpha"].append(alpha)
        hb = lsmr_projection(hist["alpha"], hist["beta"], k)
        svd = np.linalg.svd(hb, full_matrices=True)
        if rule == "gcv":
            lam_k = gcv_lambda(svd[1], svd[0][0, :], rhs1)
        elif rule == "fixed":
            lam_k = float(lam)
        else:
            raise ValueError(rule)
        y = projected_tikhonov(hb, rhs1, lam_k, svd)
        x = np.stack(basis, axis=1) @ y
        rhs = np.zeros(k + 1)
        rhs[0] = rhs1
        hist["normal_resid"].append(_norm(rhs - hb @ y))
        hist["lambda"].append(lam_k)
        if keep_iterates:
            hist["iterates"].append(x.copy())
        basis.append(v)
        if beta == 0.0 or alpha == 0.0:
            break
    return x, hist


# ------------------------------------------------------------- AB-/BA-GMRES
def sirt_weights(op):
    """R = 1 / (A 1) (each ray's length inside the volume) and C = 1 / (A^T 1)
    (each voxel's total intersection length), 0 where the sum is 0: the
    diagonal weights of the SIRT family."""
    m = op.shape[1]
    row = op.matvec(np.ones(m))
    col = op.rmatvec(np.ones(op.shape[0]))
    r = np.where(row > 0, 1.0 / np.where(row > 0, row, 1.0), 0.0)
    c = np.where(col > 0, 1.0 / np.where(col > 0, col, 1.0), 0.0)
    return r, c


class WeightedBackprojector:
    """B = C A^T R (SIRT weights): a backprojector that is not the transpose of
    A, standing in for the approximately matched backprojectors the paper's
    AB-/BA-GMRES are meant for (Sec. 2.1.4)."""

    def __init__(self, op):
        self.op = op
        self.r, self.c = sirt_weights(op)

    def __call__(self, y):
        return self.c * self.op.rmatvec(self.r * np.asarray(y, dtype=np.float64).reshape(-1))


class VoxelDrivenBackprojector:
    """A voxel-driven, interpolating backprojector, the usual fast GPU
    approximation of A^T that is not its exact transpose (Sec. 2.1.4): every
    voxel centre is projected onto every detector and the projection is
    sampled there by bilinear interpolation (zero outside the detector),
    weighted by the expected sum of A's entries of the rays through the voxel,
        w = dx dy dz mag^2 |d'| / (du dv DSD),   mag = DSD / (DSO - <c, s_hat>),
    |d'| the source-to-pixel distance of the sampled point: rays through the
    voxel are spaced du dv DSD / (|d'| mag^2) apart perpendicular to their
    direction at the voxel's depth.  Geometry conventions as the projector's
    (rotation axis z, source (DSO cos t, DSO sin t, 0), detector u along
    (-sin t, cos t, 0), v along z)."""

    def __init__(self, g):
        self.g = g
        nx, ny, nz = g.nx, g.ny, g.nz
        self.xc = (np.arange(nx) - 0.5 * (nx - 1)) * g.dx
        self.yc = (np.arange(ny) - 0.5 * (ny - 1)) * g.dy
        self.zc = (np.arange(nz) - 0.5 * (nz - 1)) * g.dz

    def __call__(self, y):
        g = self.g
        y = np.asarray(y, dtype=np.float64).reshape(g.nangles, g.nv, g.nu)
        zz, yy, xx = np.meshgrid(self.zc, self.yc, self.xc, indexing="ij")
        out = np.zeros((g.nz, g.ny, g.nx))
        vol = g.dx * g.dy * g.dz
        for a, t in enumerate(g.angles):
            ct, st = math.cos(t), math.sin(t)
            along = g.dso - (xx * ct + yy * st)
            mag = g.dsd / along
            u = (-xx * st + yy * ct) * mag
            v = zz * mag
            fu = u / g.du + 0.5 * (g.nu - 1)
            fv = v / g.dv + 0.5 * (g.nv - 1)
            iu = np.floor(fu).astype(np.int64)
            iv = np.floor(fv).astype(np.int64)
            tu = fu - iu
            tv = fv - iv
            val = np.zeros_like(fu)
            for du_, dv_, wgt in ((0, 0, (1 - tu) * (1 - tv)), (1, 0, tu * (1 - tv)),
                                  (0, 1, (1 - tu) * tv), (1, 1, tu * tv)):
                cu, cv = iu + du_, iv + dv_
                ok = (cu >= 0) & (cu < g.nu) & (cv >= 0) & (cv < g.nv)
                val += np.where(ok, wgt * y[a, np.clip(cv, 0, g.nv - 1), np.clip(cu, 0, g.nu - 1)], 0.0)
            dlen = np.sqrt(g.dsd * g.dsd + u * u + v * v)
            out += vol * mag * mag * dlen / (g.du * g.dv * g.dsd) * val
        return out.ravel()


def _arnoldi_gmres(apply, r0, iters):
    """GMRES on K_k(M, r0) for the operator `apply` = M: Arnoldi with modified
    Gram-Schmidt in FP64; y_k = argmin ||beta e_1 - Hbar_k y|| for every k.
    Returns (basis list, [y_k], [||beta e_1 - Hbar_k y_k||])."""
    beta = _norm(r0)
    if beta == 0.0:
        return [], [], []
    vs = [r0 / beta]
    h = np.zeros((iters + 1, iters))
    ys, res = [], []
    for j in range(iters):
        w = apply(vs[j])
        for i in range(j + 1):
            h[i, j] = float(np.dot(w, vs[i]))
            w = w - h[i, j] * vs[i]
        h[j + 1, j] = _norm(w)
        rhs = np.zeros(j + 2)
        rhs[0] = beta
        y = np.linalg.lstsq(h[:j + 2, :j + 1], rhs, rcond=None)[0]
        ys.append(y)
        res.append(_norm(rhs - h[:j + 2, :j + 1] @ y))
        if h[j + 1, j] == 0.0:
            break
        vs.append(w / h[j + 1, j])
    return vs, ys, res


def ab_gmres(op, b, iters, backprojector=None, keep_iterates=False):
    """AB-GMRES (Sec. 2.1.4): GMRES on min ||b - A B z|| (B as a right
    preconditioner), x_k = B z_k, z_k in K_k(A B, b).  B defaults to A^T, in
    which case x_k is the LSQR iterate.  History: ``resid`` = ||b - A x_k||
    from the Hessenberg least-squares problem."""
    bproj = backprojector or op.rmatvec
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    vs, ys, res = _arnoldi_gmres(lambda z: op.matvec(bproj(z)), b, iters)
    hist = {"resid": res, "iterates": []}
    if not ys:
        return np.zeros(op.shape[1]), hist
    if keep_iterates:
        for y in ys:
            hist["iterates"].append(bproj(np.stack(vs[:len(y)], axis=1) @ y))
        return hist["iterates"][-1].copy(), hist
    y = ys[-1]
    return bproj(np.stack(vs[:len(y)], axis=1) @ y), hist


def ba_gmres(op, b, iters, backprojector=None, keep_iterates=False):
    """BA-GMRES (Sec. 2.1.4): GMRES on min ||B (b - A x)|| (B as a left
    preconditioner), x_k in K_k(B A, B b).  B defaults to A^T, in which case
    x_k is the LSMR iterate.  History: ``resid`` = ||B (b - A x_k)||."""
    bproj = backprojector or op.rmatvec
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    vs, ys, res = _arnoldi_gmres(lambda x: bproj(op.matvec(x)), bproj(b), iters)
    hist = {"resid": res, "iterates": []}
    if not ys:
        return np.zeros(op.shape[1]), hist
    for y in (ys if keep_iterates else ys[-1:]):
        x = np.stack(vs[:len(y)], axis=1) @ y
        if keep_iterates:
            hist["iterates"].append(x)
    return x.copy(), hist


# ---------------------------------------------------------------- CGLS-TV (IRN)
def grad3(x):
    """D x for a volume x[k][j][i]: forward differences along i, j, k, zero in
    the last plane of each direction (Neumann boundary).  Returns (3, nz, ny, nx)."""
    d = np.zeros((3,) + x.shape)
    d[0, :, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    d[1, :, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    d[2, :-1, :, :] = x[1:, :, :] - x[:-1, :, :]
    return d


def grad3_adjoint(u):
    """D^T u, the adjoint of grad3 (a negative divergence)."""
    x = np.zeros(u.shape[1:])
    x[:, :, :-1] -= u[0, :, :, :-1]
    x[:, :, 1:] += u[0, :, :, :-1]
    x[:, :-1, :] -= u[1, :, :-1, :]
    x[:, 1:, :] += u[1, :, :-1, :]
    x[:-1, :, :] -= u[2, :-1, :, :]
    x[1:, :, :] += u[2, :-1, :, :]
    return x


def total_variation(x):
    """Isotropic 3D TV (Sec. 2.3): sum over voxels of |(D_i x, D_j x, D_k x)|."""
    d = grad3(x)
    return float(np.sum(np.sqrt(np.sum(d * d, axis=0))))


def irn_weights(x, tau):
    """IRN weights W(Dx) (Sec. 2.3): w = (|Dx|^2 + tau^2)^(-1/4) per voxel, so that
    ||W D x||^2 = sum |Dx|^2 / sqrt(|Dx|^2 + tau^2), which tends to TV(x) as tau -> 0."""
    d = grad3(x)
    return (np.sum(d * d, axis=0) + tau * tau) ** -0.25


CGLS_TV_CONVERGED = 1e-14     # inner CGLS stops once ||s|| falls below this fraction of its start


def cgls_tv(op, vol_shape, b, outer, inner, lam, tau, keep_iterates=False):
    """CGLS-TV (Sec. 2.3.1): iteratively reweighted norm.  Outer step k fixes
    the weights L = W(D x^(k)) and runs `inner` CGLS iterations on
        min ||A x - b||^2 + lam^2 ||L D x||^2,
    i.e. on the stacked system [A; lam L D] x ~ [b; 0], started from x^(k)
    (x^(0) = 0, so the first weights are uniform).  The paper prints the
    regularisation term unsquared; read squared, as in Eq. 6.  The inner CGLS
    stops early once its normal residual ||s|| has fallen to 1e-14 of its
    starting value (converged to FP64 working precision).
    History: ``resid`` = ||A x - b|| and ``objective`` = ||A x - b||^2 +
    lam^2 TV(x) after every outer step; ``iterates`` the outer iterates."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros(vol_shape)
    hist = {"resid": [], "objective": [], "iterates": []}
    for _ in range(outer):
        w = irn_weights(x, tau)
        # CGLS on the stacked operator, from x: residual r = [b - A x; -lam w D x]
        r_a = b - op.matvec(x.ravel())
        r_d = -lam * w * grad3(x)
        s = (op.rmatvec(r_a).reshape(vol_shape) + lam * grad3_adjoint(w * r_d))
        p = s.copy()
        gamma = float(np.sum(s * s))
        gamma0 = gamma
        for _ in range(inner):
            # converged to working precision: further steps would divide rounding by rounding
            if gamma <= CGLS_TV_CONVERGED * CGLS_TV_CONVERGED * gamma0:
                break
            q_a = op.matvec(p.ravel())
            q_d = lam * w * grad3(p)
            delta = float(np.dot(q_a, q_a) + np.sum(q_d * q_d))
            if delta == 0.0:
                break
            alpha = gamma / delta
            x = x + alpha * p
            r_a = r_a - alpha * q_a
            r_d = r_d - alpha * q_d
            s = op.rmatvec(r_a).reshape(vol_shape) + lam * grad3_adjoint(w * r_d)
            gamma_new = float(np.sum(s * s))
            p = s + (gamma_new / gamma) * p
            gamma = gamma_new
        res = _norm(op.matvec(x.ravel()) - b)
        hist["resid"].append(res)
        hist["objective"].append(res * res + lam * lam * total_variation(x))
        if keep_iterates:
            hist["iterates"].append(x.copy())
    return x, hist


# ------------------------------------------- explicit residuals and the stopping rule
def explicit_residual_stop(op, b, method, iters, stop_tol=0.0, **kw):
    """Run `method` ("cgls", "lsqr", "lsmr" or "hybrid_lsqr") for up to `iters`
    iterations, computing the explicit residual norm ||b - A x_k|| after every
    iteration (one extra product with A each), and stop at the first k whose
    residual exceeds (1 - stop_tol) times the previous one: the result is then
    x_{k-1} after k - 1 iterations.  stop_tol = 0 stops when the residual
    increases, which is what the paper's toolbox does (Sec. 3.1.1: an increase
    flags loss of orthogonality or accumulated rounding); stop_tol > 0 also
    stops when the decrease stalls.

    The iterates of a run do not depend on later iterations, so the stopped
    run is the unstopped run cut at k - 1.  Returns (x, hist) with hist of the
    method (cut at the returned iteration) plus ``explicit_resid`` (every
    computed ||b - A x_k||, including the one that triggered the stop) and
    ``stopped`` (True when the rule ended the run early).
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    fn = {"cgls": cgls, "lsqr": lsqr, "lsmr": lsmr, "hybrid_lsqr": hybrid_lsqr, "hybrid_lsmr": hybrid_lsmr}[method]
    x_full, h = fn(op, b, iters, keep_iterates=True, **kw)
    its = h["iterates"]
    resid = []
    done = len(its)
    stopped = False
    for k, xk in enumerate(its, start=1):
        resid.append(_norm(b - op.matvec(xk)))
        if k > 1 and resid[-1] > (1.0 - stop_tol) * resid[-2]:
            done = k - 1
            stopped = True
            break
    x = its[done - 1].copy() if done > 0 else np.zeros(op.shape[1])
    out = {key: (val[:done] if isinstance(val, list) and key not in ("beta", "alpha") else val)
           for key, val in h.items()}
    out["iterates"] = its[:done]
    out["explicit_resid"] = resid
    out["stopped"] = stopped
    return x, out


# ------------------------------------------------------------ dense Krylov reference
def krylov_basis(a, b, k):
    """Orthonormal basis (columns) of K_k(A^T A, A^T b), Arnoldi with full
    re-orthogonalisation (two passes of classical Gram-Schmidt), dense FP64."""
    a = np.asarray(a, dtype=np.float64)
    ata = a.T @ a
    q = a.T @ np.asarray(b, dtype=np.float64).reshape(-1)
    basis = [q / np.linalg.norm(q)]
    for _ in range(1, k):
        w = ata @ basis[-1]
        for _pass in range(2):
            for qj in basis:
                w = w - np.dot(qj, w) * qj
        basis.append(w / np.linalg.norm(w))
    return np.stack(basis, axis=1)


def krylov_reference(a, b, k, method, damp=0.0):
    """x_k by its defining minimisation over K_k (dense, for pinning the recurrences).

    method "lsqr"/"cgls": argmin ||[A; lam I] x - [b; 0]|| over K_k (Eqs. 3-4, 7);
    method "lsmr": argmin ||A^T b - (A^T A + lam^2 I) x|| over K_k (Eq. 5, 7).
    K_k(A^T A + lam^2 I, A^T b) = K_k(A^T A, A^T b) (shift invariance, Sec. 2.2.1).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    v = krylov_basis(a, b, k)
    lam2 = float(damp) ** 2
    if method in ("lsqr", "cgls"):
        aug = np.vstack([a @ v, math.sqrt(lam2) * v])
        rhs = np.concatenate([b, np.zeros(v.shape[0])])
        y = np.linalg.lstsq(aug, rhs, rcond=None)[0]
    elif method == "lsmr":
        n_op = a.T @ (a @ v) + lam2 * v
        y = np.linalg.lstsq(n_op, a.T @ b, rcond=None)[0]
    else:
        raise ValueError(method)
    return v @ y
