// Projected Tikhonov solve of hybrid LSQR (Sec. 2.2.1, Eq. 8) with the GCV
// parameter choice (Sec. 2.2.2), in FP64 on one thread block.  With
// lsmr_proj the projected problem is LSMR's instead (hybrid LSMR, the
// generalisation Sec. 2.2.2 mentions): matrix Hbar_k = [H_k^T H_k ;
// alpha_{k+1} beta_{k+1} e_k^T] and right-hand side alpha_1 beta_1 e_1, so that
// x_k minimises ||A^T (b - A x)||^2 + lambda^2 ||x||^2 over the Krylov space.
//
// At iteration k the Golub-Kahan process has produced the (k+1) x k lower
// bidiagonal H_k (H[i][i] = alpha_{i+1}, H[i+1][i] = beta_{i+2}).  This kernel
//   1. computes the SVD H_k = P Sigma Q^T by one-sided (Hestenes) Jacobi
//      rotations of the columns of H_k (round-robin pair order, one warp per
//      pair), accumulating Q;
//   2. obtains the first row of P: P[0][i] = (H Q)[0][i] / sigma_i for the k
//      singular vectors and, for the (k+1)-th, 1/||z|| with z the null vector
//      of H_k^T (z_0 = 1, z_{i+1} = -alpha_{i+1} z_i / beta_{i+2});
//   3. picks lambda_k: fixed; or the minimiser of
//         G(lam) = ||(I - H H^+_lam) beta_1 e_1||^2 / (trace(I - H H^+_lam))^2,
//      H^+_lam = (H^T H + lam^2 I)^{-1} H^T, evaluated from the SVD; the
//      minimiser is taken on a 200-point log grid over [sigma_max 1e-8,
//      sigma_max] (ties to the larger lambda) and refined by golden-section
//      search in log lambda on the neighbouring bracket to 1e-10; or (the
//      discrepancy principle) the root of ||beta_1 e_1 - H y_lam|| = nl beta_1,
//      the projected form of ||b - A x_lam|| = nl ||b||, by bisection in
//      log lambda over sigma_max [1e-8, 1e8] to 1e-10 (0 if even the
//      smallest lambda leaves the residual above the target, the upper end if
//      the largest stays below it);
//   4. forms y_k = sum_i q_i beta_1 (H Q)[0][i] / (sigma_i^2 + lam^2) and the
//      coefficients of the stored basis vectors, x_k = sum_j coef_j V_j.
#include <cfloat>
#include <cmath>

#include "solver_common.cuh"

namespace cbct {

constexpr int PS_THREADS = 256, PS_WARPS = PS_THREADS / 32;
constexpr int GCV_POINTS = 200;
constexpr double GCV_DECADES = 8.0, GCV_TOL = 1e-10;
constexpr int JACOBI_SWEEPS = 40;

__device__ double gcv_value(const double *sig, const double *p1, int k, double beta1, double lam) {
    const double l2 = lam * lam;
    double num = 0.0, filt = 0.0;
    for (int i = 0; i < k; ++i) {
        const double s2 = sig[i] * sig[i];
        const double f = l2 / (s2 + l2);
        const double t = f * beta1 * p1[i];
        num += t * t;
        filt += s2 / (s2 + l2);
    }
    const double tail = beta1 * p1[k];
    num += tail * tail;
    const double den = (double)(k + 1) - filt;
    return num / (den * den);
}

// ||beta_1 e_1 - H y_lam|| from the SVD (the GCV numerator, square-rooted).
__device__ double projected_residual(const double *sig, const double *p1, int k, double beta1, double lam) {
    const double l2 = lam * lam;
    double num = 0.0;
    for (int i = 0; i < k; ++i) {
        const double s2 = sig[i] * sig[i];
        const double f = (s2 + l2) > 0.0 ? l2 / (s2 + l2) : 1.0;
        const double t = f * beta1 * p1[i];
        num += t * t;
    }
    num += (beta1 * p1[k]) * (beta1 * p1[k]);
    return sqrt(num);
}

constexpr double DP_DECADES = 8.0, DP_TOL = 1e-10;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(PS_THREADS)
projected_solve_kernel(const double *__restrict__ alphas, const double *__restrict__ betas,
                       const double *__restrict__ scales, const int *iter_ptr, const int *stop, int rule,
                       double lambda_fixed, double noise_level, int lsmr_proj, double *work, int kmax,
                       double *coef, double *hist_lambda, double *hist_resid) {
    __shared__ int rotated;
    __shared__ double gvals[GCV_POINTS];
    __shared__ double lam_sh;
    if (*stop) return;
    const int k = *iter_ptr;
    if (k < 1 || k > kmax) return;
    const int rows = k + 1;
    double *B = work;                 // column-major (k+1) x k, column j at B + j*rows
    double *Q = B + (size_t)rows * k; // column-major k x k
    double *sig = Q + (size_t)k * k;  // k
    double *p1 = sig + k;             // k + 1
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // right-hand side beta1 e_1 of the projected problem
    const double beta1 = lsmr_proj ? alphas[0] * betas[0] : betas[0];

    for (int q = tid; q < rows * k; q += PS_THREADS) {
        const int c = q / rows, r = q % rows;
        if (!lsmr_proj) {
            B[q] = r == c ? alphas[c] : (r == c + 1 ? betas[c + 1] : 0.0);
        } else if (r < k) {               // (H^T H)[r][c]: tridiagonal
            double v = 0.0;
            if (r == c) v = alphas[c] * alphas[c] + betas[c + 1] * betas[c + 1];
            else if (r == c + 1) v = betas[c + 1] * alphas[c + 1];
            else if (c == r + 1) v = betas[r + 1] * alphas[r + 1];
            B[q] = v;
        } else {                          // last row: alpha_{k+1} beta_{k+1} e_k^T
            B[q] = c == k - 1 ? alphas[k] * betas[k] : 0.0;
        }
    }
    for (int q = tid; q < k * k; q += PS_THREADS) Q[q] = (q / k == q % k) ? 1.0 : 0.0;
    __syncthreads();

    // one-sided Jacobi: orthogonalise the columns of B, Q accumulates the rotations
    const int K = k + (k & 1);
    for (int sweep = 0; sweep < JACOBI_SWEEPS; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int pairing = 0; pairing < K - 1; ++pairing) {
            for (int pi = warp; pi < K / 2; pi += PS_WARPS) {
                int p, q;
                if (pi == 0) { p = K - 1; q = pairing; }
                else { p = (pairing + pi) % (K - 1); q = (pairing - pi + K - 1) % (K - 1); }
                if (p >= k || q >= k) continue;
                if (p > q) { const int t = p; p = q; q = t; }
                double *bp = B + (size_t)p * rows, *bq = B + (size_t)q * rows;
                double a = 0.0, b = 0.0, c = 0.0;
                for (int r = lane; r < rows; r += 32) {
                    a += bp[r] * bp[r];
                    b += bq[r] * bq[r];
                    c += bp[r] * bq[r];
                }
                a = warp_sum(a);
                b = warp_sum(b);
                c = warp_sum(c);
                if (c == 0.0 || !(fabs(c) > 1e-15 * sqrt(a * b))) continue;
                const double zeta = (b - a) / (2.0 * c);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int r = lane; r < rows; r += 32) {
                    const double x = bp[r], y = bq[r];
                    bp[r] = cs * x - sn * y;
                    bq[r] = sn * x + cs * y;
                }
                double *qp = Q + (size_t)p * k, *qq = Q + (size_t)q * k;
                for (int r = lane; r < k; r += 32) {
                    const double x = qp[r], y = qq[r];
                    qp[r] = cs * x - sn * y;
                    qq[r] = sn * x + cs * y;
                }
                if (lane == 0) rotated = 1;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }

    // singular values and the first row of P
    for (int j = warp; j < k; j += PS_WARPS) {
        const double *bj = B + (size_t)j * rows;
        double s = 0.0;
        for (int r = lane; r < rows; r += 32) s += bj[r] * bj[r];
        s = sqrt(warp_sum(s));
        if (lane == 0) {
            sig[j] = s;
            p1[j] = s > 0.0 ? bj[0] / s : 0.0;
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (!lsmr_proj) {
            // null vector of H_k^T, rescaled on the fly; p1[k] = z_0 / ||z||
            double z = 1.0, z0 = 1.0, ss = 1.0;
            for (int i = 0; i < k; ++i) {
                z = -alphas[i] * z / betas[i + 1];
                ss += z * z;
                if (ss > 1e200) { z *= 1e-100; z0 *= 1e-100; ss *= 1e-200; }
            }
            p1[k] = z0 / sqrt(ss);
        } else {
            // the first row of the orthogonal P has unit norm: its last entry is
            // the part of e_1 outside the range of Hbar_k
            double ss = 0.0;
            for (int i = 0; i < k; ++i) ss += p1[i] * p1[i];
            p1[k] = sqrt(fmax(0.0, 1.0 - ss));
        }
    }
    __syncthreads();

    // lambda_k
    if (rule == CBCT_LAMBDA_FIXED) {
        if (tid == 0) lam_sh = lambda_fixed;
    } else if (rule == CBCT_LAMBDA_DP) {
        if (tid == 0) {
            double smax = 0.0;
            for (int i = 0; i < k; ++i) smax = fmax(smax, sig[i]);
            const double target = noise_level * beta1;
            double lam = 0.0;
            if (smax > 0.0) {
                double lo = log(smax) - DP_DECADES * log(10.0), hi = log(smax) + DP_DECADES * log(10.0);
                if (projected_residual(sig, p1, k, beta1, exp(lo)) >= target) {
                    lam = 0.0;
                } else if (projected_residual(sig, p1, k, beta1, exp(hi)) <= target) {
                    lam = exp(hi);
                } else {
                    while (hi - lo > DP_TOL) {
                        const double mid = 0.5 * (lo + hi);
                        if (projected_residual(sig, p1, k, beta1, exp(mid)) < target) lo = mid;
                        else hi = mid;
                    }
                    lam = exp(0.5 * (lo + hi));
                }
            }
            lam_sh = lam;
        }
    } else {
        double smax = 0.0;
        for (int i = 0; i < k; ++i) smax = fmax(smax, sig[i]);
        const double hi = log(smax), lo = hi - GCV_DECADES * log(10.0);
        for (int i = tid; i < GCV_POINTS; i += PS_THREADS)
            gvals[i] = gcv_value(sig, p1, k, beta1, exp(lo + (hi - lo) * i / (GCV_POINTS - 1)));
        __syncthreads();
        if (tid == 0) {
            int best = 0;
            for (int i = 1; i < GCV_POINTS; ++i)
                if (gvals[i] <= gvals[best]) best = i;
            auto grid = [&](int i) { return lo + (hi - lo) * i / (GCV_POINTS - 1); };
            double a = grid(max(best - 1, 0)), c = grid(min(best + 1, GCV_POINTS - 1));
            const double invphi = (sqrt(5.0) - 1.0) / 2.0;
            double x1 = c - invphi * (c - a), x2 = a + invphi * (c - a);
            double f1 = gcv_value(sig, p1, k, beta1, exp(x1)), f2 = gcv_value(sig, p1, k, beta1, exp(x2));
            while (c - a > GCV_TOL) {
                if (f1 < f2) {
                    c = x2; x2 = x1; f2 = f1;
                    x1 = c - invphi * (c - a);
                    f1 = gcv_value(sig, p1, k, beta1, exp(x1));
                } else {
                    a = x1; x1 = x2; f1 = f2;
                    x2 = a + invphi * (c - a);
                    f2 = gcv_value(sig, p1, k, beta1, exp(x2));
                }
            }
            double t = 0.5 * (a + c);
            if (gcv_value(sig, p1, k, beta1, exp(t)) > gvals[best]) t = grid(best);
            lam_sh = smax > 0.0 ? exp(t) : 0.0;
        }
    }
    __syncthreads();
    const double lam = lam_sh, l2 = lam * lam;

    // y_k and basis coefficients: x_k = sum_j y_j v_{j+1}, v_{j+1} = V_j / (scale_j alpha_{j+1})
    for (int j = tid; j < k; j += PS_THREADS) {
        double y = 0.0;
        for (int i = 0; i < k; ++i) {
            const double s2 = sig[i] * sig[i];
            const double d = s2 + l2;
            if (d > 0.0) y += Q[(size_t)i * k + j] * beta1 * B[(size_t)i * rows] / d;
        }
        coef[j] = y / (scales[j] * alphas[j]);
    }
    if (tid == 0) {
        hist_lambda[k - 1] = lam;
        hist_resid[k - 1] = projected_residual(sig, p1, k, beta1, lam);
    }
}

cbct_status launch_projected_solve(const double *alphas, const double *betas, const double *scales,
                                   const int *iter, const int *stop, int rule, double lambda_fixed,
                                   double noise_level, int lsmr_proj, double *work, int kmax, double *coef,
                                   double *hist_lambda, double *hist_resid, cudaStream_t s) {
    projected_solve_kernel<<<1, PS_THREADS, 0, s>>>(alphas, betas, scales, iter, stop, rule, lambda_fixed,
                                                     noise_level, lsmr_proj, work, kmax, coef, hist_lambda,
                                                     hist_resid);
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

}  // namespace cbct
