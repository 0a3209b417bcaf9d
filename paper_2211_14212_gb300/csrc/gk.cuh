// Golub-Kahan state and recurrences shared by the single-problem solvers
// (solvers.cu) and the multi-problem server (serve.cu): the FP64 scalar steps
// of LSQR (Sec. 2.1.2) and LSMR (Sec. 2.1.3), as device functions with
// single-block kernel wrappers, and the fused vector updates.
#pragma once

#include "solver_common.cuh"

namespace cbct {

// ===================================================================== LSQR / LSMR
//
// Golub-Kahan bidiagonalisation (Sec. 2.1.2):
//   beta_1 u_1 = b,  alpha_1 v_1 = A^T u_1,
//   beta_{i+1} u_{i+1} = A v_i - alpha_i u_i,
//   alpha_{i+1} v_{i+1} = A^T u_{i+1} - beta_{i+1} v_i.

struct GkState {
    // bidiagonalisation
    double alpha, beta;          // current alpha_i, beta_i (true values)
    double su, sv;               // storage scales of U and V
    double su_next, sv_next;     // scales chosen for the next U / V
    double fa, fb;               // forward epilogue:  U <- fa * A V + fb * U
    double ba, bb;               // backward epilogue: V <- ba * A^T U + bb * V
    double c0;                   // U = c0 * b at the start; later the first update coefficient
    double damp;                 // Tikhonov lambda
    double sqrt_n, sqrt_m;
    // LSQR
    double rhobar, phibar, psisq;
    // LSMR
    double alphabar, zetabar, rho, rhobar_m, cbar, sbar;
    double betadd, betad, rhod, tautilde, thetatilde, zeta, dsum;
    // vector update coefficients
    double k1, k2, k3, k4;
    int iter, stop, status, scaled;
};

enum Method { M_LSQR = 0, M_LSMR = 1, M_HYBRID = 2 };

// After ||b||^2: beta_1, the scale of U and the first backprojection's coefficients.
__device__ __forceinline__ void gk_begin_step(GkState *st, double ss) {
    const double beta = sqrt(ss);
    st->iter = 0;
    st->status = CBCT_OK;
    st->stop = 0;
    if (!good(beta)) {                          // b = 0: x = 0 is the solution
        st->stop = 1;
        st->status = beta == 0.0 ? CBCT_OK : CBCT_EBREAKDOWN;
        return;
    }
    st->beta = beta;
    st->su = storage_scale(st->scaled, st->sqrt_n, beta);
    st->c0 = st->su;
    st->sv_next = 1.0;
    st->ba = st->sv_next / (st->su * beta);
    st->bb = 0.0;
}

// After A^T u_1: alpha_1, start values of the method's recurrences.
__device__ __forceinline__ void gk_begin2_step(GkState *st, double ss, int method) {
    const double alpha = sqrt(ss) / st->sv_next;
    if (!good(alpha)) {                         // A^T b = 0: x = 0 is the least-squares solution
        st->stop = 1;
        st->status = alpha == 0.0 ? CBCT_OK : CBCT_EBREAKDOWN;
        return;
    }
    st->sv = st->sv_next;
    st->alpha = alpha;
    st->c0 = 1.0 / (st->sv * alpha);            // w_1 = v_1 (LSQR), h_1 = v_1 (LSMR)
    if (method == M_LSQR) {
        st->rhobar = alpha;
        st->phibar = st->beta;
        st->psisq = 0.0;
    } else if (method == M_LSMR) {
        st->alphabar = alpha;
        st->zetabar = alpha * st->beta;
        st->rho = 1.0;
        st->rhobar_m = 1.0;
        st->cbar = 1.0;
        st->sbar = 0.0;
        st->betadd = st->beta;
        st->betad = 0.0;
        st->rhod = 1.0;
        st->tautilde = 0.0;
        st->thetatilde = 0.0;
        st->zeta = 0.0;
        st->dsum = 0.0;
    }
    st->su_next = storage_scale(st->scaled, st->sqrt_n, st->beta);
    st->fa = st->su_next / (st->sv * st->alpha);
    st->fb = -st->su_next * st->alpha / (st->su * st->beta);
}

// After U <- A v_i - alpha_i u_i: beta_{i+1} and the backprojection's coefficients.
__device__ __forceinline__ void gk_after_forward_step(GkState *st, double ss, double *beta_arr) {
    const double beta = sqrt(ss) / st->su_next;
    if (!good(beta)) {
        st->stop = 1;
        st->status = CBCT_EBREAKDOWN;
        return;
    }
    st->su = st->su_next;
    st->beta = beta;
    if (beta_arr) beta_arr[st->iter + 1] = beta;
    st->sv_next = storage_scale(st->scaled, st->sqrt_m, st->alpha);
    st->ba = st->sv_next / (st->su * beta);
    st->bb = -st->sv_next * beta / (st->sv * st->alpha);
}

// After V <- A^T u_{i+1} - beta_{i+1} v_i: alpha_{i+1}, the method's rotations,
// the vector-update coefficients and the next forward's coefficients.
__device__ __forceinline__ void gk_after_backward_step(GkState *st, double ss, int method, double *hist_r,
                                                       double *hist_n, double *alpha_arr, double *scale_arr,
                                                       int cap) {
    const double alpha = sqrt(ss) / st->sv_next;
    if (!good(alpha)) {
        st->stop = 1;
        st->status = CBCT_EBREAKDOWN;
        return;
    }
    const double beta = st->beta;
    const int it = st->iter;
    if (method == M_LSQR) {
        // rotation eliminating the damping, then the one eliminating beta_{i+1}
        const Rot r1 = givens(st->rhobar, st->damp);
        const double psi = r1.s * st->phibar;
        const double phibar1 = r1.c * st->phibar;
        st->psisq += psi * psi;
        const Rot r2 = givens(r1.r, beta);
        const double theta = r2.s * alpha;
        st->rhobar = -r2.c * alpha;
        const double phi = r2.c * phibar1;
        st->phibar = r2.s * phibar1;
        st->k1 = phi / r2.r;                        // x += k1 w
        st->k2 = 1.0 / (st->sv_next * alpha);       // w = k2 V + k3 w
        st->k3 = -theta / r2.r;
        if (it < cap) {
            hist_r[it] = sqrt(st->phibar * st->phibar + st->psisq);
            hist_n[it] = fabs(st->phibar * alpha * r2.c);
        }
    } else if (method == M_LSMR) {
        const Rot rh = givens(st->alphabar, st->damp);        // P-hat_k
        const double rho_prev = st->rho;
        const Rot rk = givens(rh.r, beta);                     // P_k
        const double theta_next = rk.s * alpha;
        st->alphabar = rk.c * alpha;
        st->rho = rk.r;
        const double rhobar_prev = st->rhobar_m;               // P-bar_k
        const double zeta_prev = st->zeta;
        const double thetabar = st->sbar * rk.r;
        const Rot rb = givens(st->cbar * rk.r, theta_next);
        st->cbar = rb.c;
        st->sbar = rb.s;
        st->rhobar_m = rb.r;
        st->zeta = rb.c * st->zetabar;
        st->zetabar = -rb.s * st->zetabar;
        st->k1 = thetabar * rk.r / (rho_prev * rhobar_prev);  // hbar = h - k1 hbar
        st->k2 = st->zeta / (rk.r * rb.r);                    // x += k2 hbar
        st->k3 = 1.0 / (st->sv_next * alpha);                 // h = k3 V + k4 h
        st->k4 = -theta_next / rk.r;
        // ||r_k|| estimate: rotations Q-hat_k, Q_k applied to (beta-double-dot, 0), then Q-tilde_{k-1}
        const double betaacute = rh.c * st->betadd;
        const double betacheck = -rh.s * st->betadd;
        const double betahat = rk.c * betaacute;
        st->betadd = -rk.s * betaacute;
        const double thetatilde_prev = st->thetatilde;
        const Rot rt = givens(st->rhod, thetabar);
        st->thetatilde = rt.s * rb.r;
        st->rhod = rt.c * rb.r;
        st->betad = -rt.s * st->betad + rt.c * betahat;
        st->tautilde = (zeta_prev - thetatilde_prev * st->tautilde) / rt.r;
        const double taud = (st->zeta - st->thetatilde * st->tautilde) / st->rhod;
        st->dsum += betacheck * betacheck;
        if (it < cap) {
            hist_r[it] = sqrt(st->dsum + (st->betad - taud) * (st->betad - taud) + st->betadd * st->betadd);
            hist_n[it] = fabs(st->zetabar);
        }
    }
    if (alpha_arr) alpha_arr[it + 1] = alpha;
    if (scale_arr) scale_arr[it + 1] = st->sv_next;
    st->sv = st->sv_next;
    st->alpha = alpha;
    st->iter = it + 1;
    st->su_next = storage_scale(st->scaled, st->sqrt_n, beta);
    st->fa = st->su_next / (st->sv * alpha);
    st->fb = -st->su_next * alpha / (st->su * beta);
}

// out = c * V (storage -> FP32); optionally zero a second vector.
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_start_dirs(const T *__restrict__ V, float *__restrict__ w, float *__restrict__ zero1,
             float *__restrict__ zero2, int64_t n, const GkState *st) {
    if (st->stop) return;
    const float c = (float)st->c0;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        w[i] = c * Storage<T>::ld_plain(V + i);
        if (zero1) zero1[i] = 0.0f;
        if (zero2) zero2[i] = 0.0f;
    }
}

// Single-block wrappers: fixed-order reduction of the partial sums, then the
// scalar step in thread 0.
static __global__ void __launch_bounds__(RED_THREADS) gk_begin(GkState *st, const double *part, int np) {
    __shared__ double red[RED_THREADS / 32];
    const double ss = reduce_partials(part, np, red);
    if (threadIdx.x == 0) gk_begin_step(st, ss);
}

static __global__ void __launch_bounds__(RED_THREADS) gk_begin2(GkState *st, const double *part, int np,
                                                                int method) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop) return;
    const double ss = reduce_partials(part, np, red);
    if (threadIdx.x == 0) gk_begin2_step(st, ss, method);
}

static __global__ void __launch_bounds__(RED_THREADS) gk_after_forward(GkState *st, const double *part, int np,
                                                                       double *beta_arr) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop) return;
    const double ss = reduce_partials(part, np, red);
    if (threadIdx.x == 0) gk_after_forward_step(st, ss, beta_arr);
}

static __global__ void __launch_bounds__(RED_THREADS) gk_after_backward(GkState *st, const double *part, int np,
                                                                        int method, double *hist_r,
                                                                        double *hist_n, double *alpha_arr,
                                                                        double *scale_arr, int cap) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop) return;
    const double ss = reduce_partials(part, np, red);
    if (threadIdx.x == 0) gk_after_backward_step(st, ss, method, hist_r, hist_n, alpha_arr, scale_arr, cap);
}

// LSQR element update: x += k1 w; w = k2 v + k3 w.
__device__ __forceinline__ void lsqr_elem(float v, float &x, float &w, float k1, float k2, float k3) {
    const float wi = w;
    x = fmaf(k1, wi, x);
    w = fmaf(k2, v, k3 * wi);
}

// LSMR element update: hbar = h - k1 hbar; x += k2 hbar; h = k3 v + k4 h.
__device__ __forceinline__ void lsmr_elem(float v, float &x, float &h, float &hbar, float k1, float k2, float k3,
                                          float k4) {
    const float hi = h;
    const float hb = fmaf(-k1, hbar, hi);
    hbar = hb;
    x = fmaf(k2, hb, x);
    h = fmaf(k3, v, k4 * hi);
}

// LSQR: x += (phi/rho) w; w = v_{i+1} - (theta/rho) w.
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_lsqr_update(const T *__restrict__ V, float *__restrict__ x, float *__restrict__ w, int64_t n, const GkState *st) {
    if (st->stop) return;
    const float k1 = (float)st->k1, k2 = (float)st->k2, k3 = (float)st->k3;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS)
        lsqr_elem(Storage<T>::ld_plain(V + i), x[i], w[i], k1, k2, k3);
}

// LSMR: hbar = h - k1 hbar; x += k2 hbar; h = v_{k+1} - (theta/rho) h.
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_lsmr_update(const T *__restrict__ V, float *__restrict__ x, float *__restrict__ h, float *__restrict__ hbar,
              int64_t n, const GkState *st) {
    if (st->stop) return;
    const float k1 = (float)st->k1, k2 = (float)st->k2, k3 = (float)st->k3, k4 = (float)st->k4;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS)
        lsmr_elem(Storage<T>::ld_plain(V + i), x[i], h[i], hbar[i], k1, k2, k3, k4);
}

}  // namespace cbct
