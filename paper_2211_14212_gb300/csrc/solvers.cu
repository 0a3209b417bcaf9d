// Krylov least-squares solvers on the GPU: CGLS (Sec. 2.1.1), LSQR (Sec. 2.1.2),
// LSMR (Sec. 2.1.3), all optionally damped by a Tikhonov lambda (Sec. 2.2,
// Eqs. 6-7), and hybrid LSQR with a per-iteration lambda_k (Sec. 2.2.1-2.2.2).
//
// Vectors live on the device in FP32 (x and the search directions) or in the
// chosen storage type (the Golub-Kahan vectors u, v and the basis V_k).  All
// scalars (norms, rotations, coefficients) are FP64 and are produced by
// single-block "finalize" kernels that reduce per-block partial sums in a fixed
// order.  Nothing returns to the host inside the iteration loop, so one
// iteration can be captured as a CUDA graph and replayed.
//
// Golub-Kahan vectors are stored unnormalised and, for FP16, multiplied by a
// power-of-two scale: U = su * beta_i u_i and V = sv * alpha_i v_i.  The scale
// factors and norms enter the coefficients of the next fused epilogue, so no
// separate normalisation pass over the vectors is needed.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "gk.cuh"
#include "solver_common.cuh"

namespace cbct {

cbct_status launch_projected_solve(const double *alphas, const double *betas, const double *scales,
                                   const int *iter, const int *stop, int rule, double lambda_fixed,
                                   double noise_level, int lsmr_proj, double *work, int kmax, double *coef,
                                   double *hist_lambda, double *hist_resid, cudaStream_t s);

// ================================================== explicit residual monitor
//
// With opts->explicit_residual, every iteration ends with r = b - A x_k (one
// forward launch whose epilogue forms b - A x and the per-block partials of
// ||r||^2) and a single-block check: record ||r||; if it exceeds
// (1 - stop_tol) times the previous value, set the method's stop flag (every
// later launch of the solve then does nothing) and mark the run as stopped by
// the rule.  x_{k-1} is kept in `xprev` (copied before each x update) and
// restored at the end.  The paper's toolbox stops on an increase of this
// explicit residual (Sec. 3.1.1).

struct ExplicitState {
    double prev;
    int count, stopped;
};

__global__ void __launch_bounds__(RED_THREADS)
k_explicit_check(const double *part, int np, ExplicitState *es, int *stop, double *hist, int cap, double tol) {
    __shared__ double red[RED_THREADS / 32];
    if (*stop) return;
    const double rr = sqrt(reduce_partials(part, np, red));
    if (threadIdx.x) return;
    const int c = es->count;
    if (c < cap) hist[c] = rr;
    es->count = c + 1;
    if (c > 0 && !(rr <= (1.0 - tol) * es->prev)) {     // increase, stall, or not finite
        *stop = 1;
        es->stopped = 1;
    }
    es->prev = rr;
}

__global__ void __launch_bounds__(VEC_THREADS)
k_copy_running(const float *__restrict__ src, float *__restrict__ dst, int64_t n, const int *stop) {
    if (*stop) return;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS)
        dst[i] = src[i];
}

// Buffers and launches of the monitor; inactive (no allocation, no launches)
// unless opts->explicit_residual.
struct ExplicitMonitor {
    bool on = false;
    float *r = nullptr, *xprev = nullptr;
    double *part = nullptr, *hist = nullptr;
    ExplicitState *es = nullptr;
    int nf = 0, cap = 0;
    double tol = 0.0;

    cbct_status init(const cbct_solve_opts *o, const DevGeom &g, int64_t n, int64_t m, Workspace &ws) {
        on = o->explicit_residual != 0;
        if (!on) return CBCT_OK;
        tol = o->stop_tol;
        cap = o->iters;
        nf = forward_num_partials(g);
        CBCT_CUDA_TRY(ws.alloc(&r, (size_t)n));
        CBCT_CUDA_TRY(ws.alloc(&xprev, (size_t)m));
        CBCT_CUDA_TRY(ws.alloc(&part, (size_t)nf));
        CBCT_CUDA_TRY(ws.alloc(&hist, (size_t)cap));
        CBCT_CUDA_TRY(ws.alloc(&es, 1));
        CBCT_CUDA_TRY(cudaMemsetAsync(es, 0, sizeof(ExplicitState), ws.s));
        CBCT_CUDA_TRY(cudaMemsetAsync(xprev, 0, sizeof(float) * m, ws.s));     // x_0 = 0
        return CBCT_OK;
    }
    // before the x update of an iteration
    void keep(const float *x, int64_t m, const int *stop, cudaStream_t s, Tracker &tr) {
        if (!on) return;
        k_copy_running<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(x, xprev, m, stop);
        ++tr.launches;
    }
    // after the x update: r = b - A x, the check
    template <typename Fwd>
    cbct_status check(Fwd &&fwd32, const float *x, const float *b_vfast, int *stop, cudaStream_t s, Tracker &tr) {
        if (!on) return CBCT_OK;
        const Epilogue e{nullptr, nullptr, -1.0, 1.0, part, stop, b_vfast};
        cbct_status st = fwd32(x, r, e);
        if (st != CBCT_OK) return st;
        k_explicit_check<<<1, RED_THREADS, 0, s>>>(part, nf, es, stop, hist, cap, tol);
        ++tr.launches;
        CBCT_CUDA_TRY(cudaGetLastError());
        return CBCT_OK;
    }
    // after the loop: restore x_{k-1} if the rule stopped the run, fill the report
    cbct_status finish(float *x, int64_t m, cudaStream_t s, cbct_solve_report *rep, int *iters_done) {
        if (!on) {
            if (rep) { rep->explicit_count = 0; rep->stopped_on_residual = 0; }
            return CBCT_OK;
        }
        ExplicitState h;
        CBCT_CUDA_TRY(cudaMemcpyAsync(&h, es, sizeof h, cudaMemcpyDeviceToHost, s));
        std::vector<double> hv((size_t)cap);
        CBCT_CUDA_TRY(cudaMemcpyAsync(hv.data(), hist, sizeof(double) * cap, cudaMemcpyDeviceToHost, s));
        CBCT_CUDA_TRY(cudaStreamSynchronize(s));
        if (h.stopped) {
            CBCT_CUDA_TRY(cudaMemcpyAsync(x, xprev, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
            *iters_done = h.count - 1;
        }
        if (rep) {
            const int c = std::min(h.count, cap);
            if (rep->explicit_resid_norm) std::memcpy(rep->explicit_resid_norm, hv.data(), sizeof(double) * c);
            rep->explicit_count = c;
            rep->stopped_on_residual = h.stopped;
        }
        return CBCT_OK;
    }
};

// ============================================ re-orthogonalised Golub-Kahan
//
// With opts->reorth, every new u and v is re-orthogonalised against all
// earlier (normalised, stored) ones by classical Gram-Schmidt applied twice
// with FP64 dot products, before its norm is taken; the norm partials of the
// fused epilogue are then replaced by fresh ones.  The number of stored
// vectors is read from the device state (st->iter + 1), so an iteration can
// still be captured once as a CUDA graph.

constexpr int RO_CHUNK = 8;

// partial[i * VEC_BLOCKS + block] = block share of w . Q_i, i < *iter + 1
__global__ void __launch_bounds__(VEC_THREADS)
k_ro_dot(const float *__restrict__ w, const float *__restrict__ Q, int64_t n, const GkState *st, double *partial) {
    __shared__ double red[VEC_THREADS / 32];
    if (st->stop) return;
    const int count = st->iter + 1;
    for (int c0 = 0; c0 < count; c0 += RO_CHUNK) {
        const int nc = min(RO_CHUNK, count - c0);
        double acc[RO_CHUNK];
#pragma unroll
        for (int q = 0; q < RO_CHUNK; ++q) acc[q] = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n;
             e += (int64_t)VEC_BLOCKS * VEC_THREADS) {
            const double we = w[e];
#pragma unroll
            for (int q = 0; q < RO_CHUNK; ++q)
                if (q < nc) acc[q] += we * (double)Q[(size_t)(c0 + q) * n + e];
        }
#pragma unroll
        for (int q = 0; q < RO_CHUNK; ++q) {
            if (q >= nc) break;
            const double sum = block_sum<VEC_THREADS>(acc[q], red);
            if (threadIdx.x == 0) partial[(size_t)(c0 + q) * VEC_BLOCKS + blockIdx.x] = sum;
        }
    }
}

// d[i] = sum of the partials of dot i (one block per possible dot; the extra blocks idle)
__global__ void __launch_bounds__(RED_THREADS) k_ro_reduce(const double *partial, const GkState *st, double *d) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop || (int)blockIdx.x > st->iter) return;
    const double sum = reduce_partials(partial + (size_t)blockIdx.x * VEC_BLOCKS, VEC_BLOCKS, red);
    if (threadIdx.x == 0) d[blockIdx.x] = sum;
}

// w -= sum_i d_i Q_i (FP64 correction)
__global__ void __launch_bounds__(VEC_THREADS)
k_ro_sub(float *__restrict__ w, const float *__restrict__ Q, const double *__restrict__ d, int64_t n, const GkState *st) {
    if (st->stop) return;
    const int count = st->iter + 1;
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        double corr = 0.0;
        for (int i = 0; i < count; ++i) corr += d[i] * (double)Q[(size_t)i * n + e];
        w[e] = (float)((double)w[e] - corr);
    }
}

// Q_{*iter + 1 + off} = w / (scale * norm): u_{i+2} = U / (su beta), v_{i+2} = V / (sv alpha)
__global__ void __launch_bounds__(VEC_THREADS)
k_ro_store(const float *__restrict__ w, float *__restrict__ Q, int64_t n, const GkState *st, int which, int off) {
    if (st->stop) return;
    const double c = which == 0 ? 1.0 / (st->su * st->beta) : 1.0 / (st->sv * st->alpha);
    float *dst = Q + (size_t)(st->iter + off) * n;
    const float cf = (float)c;
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS)
        dst[e] = w[e] * cf;
}

struct Reorth {
    bool on = false;
    float *Ub = nullptr, *Vb = nullptr;
    double *partial = nullptr, *d = nullptr;
    int cap = 0;

    cbct_status init(const cbct_solve_opts *o, int64_t n, int64_t m, Workspace &ws) {
        on = o->reorth != 0;
        if (!on) return CBCT_OK;
        cap = o->iters + 1;
        CBCT_CUDA_TRY(ws.alloc(&Ub, (size_t)cap * n));
        CBCT_CUDA_TRY(ws.alloc(&Vb, (size_t)cap * m));
        CBCT_CUDA_TRY(cudaMemsetAsync(Vb, 0, sizeof(float) * cap * m, ws.s));
        CBCT_CUDA_TRY(ws.alloc(&partial, (size_t)cap * VEC_BLOCKS));
        CBCT_CUDA_TRY(ws.alloc(&d, (size_t)cap));
        return CBCT_OK;
    }
    // two classical Gram-Schmidt passes of w against Q_0 .. Q_{iter}
    void orthogonalise(float *w, const float *Q, int64_t n, const GkState *st, cudaStream_t s, Tracker &tr) {
        for (int pass = 0; pass < 2; ++pass) {
            k_ro_dot<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, Q, n, st, partial);
            k_ro_reduce<<<cap, RED_THREADS, 0, s>>>(partial, st, d);
            k_ro_sub<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, Q, d, n, st);
        }
        tr.launches += 6;
    }
};

// ===================================================================== CGLS
//
// Conjugate gradients on the normal equations (Sec. 2.1.1), damped form on
// [A; lam I] x ~ [b; 0] (Eq. 7):
//   q = A p;  delta = ||q||^2 + lam^2 ||p||^2;  a = gamma / delta;
//   x += a p;  r -= a q;  s = A^T r - lam^2 x;  gamma' = ||s||^2;
//   p = s + (gamma'/gamma) p.

struct CgState {
    double gamma, alpha, beta, lam2;
    int iter, stop, status, pad;
};

__global__ void __launch_bounds__(RED_THREADS) cg_begin(CgState *st, const double *part, int np) {
    __shared__ double red[RED_THREADS / 32];
    const double ss = reduce_partials(part, np, red);
    if (threadIdx.x) return;
    st->iter = 0;
    st->status = CBCT_OK;
    st->stop = 0;
    st->gamma = ss;
    if (!good(ss)) {                                  // A^T b = 0: x = 0
        st->stop = 1;
        st->status = ss == 0.0 ? CBCT_OK : CBCT_EBREAKDOWN;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
cg_after_forward(CgState *st, const double *part_q, int nq, const double *part_p, int np) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop) return;
    const double qq = reduce_partials(part_q, nq, red);
    const double pp = reduce_partials(part_p, np, red);
    if (threadIdx.x) return;
    const double delta = qq + st->lam2 * pp;
    if (!good(delta)) {
        st->stop = 1;
        st->status = CBCT_EBREAKDOWN;
        return;
    }
    st->alpha = st->gamma / delta;
}

__global__ void __launch_bounds__(RED_THREADS)
cg_after_backward(CgState *st, const double *part_s, int ns, const double *part_r, int nr,
                  double *hist_r, double *hist_n, int cap) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop) return;
    const double ss = reduce_partials(part_s, ns, red);
    const double rr = reduce_partials(part_r, nr, red);
    if (threadIdx.x) return;
    const int it = st->iter;
    if (it < cap) {
        hist_r[it] = sqrt(rr);
        hist_n[it] = sqrt(ss);
    }
    st->iter = it + 1;
    if (!(ss > 0.0) || !isfinite(ss)) {               // converged exactly (or broke down)
        st->stop = 1;
        st->status = ss == 0.0 ? CBCT_OK : CBCT_EBREAKDOWN;
        return;
    }
    st->beta = ss / st->gamma;
    st->gamma = ss;
}

__global__ void __launch_bounds__(VEC_THREADS)
k_copy_sumsq(const float *__restrict__ src, float *__restrict__ dst, float *__restrict__ dst2, int64_t n,
             double *partial, const CgState *st) {
    __shared__ double red[VEC_THREADS / 32];
    if (st && st->stop) return;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        const float v = src[i];
        dst[i] = v;
        if (dst2) dst2[i] = 0.0f;
        s += (double)v * v;
    }
    s = block_sum<VEC_THREADS>(s, red);
    if (threadIdx.x == 0 && partial) partial[blockIdx.x] = s;
}

// r -= alpha q, partial ||r||^2
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_r(float *__restrict__ r, const float *__restrict__ q, int64_t n, double *partial, const CgState *st) {
    __shared__ double red[VEC_THREADS / 32];
    if (st->stop) return;
    const float a = (float)st->alpha;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        const float v = fmaf(-a, q[i], r[i]);
        r[i] = v;
        s += (double)v * v;
    }
    s = block_sum<VEC_THREADS>(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// x += alpha p; s -= lam^2 x; partial ||s||^2
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_xs(float *__restrict__ x, float *__restrict__ s, const float *__restrict__ p, int64_t n, double *partial,
        const CgState *st) {
    __shared__ double red[VEC_THREADS / 32];
    if (st->stop) return;
    const float a = (float)st->alpha, l2 = (float)st->lam2;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        const float xi = fmaf(a, p[i], x[i]);
        x[i] = xi;
        const float si = fmaf(-l2, xi, s[i]);
        s[i] = si;
        acc += (double)si * si;
    }
    acc = block_sum<VEC_THREADS>(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// p = s + beta p; partial ||p||^2
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_p(float *__restrict__ p, const float *__restrict__ s, int64_t n, double *partial, const CgState *st) {
    __shared__ double red[VEC_THREADS / 32];
    if (st->stop) return;
    const float b = (float)st->beta;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        const float v = fmaf(b, p[i], s[i]);
        p[i] = v;
        acc += (double)v * v;
    }
    acc = block_sum<VEC_THREADS>(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// ====================================================================== drivers


template <typename T>
static cbct_status gk_solve(const cbct_geometry *geom, const float *b, float *x, const cbct_solve_opts *o,
                            cbct_solve_report *rep, cudaStream_t s, Method method, bool lsmr_proj) {
    const DevGeom &g = geom->dev;
    // m: length of a volume-side vector (padded z-fastest layout); mvox: voxels
    const int64_t n = cbct_geometry_num_rays(geom), m = zf_len(geom->dev), mvox = cbct_geometry_num_voxels(geom);
    const int iters = o->iters;
    const int nf = forward_num_partials(g), nb = backward_num_partials(g);
    Workspace ws(s);
    SolveIO io{};
    cbct_status st = setup_io(geom, b, x, ws, io);
    if (st != CBCT_OK) return st;

    T *U = nullptr, *V = nullptr, *basis = nullptr;
    float *w = nullptr, *h2 = nullptr, *W = nullptr;
    double *pf = nullptr, *pb = nullptr, *pv = nullptr, *hist = nullptr;
    double *alpha_arr = nullptr, *beta_arr = nullptr, *scale_arr = nullptr, *coef = nullptr, *work = nullptr;
    GkState *dst = nullptr;
    CBCT_CUDA_TRY(ws.alloc(&U, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc(&W, (size_t)n));          // |d'| U, the transpose's input
    if (method == M_HYBRID) {
        CBCT_CUDA_TRY(ws.alloc_volumes(&basis, g, (size_t)iters + 1));
        CBCT_CUDA_TRY(ws.alloc(&alpha_arr, (size_t)iters + 2));
        CBCT_CUDA_TRY(ws.alloc(&beta_arr, (size_t)iters + 2));
        CBCT_CUDA_TRY(ws.alloc(&scale_arr, (size_t)iters + 2));
        CBCT_CUDA_TRY(ws.alloc(&coef, (size_t)iters + 1));
        CBCT_CUDA_TRY(ws.alloc(&work, (size_t)(iters + 1) * iters * 2 + 4 * (iters + 1)));
        V = basis;
    } else {
        CBCT_CUDA_TRY(ws.alloc_volumes(&V, g));
        CBCT_CUDA_TRY(ws.alloc_volumes(&w, g));
        if (method == M_LSMR) CBCT_CUDA_TRY(ws.alloc_volumes(&h2, g));
    }
    CBCT_CUDA_TRY(ws.alloc(&pf, (size_t)nf));
    CBCT_CUDA_TRY(ws.alloc(&pb, (size_t)nb));
    CBCT_CUDA_TRY(ws.alloc(&pv, (size_t)VEC_BLOCKS));
    double *pfold = nullptr;        // folded partials (k_fold_partials)
    CBCT_CUDA_TRY(ws.alloc(&pfold, (size_t)2 * FOLD_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&hist, (size_t)3 * iters));
    CBCT_CUDA_TRY(ws.alloc(&dst, 1));
    float *accum = nullptr;         // running sums of a transpose summed in passes
    if (g.angle_block < g.nangles) CBCT_CUDA_TRY(ws.alloc(&accum, (size_t)mvox));
    const int bwd_passes = backward_passes(g, accum);
    CBCT_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(double) * 3 * iters, s));

    Tracker tr;
    tr.profile = o->profile != 0;
    tr.s = s;
    // the scalar steps read the tiles' partials directly or folded first
    auto partials = [&](const double *p, int np, double *fold, const double **q, int *nq) {
        if (np > FOLD_MIN) {
            k_fold_partials<RED_THREADS><<<FOLD_BLOCKS, RED_THREADS, 0, s>>>(p, np, fold);
            ++tr.launches;
            *q = fold;
            *nq = FOLD_BLOCKS;
        } else {
            *q = p;
            *nq = np;
        }
    };
    GkState init;
    std::memset(&init, 0, sizeof init);
    init.damp = method == M_HYBRID ? 0.0 : o->lambda;
    init.sqrt_n = std::sqrt((double)n);
    init.sqrt_m = std::sqrt((double)mvox);
    init.scaled = std::is_same<T, __half>::value ? 1 : 0;
    CBCT_CUDA_TRY(cudaMemcpyAsync(dst, &init, sizeof init, cudaMemcpyHostToDevice, s));
    const cbct_dtype t = o->storage;
    const int *stop = &dst->stop;

    auto fwd = [&](const void *in, void *out, const Epilogue &e) -> cbct_status {
        cbct_status r = tr.mark(0);
        if (r == CBCT_OK) r = launch_forward(g, in, out, t, e, s, true);
        if (r == CBCT_OK) r = tr.mark(0);
        ++tr.launches;
        ++tr.fwd;
        return r;
    };
    auto fwd32 = [&](const void *in, void *out, const Epilogue &e) -> cbct_status {
        cbct_status r = tr.mark(0);
        if (r == CBCT_OK) r = launch_forward(g, in, out, CBCT_F32, e, s, true);
        if (r == CBCT_OK) r = tr.mark(0);
        ++tr.launches;
        ++tr.fwd;
        return r;
    };
    ExplicitMonitor em;
    st = em.init(o, g, n, m, ws);
    if (st != CBCT_OK) return st;
    int *stopw = &dst->stop;
    auto bwd = [&](const float *in, void *out, const Epilogue &e) -> cbct_status {
        cbct_status r = tr.mark(1);
        if (r == CBCT_OK) r = launch_backward(g, in, out, t, e, s, true, accum);
        if (r == CBCT_OK) r = tr.mark(1);
        tr.launches += bwd_passes;
        tr.bwd += bwd_passes;
        return r;
    };

    Reorth ro;
    if constexpr (std::is_same<T, float>::value) {
        st = ro.init(o, n, m, ws);
        if (st != CBCT_OK) return st;
    }
    // beta_1 u_1 = b
    k_sumsq<float><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(io.b_dev, n, pv);
    gk_begin<<<1, RED_THREADS, 0, s>>>(dst, pv, VEC_BLOCKS);
    k_scale_to<T><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(io.b_dev, U, n, &dst->c0, stop);
    tr.launches += 4;
    if constexpr (std::is_same<T, float>::value) {
        if (ro.on) {
            k_ro_store<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(U, ro.Ub, n, dst, 0, 0);       // u_1
            ++tr.launches;
        }
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    st = launch_weight(g, U, t, W, s);
    if (st != CBCT_OK) return st;
    if (method == M_HYBRID) {
        double one = 1.0;
        CBCT_CUDA_TRY(cudaMemcpyAsync(scale_arr, &one, sizeof one, cudaMemcpyHostToDevice, s));
    }
    // alpha_1 v_1 = A^T u_1
    {
        Epilogue e{&dst->ba, &dst->bb, 0, 0, pb, stop, nullptr};
        st = bwd(W, V, e);
        if (st != CBCT_OK) return st;
    }
    gk_begin2<<<1, RED_THREADS, 0, s>>>(dst, pb, nb, (int)method);
    ++tr.launches;
    if constexpr (std::is_same<T, float>::value) {
        if (ro.on) {
            k_ro_store<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(V, ro.Vb, m, dst, 1, 0);       // v_1
            ++tr.launches;
        }
    }
    if (method == M_LSQR)
        k_start_dirs<T><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(V, w, nullptr, nullptr, m, dst);
    else if (method == M_LSMR)
        k_start_dirs<T><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(V, w, h2, nullptr, m, dst);
    if (method != M_HYBRID) ++tr.launches;
    CBCT_CUDA_TRY(cudaGetLastError());
    if (method == M_HYBRID) {
        // record beta_1, alpha_1 once gk_begin2 ran
        CBCT_CUDA_TRY(cudaMemcpyAsync(beta_arr, &dst->beta, sizeof(double), cudaMemcpyDeviceToDevice, s));
        CBCT_CUDA_TRY(cudaMemcpyAsync(alpha_arr, &dst->alpha, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }

    double *hist_r = hist, *hist_n = hist + iters, *hist_l = hist + 2 * iters;
    int k = 0;
    auto one_iteration = [&]() -> cbct_status {
        T *Vin = method == M_HYBRID ? basis + (size_t)k * m : V;
        T *Vout = method == M_HYBRID ? basis + (size_t)(k + 1) * m : V;
        Epilogue ef{&dst->fa, &dst->fb, 0, 0, pf, stop, nullptr, ro.on ? nullptr : W};
        cbct_status r = fwd(Vin, U, ef);
        if (r != CBCT_OK) return r;
        bool done_fwd = false, done_bwd = false;
        if constexpr (std::is_same<T, float>::value) {
            if (ro.on) {                 // u against u_1 .. u_{i+1}, then its norm, u_{i+2}, w = |d'| u
                ro.orthogonalise(U, ro.Ub, n, dst, s, tr);
                k_sumsq<float><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(U, n, pv);
                gk_after_forward<<<1, RED_THREADS, 0, s>>>(dst, pv, VEC_BLOCKS, beta_arr);
                k_ro_store<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(U, ro.Ub, n, dst, 0, 1);
                tr.launches += 2;
                r = launch_weight(g, U, t, W, s);
                if (r != CBCT_OK) return r;
                ++tr.launches;
                done_fwd = true;
            }
        }
        if (!done_fwd) {
            const double *q;
            int nq;
            partials(pf, nf, pfold, &q, &nq);
            gk_after_forward<<<1, RED_THREADS, 0, s>>>(dst, q, nq, beta_arr);
        }
        Epilogue eb{&dst->ba, &dst->bb, 0, 0, pb, stop, method == M_HYBRID ? (const void *)Vin : nullptr};
        r = bwd(W, Vout, eb);
        if (r != CBCT_OK) return r;
        if constexpr (std::is_same<T, float>::value) {
            if (ro.on) {                 // v against v_1 .. v_{i+1}, then its norm and v_{i+2}
                ro.orthogonalise(Vout, ro.Vb, m, dst, s, tr);
                k_sumsq<float><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(Vout, m, pv);
                gk_after_backward<<<1, RED_THREADS, 0, s>>>(dst, pv, VEC_BLOCKS, (int)method, hist_r, hist_n,
                                                             alpha_arr, scale_arr, iters);
                k_ro_store<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(Vout, ro.Vb, m, dst, 1, 0);
                tr.launches += 2;
                done_bwd = true;
            }
        }
        if (!done_bwd) {
            const double *q;
            int nq;
            partials(pb, nb, pfold + FOLD_BLOCKS, &q, &nq);
            gk_after_backward<<<1, RED_THREADS, 0, s>>>(dst, q, nq, (int)method, hist_r, hist_n, alpha_arr,
                                                         scale_arr, iters);
        }
        tr.launches += 3;            // two finalize kernels + the update / projected solve
        em.keep(io.xz, m, stop, s, tr);
        if (method == M_LSQR) {
            k_lsqr_update<T><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(V, io.xz, w, m, dst);
        } else if (method == M_LSMR) {
            k_lsmr_update<T><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(V, io.xz, w, h2, m, dst);
        } else {
            // hybrid LSMR's projected residual is the normal-equation residual ||A^T r_k||
            r = launch_projected_solve(alpha_arr, beta_arr, scale_arr, &dst->iter, stop, (int)o->rule, o->lambda,
                                       o->noise_level, lsmr_proj ? 1 : 0, work, iters, coef, hist_l,
                                       lsmr_proj ? hist_n : hist_r, s);
            if (r != CBCT_OK) return r;
            if (em.on) {                 // the monitor needs x_k itself: x_k = V_k y_k
                k_combine<T><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(basis, coef, k + 1, m, io.xz, stop);
                ++tr.launches;
            }
        }
        CBCT_CUDA_TRY(cudaGetLastError());
        return em.check(fwd32, io.xz, io.b_dev, stopw, s, tr);
    };
    if (method == M_HYBRID) {
        for (k = 0; k < iters; ++k) {
            st = one_iteration();
            if (st != CBCT_OK) return st;
        }
    } else {
        const Tracker before = tr.snapshot();
        int replays = 0;
        st = run_iterations(iters, o->use_graph != 0 && !tr.profile, s, one_iteration, &replays);
        if (st != CBCT_OK) return st;
        tr.scale_since(before, replays);
    }

    // read back the state to learn how many iterations completed
    GkState fin;
    std::vector<double> h((size_t)3 * iters);
    CBCT_CUDA_TRY(cudaMemcpyAsync(&fin, dst, sizeof fin, cudaMemcpyDeviceToHost, s));
    CBCT_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * 3 * iters, cudaMemcpyDeviceToHost, s));
    CBCT_CUDA_TRY(cudaStreamSynchronize(s));
    if (method == M_HYBRID && fin.iter > 0 && !em.on) {
        // x_k = V_k y_k with the coefficients of the last completed projected solve
        k_combine<T><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(basis, coef, fin.iter, m, io.xz);
        ++tr.launches;
        CBCT_CUDA_TRY(cudaGetLastError());
    }
    int done = fin.iter;
    st = em.finish(io.xz, m, s, rep, &done);
    if (st != CBCT_OK) return st;
    st = finish_io(geom, io, s);
    if (st != CBCT_OK) return st;
    ++tr.launches;                   // the final re-layout of x
    if (io.x_is_host || method == M_HYBRID) CBCT_CUDA_TRY(cudaStreamSynchronize(s));
    copy_report(rep, done, h, iters);
    tr.fill(rep);
    if (fin.status == CBCT_EBREAKDOWN) set_error("Krylov breakdown: a norm became zero or non-finite");
    return (cbct_status)fin.status;
}

static cbct_status cgls_solve(const cbct_geometry *geom, const float *b, float *x, const cbct_solve_opts *o,
                              cbct_solve_report *rep, cudaStream_t s) {
    const DevGeom &g = geom->dev;
    // m: length of a volume-side vector (padded z-fastest layout); mvox: voxels
    const int64_t n = cbct_geometry_num_rays(geom), m = zf_len(geom->dev), mvox = cbct_geometry_num_voxels(geom);
    const int iters = o->iters;
    const int nf = forward_num_partials(g);
    Workspace ws(s);
    SolveIO io{};
    cbct_status st = setup_io(geom, b, x, ws, io);
    if (st != CBCT_OK) return st;
    float *r = nullptr, *q = nullptr, *sv = nullptr, *p = nullptr, *wr = nullptr;
    double *pq = nullptr, *pp = nullptr, *pr = nullptr, *ps = nullptr, *hist = nullptr;
    CgState *dst = nullptr;
    CBCT_CUDA_TRY(ws.alloc(&r, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc(&q, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc(&wr, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc_volumes(&sv, g));
    CBCT_CUDA_TRY(ws.alloc_volumes(&p, g));
    CBCT_CUDA_TRY(ws.alloc(&pq, (size_t)nf));
    CBCT_CUDA_TRY(ws.alloc(&pp, (size_t)VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&pr, (size_t)VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&ps, (size_t)VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&hist, (size_t)3 * iters));
    CBCT_CUDA_TRY(ws.alloc(&dst, 1));
    CBCT_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(double) * 3 * iters, s));
    float *accum = nullptr;         // running sums of a transpose summed in passes
    if (g.angle_block < g.nangles) CBCT_CUDA_TRY(ws.alloc(&accum, (size_t)mvox));
    const int bwd_passes = backward_passes(g, accum);
    Tracker tr;
    tr.profile = o->profile != 0;
    tr.s = s;
    auto fwd = [&](const void *in, void *out, const Epilogue &e) -> cbct_status {
        cbct_status r = tr.mark(0);
        if (r == CBCT_OK) r = launch_forward(g, in, out, CBCT_F32, e, s, true);
        if (r == CBCT_OK) r = tr.mark(0);
        ++tr.launches;
        ++tr.fwd;
        return r;
    };
    auto bwd = [&](const float *in, void *out, const Epilogue &e) -> cbct_status {
        cbct_status r = tr.mark(1);
        if (r == CBCT_OK) r = launch_backward(g, in, out, CBCT_F32, e, s, true, accum);
        if (r == CBCT_OK) r = tr.mark(1);
        tr.launches += bwd_passes;
        tr.bwd += bwd_passes;
        return r;
    };
    CgState init{};
    init.lam2 = o->lambda * o->lambda;
    CBCT_CUDA_TRY(cudaMemcpyAsync(dst, &init, sizeof init, cudaMemcpyHostToDevice, s));
    const int *stop = &dst->stop;
    int *stopw = &dst->stop;
    ExplicitMonitor em;
    st = em.init(o, g, n, m, ws);
    if (st != CBCT_OK) return st;

    // r = b; s = A^T r; gamma = ||s||^2; p = s
    k_copy_sumsq<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(io.b_dev, r, nullptr, n, nullptr, nullptr);
    st = launch_weight(g, r, CBCT_F32, wr, s);
    if (st != CBCT_OK) return st;
    tr.launches += 2;
    {
        Epilogue e{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
        st = bwd(wr, sv, e);
        if (st != CBCT_OK) return st;
    }
    k_copy_sumsq<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(sv, p, nullptr, m, pp, nullptr);
    cg_begin<<<1, RED_THREADS, 0, s>>>(dst, pp, VEC_BLOCKS);
    tr.launches += 2;
    CBCT_CUDA_TRY(cudaGetLastError());

    double *hist_r = hist, *hist_n = hist + iters;
    auto one_iteration = [&]() -> cbct_status {
        Epilogue ef{nullptr, nullptr, 1.0, 0.0, pq, stop, nullptr};
        cbct_status rr = fwd(p, q, ef);
        if (rr != CBCT_OK) return rr;
        cg_after_forward<<<1, RED_THREADS, 0, s>>>(dst, pq, nf, pp, VEC_BLOCKS);
        k_cg_r<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(r, q, n, pr, dst);
        rr = launch_weight(g, r, CBCT_F32, wr, s);        // the transpose's input |d'| r
        if (rr != CBCT_OK) return rr;
        Epilogue eb{nullptr, nullptr, 1.0, 0.0, nullptr, stop, nullptr};
        rr = bwd(wr, sv, eb);
        if (rr != CBCT_OK) return rr;
        em.keep(io.xz, m, stop, s, tr);
        k_cg_xs<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(io.xz, sv, p, m, ps, dst);
        cg_after_backward<<<1, RED_THREADS, 0, s>>>(dst, ps, VEC_BLOCKS, pr, VEC_BLOCKS, hist_r, hist_n, iters);
        k_cg_p<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(p, sv, m, pp, dst);
        tr.launches += 6;
        CBCT_CUDA_TRY(cudaGetLastError());
        return em.check(fwd, io.xz, io.b_dev, stopw, s, tr);
    };
    const Tracker before = tr.snapshot();
    int replays = 0;
    st = run_iterations(iters, o->use_graph != 0 && !tr.profile, s, one_iteration, &replays);
    if (st != CBCT_OK) return st;
    tr.scale_since(before, replays);
    CgState fin;
    std::vector<double> h((size_t)3 * iters);
    CBCT_CUDA_TRY(cudaMemcpyAsync(&fin, dst, sizeof fin, cudaMemcpyDeviceToHost, s));
    CBCT_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * 3 * iters, cudaMemcpyDeviceToHost, s));
    CBCT_CUDA_TRY(cudaStreamSynchronize(s));
    int done = fin.iter;
    st = em.finish(io.xz, m, s, rep, &done);
    if (st != CBCT_OK) return st;
    st = finish_io(geom, io, s);
    if (st != CBCT_OK) return st;
    ++tr.launches;                   // the final re-layout of x
    CBCT_CUDA_TRY(cudaStreamSynchronize(s));
    copy_report(rep, done, h, iters);
    tr.fill(rep);
    if (fin.status == CBCT_EBREAKDOWN) set_error("Krylov breakdown: a norm became zero or non-finite");
    return (cbct_status)fin.status;
}

static cbct_status dispatch_gk(const cbct_geometry *g, const float *b, float *x, const cbct_solve_opts *o,
                               cbct_solve_report *rep, cbct_stream stream, Method method,
                               bool lsmr_proj = false) {
    cbct_status st = check_solve_args(g, b, x, o);
    if (st != CBCT_OK) return st;
    if (method == M_HYBRID && o->rule != CBCT_LAMBDA_FIXED && o->rule != CBCT_LAMBDA_GCV &&
        o->rule != CBCT_LAMBDA_DP) {
        set_error("hybrid LSQR: unknown lambda rule");
        return CBCT_EINVAL;
    }
    if (method == M_HYBRID && o->rule == CBCT_LAMBDA_DP && !(o->noise_level >= 0.0 && o->noise_level < 1.0)) {
        set_error("hybrid LSQR: the discrepancy principle needs 0 <= noise_level < 1");
        return CBCT_EINVAL;
    }
    if (o->reorth && o->storage != CBCT_F32) {
        set_error("re-orthogonalisation needs FP32 storage");
        return CBCT_EINVAL;
    }
    if (lsmr_proj && o->rule == CBCT_LAMBDA_DP) {
        set_error("hybrid LSMR: lambda by GCV or fixed (the discrepancy principle bounds ||r||, not ||A^T r||)");
        return CBCT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    switch (o->storage) {
    case CBCT_F16: return gk_solve<__half>(g, b, x, o, rep, s, method, lsmr_proj);
    case CBCT_BF16: return gk_solve<__nv_bfloat16>(g, b, x, o, rep, s, method, lsmr_proj);
    default: return gk_solve<float>(g, b, x, o, rep, s, method, lsmr_proj);
    }
}

}  // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_lsqr_solve(const cbct_geometry *g, const float *b, float *x, const cbct_solve_opts *o,
                                       cbct_solve_report *rep, cbct_stream stream) {
    return dispatch_gk(g, b, x, o, rep, stream, M_LSQR);
}

extern "C" cbct_status cbct_lsmr_solve(const cbct_geometry *g, const float *b, float *x, const cbct_solve_opts *o,
                                       cbct_solve_report *rep, cbct_stream stream) {
    return dispatch_gk(g, b, x, o, rep, stream, M_LSMR);
}

extern "C" cbct_status cbct_hybrid_lsqr_solve(const cbct_geometry *g, const float *b, float *x,
                                              const cbct_solve_opts *o, cbct_solve_report *rep, cbct_stream stream) {
    return dispatch_gk(g, b, x, o, rep, stream, M_HYBRID);
}

extern "C" cbct_status cbct_hybrid_lsmr_solve(const cbct_geometry *g, const float *b, float *x,
                                              const cbct_solve_opts *o, cbct_solve_report *rep, cbct_stream stream) {
    return dispatch_gk(g, b, x, o, rep, stream, M_HYBRID, true);
}

extern "C" cbct_status cbct_cgls_solve(const cbct_geometry *g, const float *b, float *x, const cbct_solve_opts *o,
                                       cbct_solve_report *rep, cbct_stream stream) {
    cbct_status st = check_solve_args(g, b, x, o);
    if (st != CBCT_OK) return st;
    if (o->storage != CBCT_F32) {
        set_error("CGLS supports FP32 storage only");
        return CBCT_EINVAL;
    }
    if (o->reorth) {
        set_error("CGLS has no Golub-Kahan basis to re-orthogonalise");
        return CBCT_EINVAL;
    }
    return cgls_solve(g, b, x, o, rep, (cudaStream_t)stream);
}
