// CGLS-TV (Sec. 2.3.1): isotropic 3D total variation by iteratively reweighted
// norms.  Outer step k fixes the weights w = (|D x^(k)|^2 + tau^2)^(-1/4) and
// runs CGLS on the stacked system
//     [A ; lam W D] x ~ [b ; 0]
// from x^(k); the regularisation term lam^2 ||W D x||^2 tends to lam^2 TV(x).
// D is the forward-difference gradient along i, j, k with a zero last
// difference (Neumann boundary); its adjoint is applied in the same kernel that
// adds lam D^T (W r_D) to the backprojection.  Volumes are z-fastest
// (v = (j nx + i) nz + k), the gradient part of a stacked vector is three
// volumes (components i, j, k).  FP32 vectors, FP64 scalars and norms.
#include <cmath>
#include <vector>

#include "solver_common.cuh"

namespace cbct {

struct TvState {
    double gamma, gamma0, alpha, beta, lam;
    int iter, stop, pad0, pad1;
};

constexpr double TV_CONVERGED = 1e-14;     // inner CGLS stops once ||s|| <= this x its start

// Voxel coordinates of the padded z-fastest layout (index v =
// ZF_GUARD + (j nx + i) (nz + 2) + 1 + k); pads and guards have none.
struct VolIndex {
    int nx, ny, nz;
    __device__ __forceinline__ int64_t len() const { return (int64_t)nx * ny * (nz + 2) + 2 * ZF_GUARD; }
    __device__ __forceinline__ int64_t oi() const { return nz + 2; }
    __device__ __forceinline__ int64_t oj() const { return (int64_t)nx * (nz + 2); }
    __device__ __forceinline__ bool coords(int64_t v, int &i, int &j, int &k) const {
        const int64_t c = v - ZF_GUARD;
        if (c < 0) return false;
        const int64_t col = c / (nz + 2);
        if (col >= (int64_t)nx * ny) return false;
        k = (int)(c - col * (nz + 2)) - 1;
        if (k < 0 || k >= nz) return false;
        i = (int)(col % nx);
        j = (int)(col / nx);
        return true;
    }
};

// w = (|D x|^2 + tau^2)^(-1/4)
__global__ void __launch_bounds__(VEC_THREADS)
k_tv_weights(const float *__restrict__ x, float *__restrict__ w, VolIndex vi, float tau) {
    const int64_t m = vi.len(), oi = vi.oi(), oj = vi.oj();
    for (int64_t v = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; v < m; v += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        int i, j, k;
        if (!vi.coords(v, i, j, k)) continue;
        const float xv = x[v];
        const float di = i < vi.nx - 1 ? x[v + oi] - xv : 0.0f;
        const float dj = j < vi.ny - 1 ? x[v + oj] - xv : 0.0f;
        const float dk = k < vi.nz - 1 ? x[v + 1] - xv : 0.0f;
        w[v] = (float)pow((double)di * di + (double)dj * dj + (double)dk * dk + (double)tau * tau, -0.25);
    }
}

// out = c * w * D x (three components), partial ||out||^2; c = coef * scale (device scalar or value)
__global__ void __launch_bounds__(VEC_THREADS)
k_grad_w(const float *__restrict__ x, const float *__restrict__ w, float *__restrict__ out, VolIndex vi, double c,
         double *partial, const int *stop) {
    __shared__ double red[VEC_THREADS / 32];
    if (stop && *stop) return;
    const int64_t m = vi.len(), oi = vi.oi(), oj = vi.oj();
    double ss = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; v < m; v += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        int i, j, k;
        if (!vi.coords(v, i, j, k)) continue;
        const float xv = x[v];
        const float cw = (float)(c * (double)w[v]);
        const float gi = cw * (i < vi.nx - 1 ? x[v + oi] - xv : 0.0f);
        const float gj = cw * (j < vi.ny - 1 ? x[v + oj] - xv : 0.0f);
        const float gk = cw * (k < vi.nz - 1 ? x[v + 1] - xv : 0.0f);
        out[v] = gi;
        out[m + v] = gj;
        out[2 * m + v] = gk;
        ss += (double)gi * gi + (double)gj * gj + (double)gk * gk;
    }
    if (partial) {
        ss = block_sum<VEC_THREADS>(ss, red);
        if (threadIdx.x == 0) partial[blockIdx.x] = ss;
    }
}

// s += lam D^T (w r_d), partial ||s||^2
__global__ void __launch_bounds__(VEC_THREADS)
k_div_w_add(const float *__restrict__ rd, const float *__restrict__ w, float *__restrict__ s, VolIndex vi, double lam,
            double *partial, const int *stop) {
    __shared__ double red[VEC_THREADS / 32];
    if (stop && *stop) return;
    const int64_t m = vi.len(), oi = vi.oi(), oj = vi.oj();
    double ss = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; v < m; v += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        int i, j, k;
        if (!vi.coords(v, i, j, k)) continue;
        // (D_c^T u)[v] = u[v - o_c] (if the previous voxel's difference exists) - u[v] (if v's exists)
        const float wv = w[v];
        double t = 0.0;
        if (i >= 1) t += (double)w[v - oi] * rd[v - oi];
        if (i < vi.nx - 1) t -= (double)wv * rd[v];
        if (j >= 1) t += (double)w[v - oj] * rd[m + v - oj];
        if (j < vi.ny - 1) t -= (double)wv * rd[m + v];
        if (k >= 1) t += (double)w[v - 1] * rd[2 * m + v - 1];
        if (k < vi.nz - 1) t -= (double)wv * rd[2 * m + v];
        const float sv = (float)((double)s[v] + lam * t);
        s[v] = sv;
        ss += (double)sv * sv;
    }
    ss = block_sum<VEC_THREADS>(ss, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = ss;
}

// gamma = ||s||^2 at the start of an outer step
__global__ void __launch_bounds__(RED_THREADS) k_tv_begin(TvState *st, const double *part) {
    __shared__ double red[RED_THREADS / 32];
    const double g = reduce_partials(part, VEC_BLOCKS, red);
    if (threadIdx.x) return;
    st->gamma = g;
    st->gamma0 = g;
    st->stop = !(g > 0.0) || !isfinite(g);
}

// alpha = gamma / (||q_A||^2 + ||q_D||^2)
__global__ void __launch_bounds__(RED_THREADS)
k_tv_alpha(TvState *st, const double *part_a, int na, const double *part_d) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop) return;
    const double qa = reduce_partials(part_a, na, red);
    const double qd = reduce_partials(part_d, VEC_BLOCKS, red);
    if (threadIdx.x) return;
    const double delta = qa + qd;
    if (!(delta > 0.0) || !isfinite(delta)) {
        st->stop = 1;
        return;
    }
    st->alpha = st->gamma / delta;
}

// gamma' = ||s||^2, beta, the history; stop once converged
__global__ void __launch_bounds__(RED_THREADS)
k_tv_beta(TvState *st, const double *part_s, const double *part_r, double *hist_r, double *hist_n, int cap) {
    __shared__ double red[RED_THREADS / 32];
    if (st->stop) return;
    const double g = reduce_partials(part_s, VEC_BLOCKS, red);
    const double rr = reduce_partials(part_r, VEC_BLOCKS, red);
    if (threadIdx.x) return;
    const int it = st->iter;
    if (it < cap) {
        hist_r[it] = sqrt(rr);
        hist_n[it] = sqrt(g);
    }
    st->iter = it + 1;
    st->beta = g / st->gamma;
    st->gamma = g;
    if (!isfinite(g) || g <= TV_CONVERGED * TV_CONVERGED * st->gamma0) st->stop = 1;
}

// y += sign * alpha * x (alpha from the state), optional partial ||y||^2
__global__ void __launch_bounds__(VEC_THREADS)
k_tv_axpy(float *__restrict__ y, const float *__restrict__ x, int64_t n, const TvState *st, double sign,
          double *partial) {
    __shared__ double red[VEC_THREADS / 32];
    if (st->stop) return;
    const float a = (float)(sign * st->alpha);
    double ss = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        const float v = fmaf(a, x[e], y[e]);
        y[e] = v;
        ss += (double)v * v;
    }
    if (partial) {
        ss = block_sum<VEC_THREADS>(ss, red);
        if (threadIdx.x == 0) partial[blockIdx.x] = ss;
    }
}

// p = s + beta p (skipped after the stop, like every update)
__global__ void __launch_bounds__(VEC_THREADS)
k_tv_p(float *__restrict__ p, const float *__restrict__ s, int64_t n, const TvState *st, int first) {
    if (!first && st->stop) return;
    const float b = first ? 0.0f : (float)st->beta;
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS)
        p[e] = first ? s[e] : fmaf(b, p[e], s[e]);
}

__global__ void k_tv_reset(TvState *st) {
    st->stop = 0;
}

static cbct_status cgls_tv_solve(const cbct_geometry *geom, const float *b, float *x, const cbct_solve_opts *o,
                                 cbct_solve_report *rep, cudaStream_t s) {
    const DevGeom &g = geom->dev;
    // m: length of a volume-side vector (padded z-fastest layout, pads kept at zero)
    const int64_t n = cbct_geometry_num_rays(geom), m = zf_len(geom->dev);
    const int iters = o->iters, outer = o->tv_outer;
    const double lam = o->lambda;
    const VolIndex vi{g.nx, g.ny, g.nz};
    const int nf = forward_num_partials(g);
    Workspace ws(s);
    SolveIO io{};
    cbct_status st = setup_io(geom, b, x, ws, io);
    if (st != CBCT_OK) return st;
    float *w = nullptr, *ra = nullptr, *rd = nullptr, *qa = nullptr, *qd = nullptr, *p = nullptr, *sv = nullptr,
          *wa = nullptr;
    double *pf = nullptr, *pd = nullptr, *ps = nullptr, *pr = nullptr, *hist = nullptr;
    TvState *dst = nullptr;
    CBCT_CUDA_TRY(ws.alloc_volumes(&w, g));
    CBCT_CUDA_TRY(ws.alloc(&ra, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc(&qa, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc(&wa, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc_volumes(&rd, g, 3));
    CBCT_CUDA_TRY(ws.alloc_volumes(&qd, g, 3));
    CBCT_CUDA_TRY(ws.alloc_volumes(&p, g));
    CBCT_CUDA_TRY(ws.alloc_volumes(&sv, g));
    CBCT_CUDA_TRY(ws.alloc(&pf, (size_t)nf));
    CBCT_CUDA_TRY(ws.alloc(&pd, (size_t)VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&ps, (size_t)VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&pr, (size_t)VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&hist, (size_t)3 * iters));
    CBCT_CUDA_TRY(ws.alloc(&dst, 1));
    CBCT_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(double) * 3 * iters, s));
    CBCT_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(TvState), s));
    Tracker tr;
    tr.s = s;
    const int *stop = &dst->stop;
    auto fwd = [&](const float *in, float *out, const Epilogue &e) -> cbct_status {
        ++tr.launches;
        ++tr.fwd;
        return launch_forward(g, in, out, CBCT_F32, e, s, true);
    };
    // s = A^T r_A + lam D^T (W r_D), partial ||s||^2
    auto normal = [&]() -> cbct_status {
        cbct_status r = launch_weight(g, ra, CBCT_F32, wa, s);
        const Epilogue e{nullptr, nullptr, 1.0, 0.0, nullptr, stop, nullptr};
        if (r == CBCT_OK) r = launch_backward(g, wa, sv, CBCT_F32, e, s, true, nullptr);
        k_div_w_add<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(rd, w, sv, vi, lam, ps, stop);
        tr.launches += 3;
        ++tr.bwd;
        return r;
    };
    double *hist_r = hist, *hist_n = hist + iters;
    int it = 0;
    for (int k = 0; k < outer && it < iters; ++k) {
        const int inner = (iters - it) / (outer - k);          // spread the iterations over the outer steps
        k_tv_reset<<<1, 1, 0, s>>>(dst);
        k_tv_weights<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(io.xz, w, vi, (float)o->tv_tau);
        // r_A = b - A x, r_D = -lam W D x
        const Epilogue er{nullptr, nullptr, -1.0, 1.0, nullptr, nullptr, io.b_dev};
        st = fwd(io.xz, ra, er);
        if (st != CBCT_OK) return st;
        k_grad_w<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(io.xz, w, rd, vi, -lam, nullptr, nullptr);
        tr.launches += 3;
        st = normal();
        if (st != CBCT_OK) return st;
        k_tv_begin<<<1, RED_THREADS, 0, s>>>(dst, ps);
        k_tv_p<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(p, sv, m, dst, 1);
        tr.launches += 2;
        for (int q = 0; q < inner; ++q, ++it) {
            const Epilogue ef{nullptr, nullptr, 1.0, 0.0, pf, stop, nullptr};
            st = fwd(p, qa, ef);                                         // q_A = A p
            if (st != CBCT_OK) return st;
            k_grad_w<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(p, w, qd, vi, lam, pd, stop);   // q_D = lam W D p
            k_tv_alpha<<<1, RED_THREADS, 0, s>>>(dst, pf, nf, pd);
            k_tv_axpy<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(io.xz, p, m, dst, 1.0, nullptr);    // x += alpha p
            k_tv_axpy<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(ra, qa, n, dst, -1.0, pr);         // r_A -= alpha q_A
            k_tv_axpy<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(rd, qd, 3 * m, dst, -1.0, nullptr); // r_D -= alpha q_D
            tr.launches += 5;
            st = normal();
            if (st != CBCT_OK) return st;
            k_tv_beta<<<1, RED_THREADS, 0, s>>>(dst, ps, pr, hist_r + 0, hist_n, iters);
            k_tv_p<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(p, sv, m, dst, 0);
            tr.launches += 2;
            CBCT_CUDA_TRY(cudaGetLastError());
        }
    }
    TvState fin;
    std::vector<double> h((size_t)3 * iters);
    CBCT_CUDA_TRY(cudaMemcpyAsync(&fin, dst, sizeof fin, cudaMemcpyDeviceToHost, s));
    CBCT_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * 3 * iters, cudaMemcpyDeviceToHost, s));
    st = finish_io(geom, io, s);
    if (st != CBCT_OK) return st;
    ++tr.launches;
    CBCT_CUDA_TRY(cudaStreamSynchronize(s));
    copy_report(rep, fin.iter, h, iters);
    tr.fill(rep);
    if (rep) {
        rep->explicit_count = 0;
        rep->stopped_on_residual = 0;
    }
    return CBCT_OK;
}

}  // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_cgls_tv_solve(const cbct_geometry *g, const float *b, float *x, const cbct_solve_opts *o,
                                          cbct_solve_report *rep, cbct_stream stream) {
    cbct_status st = check_solve_args(g, b, x, o);
    if (st != CBCT_OK) return st;
    if (o->storage != CBCT_F32) { set_error("CGLS-TV supports FP32 storage only"); return CBCT_EINVAL; }
    if (o->tv_outer < 1 || o->tv_outer > o->iters) {
        set_error("CGLS-TV: need 1 <= tv_outer <= iters");
        return CBCT_EINVAL;
    }
    if (!(o->tv_tau > 0.0) || !std::isfinite(o->tv_tau)) { set_error("CGLS-TV: tv_tau must be > 0"); return CBCT_EINVAL; }
    if (o->explicit_residual) {
        set_error("CGLS-TV: the explicit-residual monitor is not available");
        return CBCT_EINVAL;
    }
    return cgls_tv_solve(g, b, x, o, rep, (cudaStream_t)stream);
}
