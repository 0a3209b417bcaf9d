// AB-GMRES and BA-GMRES (Sec. 2.1.4): GMRES with the backprojector B as a
// right (AB) or left (BA) preconditioner, the paper's answer to backprojectors
// that are only approximately the transpose of A.
//
//   AB: min ||b - A B z|| over z in K_k(A B, b),        x_k = B z_k
//   BA: min ||B (b - A x)|| over x in K_k(B A, B b),    x_k itself
//
// B is A^T (then AB-GMRES computes LSQR's iterates and BA-GMRES LSMR's, in
// exact arithmetic), the SIRT-weighted C A^T R, R = 1 / (A 1) per ray and
// C = 1 / (A^T 1) per voxel, or the voxel-driven interpolating backprojector
// of vdbp.cu; the last two are not the transpose of A.
//
// Arnoldi runs on the device: the Krylov vectors are FP32 (projection-side,
// v-fastest, for AB; volume-side, z-fastest, for BA), each new vector is
// orthogonalised against all earlier ones by classical Gram-Schmidt applied
// twice with FP64 dot products (fixed-order block reductions), and the
// Hessenberg matrix is kept in FP64.  After the last iteration the host solves
// the (k+1) x k least-squares problems by Givens rotations (every k, for the
// residual history) and the device forms x_k.
#include <algorithm>
#include <cmath>
#include <vector>

#include "solver_common.cuh"

namespace cbct {

constexpr int MD_CHUNK = 8;     // dot products accumulated per pass over w

// partial[i * VEC_BLOCKS + block] = this block's share of w . V_i, i < count
__global__ void __launch_bounds__(VEC_THREADS)
k_multi_dot(const float *__restrict__ w, const float *__restrict__ V, int count, int64_t n, double *partial) {
    __shared__ double red[VEC_THREADS / 32];
    for (int c0 = 0; c0 < count; c0 += MD_CHUNK) {
        const int nc = min(MD_CHUNK, count - c0);
        double acc[MD_CHUNK];
#pragma unroll
        for (int q = 0; q < MD_CHUNK; ++q) acc[q] = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n;
             e += (int64_t)VEC_BLOCKS * VEC_THREADS) {
            const double we = w[e];
#pragma unroll
            for (int q = 0; q < MD_CHUNK; ++q)
                if (q < nc) acc[q] += we * (double)V[(size_t)(c0 + q) * n + e];
        }
#pragma unroll
        for (int q = 0; q < MD_CHUNK; ++q) {
            if (q >= nc) break;
            const double s = block_sum<VEC_THREADS>(acc[q], red);
            if (threadIdx.x == 0) partial[(size_t)(c0 + q) * VEC_BLOCKS + blockIdx.x] = s;
            __syncthreads();
        }
    }
}

// h[i] (+)= sum of the partials of dot i, fixed order; one block per dot
__global__ void __launch_bounds__(RED_THREADS)
k_reduce_dots(const double *partial, double *h, int accumulate) {
    __shared__ double red[RED_THREADS / 32];
    const double s = reduce_partials(partial + (size_t)blockIdx.x * VEC_BLOCKS, VEC_BLOCKS, red);
    if (threadIdx.x == 0) h[blockIdx.x] = accumulate ? h[blockIdx.x] + s : s;
}

// w -= sum_i c_i V_i  (c = the dots of this pass, FP64; the correction is summed in FP64)
__global__ void __launch_bounds__(VEC_THREADS)
k_multi_axpy(float *__restrict__ w, const float *__restrict__ V, const double *__restrict__ c, int count, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        double corr = 0.0;
        for (int i = 0; i < count; ++i) corr += c[i] * (double)V[(size_t)i * n + e];
        w[e] = (float)((double)w[e] - corr);
    }
}

// h_{j+1,j} = ||w|| from the partials; hcol[j+1] = h_{j+1,j}
__global__ void __launch_bounds__(RED_THREADS) k_column_norm(const double *partial, double *hcol, int j) {
    __shared__ double red[RED_THREADS / 32];
    const double ss = reduce_partials(partial, VEC_BLOCKS, red);
    if (threadIdx.x == 0) hcol[j + 1] = sqrt(ss);
}

// v_next = w / h (zero vector if h is zero: the Krylov space is exhausted)
__global__ void __launch_bounds__(VEC_THREADS)
k_normalise(const float *__restrict__ w, float *__restrict__ v, const double *h, int64_t n) {
    const double hv = *h;
    const float inv = hv > 0.0 ? (float)(1.0 / hv) : 0.0f;
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS)
        v[e] = w[e] * inv;
}

// y = d * x elementwise (the SIRT weights)
__global__ void __launch_bounds__(VEC_THREADS)
k_diag(const float *__restrict__ d, const float *__restrict__ x, float *__restrict__ y, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS)
        y[e] = d[e] * x[e];
}

// d = 1 / s where s > 0, else 0
__global__ void __launch_bounds__(VEC_THREADS) k_invert(float *d, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS)
        d[e] = d[e] > 0.0f ? 1.0f / d[e] : 0.0f;
}

__global__ void __launch_bounds__(VEC_THREADS) k_fill(float *d, int64_t n, float v) {
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS)
        d[e] = v;
}

// x = sum_i y_i V_i (FP64 coefficients, FP64 accumulation)
__global__ void __launch_bounds__(VEC_THREADS)
k_combine_f(const float *__restrict__ V, const double *__restrict__ y, int count, int64_t n, float *__restrict__ x) {
    for (int64_t e = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; e < n; e += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        double acc = 0.0;
        for (int i = 0; i < count; ++i) acc += y[i] * (double)V[(size_t)i * n + e];
        x[e] = (float)acc;
    }
}

// h[i] (+)= the dot of pass 2 (also returned in d for the axpy), one block per dot
__global__ void __launch_bounds__(RED_THREADS)
k_reduce_dots_add(const double *partial, double *d, double *h) {
    __shared__ double red[RED_THREADS / 32];
    const double s = reduce_partials(partial + (size_t)blockIdx.x * VEC_BLOCKS, VEC_BLOCKS, red);
    if (threadIdx.x == 0) {
        d[blockIdx.x] = s;
        h[blockIdx.x] += s;
    }
}

// A and the backprojector B on the solver layouts (volumes z-fastest,
// projections v-fastest), FP32.
struct GmresOperator {
    const DevGeom &g;
    cudaStream_t s;
    Tracker &tr;
    int64_t n, m;
    bool weighted = false;
    float *R = nullptr, *C = nullptr;    // SIRT weights (weighted only)
    float *tn = nullptr, *tm = nullptr, *wbuf = nullptr;

    cbct_status A(const float *x, float *y) {
        const Epilogue e{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
        ++tr.launches;
        ++tr.fwd;
        return launch_forward(g, x, y, CBCT_F32, e, s, true);
    }
    bool voxel_driven = false;

    // x = B y
    cbct_status B(const float *y, float *x) {
        if (voxel_driven) {
            ++tr.launches;
            ++tr.bwd;
            return launch_voxel_backproject(g, y, x, true, s);
        }
        const float *src = y;
        if (weighted) {
            k_diag<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(R, y, tn, n);
            ++tr.launches;
            src = tn;
        }
        cbct_status st = launch_weight(g, src, CBCT_F32, wbuf, s);
        if (st != CBCT_OK) return st;
        const Epilogue e{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
        st = launch_backward(g, wbuf, weighted ? tm : x, CBCT_F32, e, s, true, nullptr);
        if (st != CBCT_OK) return st;
        tr.launches += 2;
        ++tr.bwd;
        if (weighted) {
            k_diag<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(C, tm, x, m);
            ++tr.launches;
        }
        CBCT_CUDA_TRY(cudaGetLastError());
        return CBCT_OK;
    }
};

static cbct_status gmres_solve(const cbct_geometry *geom, const float *b, float *x, const cbct_solve_opts *o,
                               cbct_solve_report *rep, cudaStream_t s, bool ab) {
    const DevGeom &g = geom->dev;
    // m: length of a volume-side vector (padded z-fastest layout, pads kept at zero)
    const int64_t n = cbct_geometry_num_rays(geom), m = zf_len(geom->dev);
    const int iters = o->iters;
    const int64_t len = ab ? n : m;                 // Krylov vectors: projections (AB) or volumes (BA)
    const int ld = iters + 1;                       // Hessenberg: column-major (iters + 1) x iters
    Workspace ws(s);
    SolveIO io{};
    cbct_status st = setup_io(geom, b, x, ws, io);
    if (st != CBCT_OK) return st;
    Tracker tr;
    tr.s = s;
    GmresOperator op{g, s, tr, n, m};
    op.weighted = o->gmres_backprojector == 1;
    op.voxel_driven = o->gmres_backprojector == 2;
    float *V = nullptr, *w = nullptr, *yn = nullptr, *xm = nullptr;
    double *partial = nullptr, *pn = nullptr, *H = nullptr, *d2 = nullptr, *beta = nullptr, *ycoef = nullptr;
    if (ab) {
        CBCT_CUDA_TRY(ws.alloc(&V, (size_t)(iters + 1) * len));
        CBCT_CUDA_TRY(ws.alloc(&w, (size_t)len));
    } else {
        CBCT_CUDA_TRY(ws.alloc_volumes(&V, g, (size_t)iters + 1));
        CBCT_CUDA_TRY(ws.alloc_volumes(&w, g));
    }
    CBCT_CUDA_TRY(ws.alloc(&yn, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc_volumes(&xm, g));
    CBCT_CUDA_TRY(ws.alloc(&op.tn, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc_volumes(&op.tm, g));
    CBCT_CUDA_TRY(ws.alloc(&op.wbuf, (size_t)n));
    CBCT_CUDA_TRY(ws.alloc(&partial, (size_t)(iters + 1) * VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&pn, (size_t)VEC_BLOCKS));
    CBCT_CUDA_TRY(ws.alloc(&H, (size_t)ld * iters));
    CBCT_CUDA_TRY(ws.alloc(&d2, (size_t)iters + 1));
    CBCT_CUDA_TRY(ws.alloc(&beta, 1));
    CBCT_CUDA_TRY(ws.alloc(&ycoef, (size_t)iters));
    CBCT_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(double) * ld * iters, s));
    if (op.weighted) {                  // R = 1 / (A 1), C = 1 / (A^T 1)
        CBCT_CUDA_TRY(ws.alloc(&op.R, (size_t)n));
        CBCT_CUDA_TRY(ws.alloc_volumes(&op.C, g));
        st = launch_fill_volume(g, xm, 1.0f, s);         // the ones vector (pads stay zero)
        if (st != CBCT_OK) return st;
        st = op.A(xm, op.R);
        if (st != CBCT_OK) return st;
        k_invert<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(op.R, n);
        k_fill<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(yn, n, 1.0f);
        op.weighted = false;            // C = 1 / (A^T 1): the plain transpose of the ones
        st = op.B(yn, op.C);
        op.weighted = true;
        if (st != CBCT_OK) return st;
        k_invert<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(op.C, m);
        tr.launches += 4;
    }
    // r0 = b (AB) or B b (BA); beta = ||r0||; v_0 = r0 / beta
    if (ab) {
        CBCT_CUDA_TRY(cudaMemcpyAsync(w, io.b_dev, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    } else {
        st = op.B(io.b_dev, w);
        if (st != CBCT_OK) return st;
    }
    k_sumsq<float><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, len, pn);
    k_column_norm<<<1, RED_THREADS, 0, s>>>(pn, beta, -1);
    k_normalise<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, V, beta, len);
    tr.launches += 3;
    CBCT_CUDA_TRY(cudaGetLastError());

    for (int j = 0; j < iters; ++j) {
        const float *vj = V + (size_t)j * len;
        if (ab) {                       // w = A (B v_j)
            st = op.B(vj, xm);
            if (st == CBCT_OK) st = op.A(xm, w);
        } else {                        // w = B (A v_j)
            st = op.A(vj, yn);
            if (st == CBCT_OK) st = op.B(yn, w);
        }
        if (st != CBCT_OK) return st;
        double *hcol = H + (size_t)j * ld;
        // classical Gram-Schmidt, twice; FP64 dots
        k_multi_dot<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, V, j + 1, len, partial);
        k_reduce_dots<<<j + 1, RED_THREADS, 0, s>>>(partial, hcol, 0);
        k_multi_axpy<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, V, hcol, j + 1, len);
        k_multi_dot<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, V, j + 1, len, partial);
        k_reduce_dots_add<<<j + 1, RED_THREADS, 0, s>>>(partial, d2, hcol);
        k_multi_axpy<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, V, d2, j + 1, len);
        k_sumsq<float><<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, len, pn);
        k_column_norm<<<1, RED_THREADS, 0, s>>>(pn, hcol, j);
        k_normalise<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(w, V + (size_t)(j + 1) * len, hcol + j + 1, len);
        tr.launches += 9;
        CBCT_CUDA_TRY(cudaGetLastError());
    }

    // least squares min ||beta e_1 - Hbar_k y|| by Givens rotations on the host
    std::vector<double> h((size_t)ld * iters);
    double beta_h = 0.0;
    CBCT_CUDA_TRY(cudaMemcpyAsync(h.data(), H, sizeof(double) * ld * iters, cudaMemcpyDeviceToHost, s));
    CBCT_CUDA_TRY(cudaMemcpyAsync(&beta_h, beta, sizeof(double), cudaMemcpyDeviceToHost, s));
    CBCT_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<double> hist((size_t)3 * iters, 0.0), gv((size_t)iters + 1, 0.0), cs(iters), sn(iters);
    int done = 0;
    if (beta_h > 0.0 && std::isfinite(beta_h)) {
        gv[0] = beta_h;
        for (int j = 0; j < iters; ++j) {
            double *col = h.data() + (size_t)j * ld;
            bool ok = true;
            for (int i = 0; i <= j + 1; ++i) ok = ok && std::isfinite(col[i]);
            if (!ok) break;
            for (int i = 0; i < j; ++i) {                 // earlier rotations
                const double t = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t;
            }
            const double sub = col[j + 1];                  // h_{j+1,j}
            const double r = std::hypot(col[j], sub);
            if (r == 0.0) break;
            cs[j] = col[j] / r;
            sn[j] = sub / r;
            col[j] = r;
            col[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            done = j + 1;
            (ab ? hist[j] : hist[iters + j]) = std::fabs(gv[j + 1]);
            if (sub == 0.0) break;                          // Krylov space exhausted: exact solution
        }
    }
    // back substitution R y = g
    std::vector<double> y((size_t)std::max(done, 1), 0.0);
    for (int i = done - 1; i >= 0; --i) {
        double t = gv[i];
        for (int q = i + 1; q < done; ++q) t -= h[(size_t)q * ld + i] * y[q];
        y[i] = t / h[(size_t)i * ld + i];
    }
    if (done > 0) {
        CBCT_CUDA_TRY(cudaMemcpyAsync(ycoef, y.data(), sizeof(double) * done, cudaMemcpyHostToDevice, s));
        if (ab) {                       // x = B (V_k y)
            k_combine_f<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(V, ycoef, done, n, yn);
            ++tr.launches;
            st = op.B(yn, io.xz);
            if (st != CBCT_OK) return st;
        } else {
            k_combine_f<<<VEC_BLOCKS, VEC_THREADS, 0, s>>>(V, ycoef, done, m, io.xz);
            ++tr.launches;
        }
        CBCT_CUDA_TRY(cudaGetLastError());
    }
    st = finish_io(geom, io, s);
    if (st != CBCT_OK) return st;
    ++tr.launches;
    CBCT_CUDA_TRY(cudaStreamSynchronize(s));
    copy_report(rep, done, hist, iters);
    tr.fill(rep);
    if (rep) {
        rep->explicit_count = 0;
        rep->stopped_on_residual = 0;
    }
    return CBCT_OK;
}

static cbct_status dispatch_gmres(const cbct_geometry *g, const float *b, float *x, const cbct_solve_opts *o,
                                  cbct_solve_report *rep, cbct_stream stream, bool ab) {
    cbct_status st = check_solve_args(g, b, x, o);
    if (st != CBCT_OK) return st;
    if (o->storage != CBCT_F32) { set_error("GMRES supports FP32 storage only"); return CBCT_EINVAL; }
    if (o->explicit_residual) {
        set_error("GMRES: the explicit-residual monitor is not available (GMRES minimises its residual)");
        return CBCT_EINVAL;
    }
    if (o->gmres_backprojector < 0 || o->gmres_backprojector > 2) {
        set_error("GMRES: gmres_backprojector must be 0 (A^T), 1 (SIRT-weighted) or 2 (voxel-driven)");
        return CBCT_EINVAL;
    }
    return gmres_solve(g, b, x, o, rep, (cudaStream_t)stream, ab);
}

}  // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_ab_gmres_solve(const cbct_geometry *g, const float *b, float *x,
                                           const cbct_solve_opts *o, cbct_solve_report *rep, cbct_stream stream) {
    return dispatch_gmres(g, b, x, o, rep, stream, true);
}

extern "C" cbct_status cbct_ba_gmres_solve(const cbct_geometry *g, const float *b, float *x,
                                           const cbct_solve_opts *o, cbct_solve_report *rep, cbct_stream stream) {
    return dispatch_gmres(g, b, x, o, rep, stream, false);
}
