// Cone-beam projectors for sm_103a: the Siddon forward projection y = A x
// (one thread per detector pixel, Sec. 1 Eq. 1) and its exact transpose
// x = A^T y (volume bricks accumulated in shared memory).
//
// Both traverse rays with the same incremental Siddon step over voxel planes.
// Plane crossings come from the per-ray affine tables of DevGeom through one
// fma each, so a ray/voxel segment has the same FP32 length in both kernels:
// the backprojector is the transpose of the forward projector, not an
// approximation of it (the paper traces Krylov instabilities to unmatched
// backprojectors, Sec. 2.1.4 and Sec. 4).
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace cbct {

// ------------------------------------------------------------ ray traversal

// One axis of the traversal: current voxel index i, step s (+1/-1), index of
// the plane through which the ray leaves the current voxel (as float) and
// the alpha of that crossing.
struct Axis {
    int i, s;
    float p, e;
};

// Alpha at which a ray crosses plane p of one axis (plane spacing delta):
// (p * delta + P0) * I, rounded twice.  Both projectors use only this.
__device__ __forceinline__ float plane_alpha(float p, float delta, float P0, float I) {
    return __fmul_rn(__fmaf_rn(p, delta, P0), I);
}

// Clip alpha interval [amin, amax] to the slab between planes plo and phi.
// I == 0 marks a ray parallel to the planes whose voxel index is P0.
__device__ __forceinline__ void clip_slab(float P0, float I, float delta, int plo, int phi,
                                          float &amin, float &amax, bool &miss) {
    if (I == 0.0f) {
        if (!(P0 >= (float)plo && P0 < (float)phi)) miss = true;
        return;
    }
    const float a0 = plane_alpha((float)plo, delta, P0, I), a1 = plane_alpha((float)phi, delta, P0, I);
    amin = fmaxf(amin, fminf(a0, a1));
    amax = fminf(amax, fmaxf(a0, a1));
}

// Voxel index on one axis at alpha0 (the start of the traversal), restricted
// to voxels [lo, hi).  The estimate from the ray position is corrected by
// comparing with the crossing alphas themselves, so the start voxel is exactly
// the one whose alpha interval [entry, exit) contains alpha0.
__device__ __forceinline__ Axis axis_start(float P0, float I, float delta, float alpha0, int lo, int hi) {
    Axis st;
    if (I == 0.0f) {            // parallel: fixed index, never crossed
        st.i = (int)P0;
        st.s = 0;
        st.p = 0.0f;
        st.e = FLT_MAX;
        return st;
    }
    // position relative to the lower face: alpha * d - P0 = alpha / I - P0
    int i = (int)floorf((__fdividef(alpha0, I) - P0) / delta);
    i = max(lo, min(hi - 1, i));
    if (I > 0.0f) {             // alpha grows with the plane index: voxel i = [alpha(i), alpha(i+1))
        if (i + 1 < hi && plane_alpha((float)(i + 1), delta, P0, I) <= alpha0) ++i;
        if (i > lo && plane_alpha((float)i, delta, P0, I) > alpha0) --i;
        st.s = 1;
        st.p = (float)(i + 1);
    } else {                    // alpha falls with the plane index: voxel i = [alpha(i+1), alpha(i))
        if (i > lo && plane_alpha((float)i, delta, P0, I) <= alpha0) --i;
        if (i + 1 < hi && plane_alpha((float)(i + 1), delta, P0, I) > alpha0) ++i;
        st.s = -1;
        st.p = (float)i;
    }
    st.i = i;
    st.e = plane_alpha(st.p, delta, P0, I);
    return st;
}

// Traverse ray (xy, z) through the voxel box [lo, hi) (per axis) and call
// f(linear index inside the box, alpha length) for every segment, in order.
// Linear index = ((k - lo_z) * sy + (j - lo_y)) * sx + (i - lo_x).
// Returns false if the ray misses the box.
template <typename F>
__device__ __forceinline__ bool trace_box(const DevGeom &g, float4 xy, float2 z, int lox, int hix, int loy,
                                          int hiy, int loz, int hiz, int sxs, int sys, F &&f) {
    float amin = -FLT_MAX, amax = FLT_MAX;
    bool miss = false;
    clip_slab(xy.x, xy.y, g.dx, lox, hix, amin, amax, miss);
    clip_slab(xy.z, xy.w, g.dy, loy, hiy, amin, amax, miss);
    clip_slab(z.x, z.y, g.dz, loz, hiz, amin, amax, miss);
    if (miss || !(amin < amax)) return false;

    Axis ax = axis_start(xy.x, xy.y, g.dx, amin, lox, hix);
    Axis ay = axis_start(xy.z, xy.w, g.dy, amin, loy, hiy);
    Axis az = axis_start(z.x, z.y, g.dz, amin, loz, hiz);
    int idx = ((az.i - loz) * sys + (ay.i - loy)) * sxs + (ax.i - lox);
    const int stride_y = sxs, stride_z = sxs * sys;
    float cur = amin;
    const int maxsteps = (hix - lox) + (hiy - loy) + (hiz - loz) + 1;
#pragma unroll 1
    for (int n = 0; n < maxsteps; ++n) {
        const float e = fminf(fminf(ax.e, ay.e), az.e);
        f(idx, e - cur);
        cur = e;
        if (e == ax.e) {
            ax.i += ax.s;
            if ((unsigned)(ax.i - lox) >= (unsigned)(hix - lox)) break;
            idx += ax.s;
            ax.p += (float)ax.s;
            ax.e = plane_alpha(ax.p, g.dx, xy.x, xy.y);
        } else if (e == ay.e) {
            ay.i += ay.s;
            if ((unsigned)(ay.i - loy) >= (unsigned)(hiy - loy)) break;
            idx += ay.s * stride_y;
            ay.p += (float)ay.s;
            ay.e = plane_alpha(ay.p, g.dy, xy.z, xy.w);
        } else {
            az.i += az.s;
            if ((unsigned)(az.i - loz) >= (unsigned)(hiz - loz)) break;
            idx += az.s * stride_z;
            az.p += (float)az.s;
            az.e = plane_alpha(az.p, g.dz, z.x, z.y);
        }
    }
    return true;
}

// ------------------------------------------------------------- forward A x

constexpr int FWD_TX = 32, FWD_TY = 4, FWD_THREADS = FWD_TX * FWD_TY;

template <typename T, bool COMP>
__global__ void __launch_bounds__(FWD_THREADS)
forward_kernel(DevGeom g, const T *__restrict__ vol, T *__restrict__ proj, Epilogue epi) {
    __shared__ double red[FWD_THREADS / 32];
    if (epi.stop && *epi.stop) return;
    const int iu = blockIdx.x * FWD_TX + (threadIdx.x % FWD_TX);
    const int iv = blockIdx.y * FWD_TY + (threadIdx.x / FWD_TX);
    const int a = blockIdx.z;
    const bool valid = iu < g.nu && iv < g.nv;
    float acc = 0.0f, comp = 0.0f;
    if (valid) {
        const float4 xy = g.ray_xy[(size_t)a * g.nu + iu];
        const float2 zt = g.ray_z[iv];
        auto seg = [&](int idx, float len) {
            const float term = len * Storage<T>::load(vol + idx);
            if (COMP) {          // Kahan-compensated running sum
                const float yk = term - comp;
                const float t = acc + yk;
                comp = (t - acc) - yk;
                acc = t;
            } else {
                acc += term;
            }
        };
        trace_box(g, xy, zt, 0, g.nx, 0, g.ny, 0, g.nz, g.nx, g.ny, seg);
        acc *= g.ray_len[(size_t)iv * g.nu + iu];
    }
    double sq = 0.0;
    if (valid) {
        const size_t r = ((size_t)a * g.nv + iv) * g.nu + iu;
        const double bcoef = epi_b(epi);
        double out = epi_a(epi) * (double)acc;
        if (bcoef != 0.0) {
            const T *oldp = epi.old ? (const T *)epi.old : (const T *)proj;
            out += bcoef * (double)Storage<T>::ld_plain(oldp + r);
        }
        const float stored = Storage<T>::round((float)out);
        Storage<T>::store(proj + r, stored);
        sq = (double)stored * (double)stored;
    }
    if (epi.partial) {
        const double s = block_sum<FWD_THREADS>(sq, red);
        if (threadIdx.x == 0) {
            const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            epi.partial[b] = s;
        }
    }
}

__global__ void __launch_bounds__(FWD_THREADS)
count_kernel(DevGeom g, unsigned long long *count) {
    __shared__ double red[FWD_THREADS / 32];
    const int iu = blockIdx.x * FWD_TX + (threadIdx.x % FWD_TX);
    const int iv = blockIdx.y * FWD_TY + (threadIdx.x / FWD_TX);
    const int a = blockIdx.z;
    int c = 0;
    if (iu < g.nu && iv < g.nv) {
        const float4 xy = g.ray_xy[(size_t)a * g.nu + iu];
        const float2 zt = g.ray_z[iv];
        auto seg = [&](int, float len) { c += len > 0.0f; };
        trace_box(g, xy, zt, 0, g.nx, 0, g.ny, 0, g.nz, g.nx, g.ny, seg);
    }
    const double s = block_sum<FWD_THREADS>((double)c, red);
    if (threadIdx.x == 0) atomicAdd(count, (unsigned long long)s);
}

static dim3 forward_grid(const DevGeom &g) {
    return dim3((g.nu + FWD_TX - 1) / FWD_TX, (g.nv + FWD_TY - 1) / FWD_TY, g.nangles);
}

int forward_num_blocks(const DevGeom &g) {
    dim3 gr = forward_grid(g);
    return (int)(gr.x * gr.y * gr.z);
}

cbct_status launch_forward(const DevGeom &g, const void *x, void *y, cbct_dtype t,
                           const Epilogue &epi, cudaStream_t s) {
    const dim3 grid = forward_grid(g);
    switch (t) {
    case CBCT_F32:
        forward_kernel<float, false><<<grid, FWD_THREADS, 0, s>>>(g, (const float *)x, (float *)y, epi);
        break;
    case CBCT_F16:
        forward_kernel<__half, true><<<grid, FWD_THREADS, 0, s>>>(g, (const __half *)x, (__half *)y, epi);
        break;
    case CBCT_BF16:
        forward_kernel<__nv_bfloat16, true><<<grid, FWD_THREADS, 0, s>>>(
            g, (const __nv_bfloat16 *)x, (__nv_bfloat16 *)y, epi);
        break;
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

cbct_status launch_count(const DevGeom &g, unsigned long long *count_dev, cudaStream_t s) {
    count_kernel<<<forward_grid(g), FWD_THREADS, 0, s>>>(g, count_dev);
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

// ---------------------------------------------------------- transpose A^T y
//
// One CTA owns a brick of BX x BY x BZ voxels, accumulated in shared memory.
// For every angle it finds the detector window onto which the brick projects
// (the eight projected corners), then each thread takes rays of that window
// and walks them through the brick with the forward traversal, adding
// len * |d'| * y to the voxels it meets.  After the last angle the brick is
// written once (fused epilogue), so no global atomics are needed.

constexpr int BWD_BX = 16, BWD_BY = 16, BWD_BZ = 8, BWD_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(BWD_THREADS)
backward_kernel(DevGeom g, const T *__restrict__ proj, T *__restrict__ vol, Epilogue epi) {
    __shared__ float sacc[BWD_BZ * BWD_BY * BWD_BX];
    __shared__ double red[BWD_THREADS / 32];
    if (epi.stop && *epi.stop) return;
    const int bx = blockIdx.x * BWD_BX, by = blockIdx.y * BWD_BY, bz = blockIdx.z * BWD_BZ;
    const int ex = min(BWD_BX, g.nx - bx), ey = min(BWD_BY, g.ny - by), ez = min(BWD_BZ, g.nz - bz);
    for (int q = threadIdx.x; q < BWD_BZ * BWD_BY * BWD_BX; q += BWD_THREADS) sacc[q] = 0.0f;
    __syncthreads();

    // brick corners (mm) for the footprint windows
    const float x0 = g.bx0 + bx * g.dx, x1 = g.bx0 + (bx + ex) * g.dx;
    const float y0 = g.by0 + by * g.dy, y1 = g.by0 + (by + ey) * g.dy;
    const float z0 = g.bz0 + bz * g.dz, z1 = g.bz0 + (bz + ez) * g.dz;
    const float cu = 0.5f * (g.nu - 1), cv = 0.5f * (g.nv - 1);

    for (int a = 0; a < g.nangles; ++a) {
        const float2 cs = g.trig[a];
        float umin = FLT_MAX, umax = -FLT_MAX, vmin = FLT_MAX, vmax = -FLT_MAX;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float px = (c & 1) ? x1 : x0, py = (c & 2) ? y1 : y0;
            const float along = g.dso - (px * cs.x + py * cs.y);   // > 0: source outside
            const float across = -px * cs.y + py * cs.x;
            const float mag = g.dsd / along;
            const float u = across * mag;
            umin = fminf(umin, u);
            umax = fmaxf(umax, u);
            vmin = fminf(vmin, fminf(z0 * mag, z1 * mag));
            vmax = fmaxf(vmax, fmaxf(z0 * mag, z1 * mag));
        }
        const int iu0 = max(0, (int)ceilf(umin / g.du + cu - 0.01f));
        const int iu1 = min(g.nu - 1, (int)floorf(umax / g.du + cu + 0.01f));
        const int iv0 = max(0, (int)ceilf(vmin / g.dv + cv - 0.01f));
        const int iv1 = min(g.nv - 1, (int)floorf(vmax / g.dv + cv + 0.01f));
        if (iu0 > iu1 || iv0 > iv1) continue;
        const int nwu = iu1 - iu0 + 1;
        const int nwin = nwu * (iv1 - iv0 + 1);
        const T *pa = proj + (size_t)a * g.nv * g.nu;
        const float4 *xya = g.ray_xy + (size_t)a * g.nu;
        for (int r = threadIdx.x; r < nwin; r += BWD_THREADS) {
            const int iv = iv0 + r / nwu, iu = iu0 + r % nwu;
            const size_t pix = (size_t)iv * g.nu + iu;
            const float w = Storage<T>::load(pa + pix) * g.ray_len[pix];
            if (w == 0.0f) continue;
            const float4 xy = xya[iu];
            const float2 zt = g.ray_z[iv];
            auto seg = [&](int idx, float len) { atomicAdd(&sacc[idx], len * w); };
            trace_box(g, xy, zt, bx, bx + ex, by, by + ey, bz, bz + ez, BWD_BX, BWD_BY, seg);
        }
    }
    __syncthreads();

    const double acoef = epi_a(epi), bcoef = epi_b(epi);
    double sq = 0.0;
    for (int q = threadIdx.x; q < BWD_BZ * BWD_BY * BWD_BX; q += BWD_THREADS) {
        const int i = q % BWD_BX, j = (q / BWD_BX) % BWD_BY, k = q / (BWD_BX * BWD_BY);
        if (i >= ex || j >= ey || k >= ez) continue;
        const size_t v = ((size_t)(bz + k) * g.ny + (by + j)) * g.nx + (bx + i);
        double out = acoef * (double)sacc[q];
        if (bcoef != 0.0) {
            const T *oldp = epi.old ? (const T *)epi.old : (const T *)vol;
            out += bcoef * (double)Storage<T>::ld_plain(oldp + v);
        }
        const float stored = Storage<T>::round((float)out);
        Storage<T>::store(vol + v, stored);
        sq += (double)stored * (double)stored;
    }
    if (epi.partial) {
        const double s = block_sum<BWD_THREADS>(sq, red);
        if (threadIdx.x == 0) {
            const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            epi.partial[b] = s;
        }
    }
}

static dim3 backward_grid(const DevGeom &g) {
    return dim3((g.nx + BWD_BX - 1) / BWD_BX, (g.ny + BWD_BY - 1) / BWD_BY, (g.nz + BWD_BZ - 1) / BWD_BZ);
}

int backward_num_blocks(const DevGeom &g) {
    dim3 gr = backward_grid(g);
    return (int)(gr.x * gr.y * gr.z);
}

cbct_status launch_backward(const DevGeom &g, const void *y, void *x, cbct_dtype t,
                            const Epilogue &epi, cudaStream_t s) {
    const dim3 grid = backward_grid(g);
    switch (t) {
    case CBCT_F32:
        backward_kernel<float><<<grid, BWD_THREADS, 0, s>>>(g, (const float *)y, (float *)x, epi);
        break;
    case CBCT_F16:
        backward_kernel<__half><<<grid, BWD_THREADS, 0, s>>>(g, (const __half *)y, (__half *)x, epi);
        break;
    case CBCT_BF16:
        backward_kernel<__nv_bfloat16><<<grid, BWD_THREADS, 0, s>>>(
            g, (const __nv_bfloat16 *)y, (__nv_bfloat16 *)x, epi);
        break;
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

}  // namespace cbct

using namespace cbct;

static cbct_status check_pair(const cbct_geometry *g, const void *a, const void *b, cbct_dtype t) {
    if (!g || !a || !b) { set_error("null geometry or buffer"); return CBCT_EINVAL; }
    if (t != CBCT_F32 && t != CBCT_F16 && t != CBCT_BF16) { set_error("unknown dtype"); return CBCT_EINVAL; }
    return CBCT_OK;
}

extern "C" cbct_status cbct_project(const cbct_geometry *g, const void *x, void *y, cbct_dtype t,
                                    cbct_stream stream) {
    cbct_status st = check_pair(g, x, y, t);
    if (st != CBCT_OK) return st;
    Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
    return launch_forward(g->dev, x, y, t, epi, (cudaStream_t)stream);
}

extern "C" cbct_status cbct_backproject(const cbct_geometry *g, const void *y, void *x, cbct_dtype t,
                                        cbct_stream stream) {
    cbct_status st = check_pair(g, y, x, t);
    if (st != CBCT_OK) return st;
    Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
    return launch_backward(g->dev, y, x, t, epi, (cudaStream_t)stream);
}

extern "C" cbct_status cbct_count_nnz(const cbct_geometry *g, int64_t *nnz, cbct_stream stream) {
    if (!g || !nnz) { set_error("cbct_count_nnz: null argument"); return CBCT_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync(&d, sizeof(unsigned long long), s));
    cbct_status st = CBCT_OK;
    cudaError_t err = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
    if (err == cudaSuccess) {
        st = launch_count(g->dev, d, s);
        unsigned long long h = 0;
        if (st == CBCT_OK) {
            err = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s);
            if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        }
        *nnz = (int64_t)h;
    }
    cudaFreeAsync(d, s);
    if (err != cudaSuccess) return cuda_fail(err, "cbct_count_nnz");
    return st;
}
