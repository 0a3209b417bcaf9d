// Cone-beam projectors for sm_103a: the Siddon forward projection y = A x
// (Sec. 1, Eq. 1: one ray per detector pixel) and its exact transpose
// x = A^T y.
//
// Work layout ("ray-column warps").  In a circular cone-beam scan every ray of
// one detector column (angle a, column iu) has the same projection onto the
// xy plane, so all of them cross the x and y voxel planes at the same alpha
// (the x/y tables depend on (a, iu) only).  A warp therefore takes 32
// consecutive detector rows of one column: the x/y plane stepping is
// identical in all lanes (no divergence), and each lane only tracks its own z
// crossings, which are rare (|dz/d| <= the cone half-angle).  Volumes are read
// in a z-fastest layout x[j][i][k] so that the 32 lanes of a warp, which sit
// at ~17 consecutive k of one voxel column, gather one contiguous run.
//
// Both kernels walk the same traversal (trace_column) and take every plane
// crossing from the per-ray tables of DevGeom through plane_alpha, so a
// ray/voxel segment has the same FP32 length in both: the backprojector is the
// transpose of the forward projector, not an approximation of it (the paper
// traces Krylov instabilities to unmatched backprojectors, Sec. 2.1.4, Sec. 4).
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace cbct {

// ------------------------------------------------------------ ray traversal

// One axis of one ray: offset f = plane(pq) - q, inverse direction I, and the
// index pq of the plane nearest to the ray origin (the fixed voxel index when
// I == 0, a ray parallel to the axis' planes).
struct RayAxis {
    float f, I, pq;
};

// Alpha at which a ray crosses plane pq + r of one axis (plane spacing delta):
// (r * delta + f) * I, rounded twice.  Both projectors use only this.
__device__ __forceinline__ float plane_alpha(float r, float delta, const RayAxis &a) {
    return __fmul_rn(__fmaf_rn(r, delta, a.f), a.I);
}

// One axis of the traversal: current voxel index i, step s (+1/-1, 0 when the
// ray is parallel to the axis' planes), index of the plane through which the
// ray leaves the current voxel (relative to pq, as float) and the alpha of
// that crossing.
struct Axis {
    int i, s;
    float r, e;
};

// Clip alpha interval [amin, amax] to the slab between planes plo and phi.
__device__ __forceinline__ void clip_slab(const RayAxis &ra, float delta, int plo, int phi, float &amin,
                                          float &amax, bool &miss) {
    if (ra.I == 0.0f) {
        if (!(ra.pq >= (float)plo && ra.pq < (float)phi)) miss = true;
        return;
    }
    const float a0 = plane_alpha((float)plo - ra.pq, delta, ra), a1 = plane_alpha((float)phi - ra.pq, delta, ra);
    amin = fmaxf(amin, fminf(a0, a1));
    amax = fminf(amax, fmaxf(a0, a1));
}

// Voxel index on one axis at alpha0, within [lo - 1, hi] (lo - 1 and hi stand
// for "before" and "beyond" the range).  The estimate from the ray position is
// corrected by comparing with the crossing alphas themselves, so the result is
// exactly the voxel whose alpha interval [entry, exit) contains alpha0.  The
// exit crossing is returned; it is FLT_MAX when the ray is outside the range
// and moving away from it.
__device__ __forceinline__ Axis axis_start(const RayAxis &ra, float delta, float alpha0, int lo, int hi) {
    Axis st;
    if (ra.I == 0.0f) {         // parallel: fixed index, never crossed
        st.i = (int)ra.pq;
        st.s = 0;
        st.r = 0.0f;
        st.e = FLT_MAX;
        return st;
    }
    // plane coordinate of the ray at alpha0: pq + (alpha0 / I - f) / delta
    int i = (int)floorf(ra.pq + (__fdividef(alpha0, ra.I) - ra.f) / delta);
    i = max(lo - 1, min(hi, i));
    auto al = [&](int p) { return plane_alpha((float)p - ra.pq, delta, ra); };
    if (ra.I > 0.0f) {          // alpha grows with the plane index: voxel i = [alpha(i), alpha(i+1))
        if (i < hi && al(i + 1) <= alpha0) ++i;
        if (i >= lo && al(i) > alpha0) --i;
        st.s = 1;
        st.r = (float)(i + 1) - ra.pq;
        st.e = i < hi ? plane_alpha(st.r, delta, ra) : FLT_MAX;
    } else {                    // alpha falls with the plane index: voxel i = [alpha(i+1), alpha(i))
        if (i >= lo && al(i) <= alpha0) --i;
        if (i < hi && al(i + 1) > alpha0) ++i;
        st.s = -1;
        st.r = (float)i - ra.pq;
        st.e = i >= lo ? plane_alpha(st.r, delta, ra) : FLT_MAX;
    }
    st.i = i;
    return st;
}

// Walk one ray through the box [lox,hix) x [loy,hiy) x [loz,hiz) of voxels.
// x/y are stepped together by the whole warp (the xy tables are the same in
// every lane); z is per lane.  For every segment inside the box it calls
//     f(i, j, k, alpha_length)
// in order along the ray.  Lanes whose ray lies outside the box in z simply
// make no calls.  Returns false (uniformly) if the xy projection misses the box.
template <typename F>
__device__ __forceinline__ bool trace_column(const DevGeom &g, const RayAxis &rx, const RayAxis &ry,
                                             const RayAxis &rz, int lox, int hix, int loy, int hiy, int loz,
                                             int hiz, F &&f) {
    float amin = -FLT_MAX, amax = FLT_MAX;
    bool miss = false;
    clip_slab(rx, g.dx, lox, hix, amin, amax, miss);
    clip_slab(ry, g.dy, loy, hiy, amin, amax, miss);
    if (miss || !(amin < amax)) return false;

    Axis ax = axis_start(rx, g.dx, amin, lox, hix);
    Axis ay = axis_start(ry, g.dy, amin, loy, hiy);
    Axis az = axis_start(rz, g.dz, amin, loz, hiz);
    if (az.s == 0 && (az.i < loz || az.i >= hiz)) az.i = loz - 1;   // parallel outside: never inside
    float cur = amin;
    const int maxsteps = (hix - lox) + (hiy - loy) + 1;
#pragma unroll 1
    for (int n = 0; n < maxsteps; ++n) {
        const float e = fminf(ax.e, ay.e);
        // z crossings of this lane inside the current xy cell
#pragma unroll 1
        while (az.e < e) {
            if (az.i >= loz && az.i < hiz) f(ax.i, ay.i, az.i, az.e - cur);
            cur = az.e;
            az.i += az.s;
            az.r += (float)az.s;
            az.e = (az.i >= loz && az.i < hiz) ? plane_alpha(az.r, g.dz, rz) : FLT_MAX;
        }
        if (az.i >= loz && az.i < hiz) f(ax.i, ay.i, az.i, e - cur);
        cur = e;
        if (e == ax.e) {
            ax.i += ax.s;
            if ((unsigned)(ax.i - lox) >= (unsigned)(hix - lox)) break;
            ax.r += (float)ax.s;
            ax.e = plane_alpha(ax.r, g.dx, rx);
        } else {
            ay.i += ay.s;
            if ((unsigned)(ay.i - loy) >= (unsigned)(hiy - loy)) break;
            ay.r += (float)ay.s;
            ay.e = plane_alpha(ay.r, g.dy, ry);
        }
    }
    return true;
}

// Table entries of ray (a, iu, iv); rows outside [0, nv) get a z axis that is
// parallel and outside every box, so the lane follows the warp without effect.
__device__ __forceinline__ void load_ray(const DevGeom &g, int a, int iu, int iv, bool row_ok, RayAxis &rx,
                                         RayAxis &ry, RayAxis &rz) {
    const float4 xy = g.ray_xy[(size_t)a * g.nu + iu];
    const float2 q = g.ray_xyq[(size_t)a * g.nu + iu];
    rx = RayAxis{xy.x, xy.y, q.x};
    ry = RayAxis{xy.z, xy.w, q.y};
    if (row_ok) {
        const float4 z = g.ray_z[iv];
        rz = RayAxis{z.x, z.y, z.z};
    } else {
        rz = RayAxis{0.0f, 0.0f, (float)(g.nz + 1)};
    }
}

// ------------------------------------------------------------- forward A x
//
// Block = 8 warps = 8 adjacent detector columns (iu) x 32 detector rows (iv)
// of one angle.  The volume is read z-fastest: vol[(j * nx + i) * nz + k].

constexpr int FWD_ROWS = 32, FWD_COLS = 8, FWD_THREADS = FWD_ROWS * FWD_COLS;

template <typename T, bool COMP>
__global__ void __launch_bounds__(FWD_THREADS)
forward_kernel(DevGeom g, const T *__restrict__ vol, T *__restrict__ proj, Epilogue epi) {
    __shared__ double red[FWD_THREADS / 32];
    if (epi.stop && *epi.stop) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int iu = blockIdx.x * FWD_COLS + warp;
    const int iv = blockIdx.y * FWD_ROWS + lane;
    const int a = blockIdx.z;
    const bool col_ok = iu < g.nu;            // uniform across the warp
    const bool valid = col_ok && iv < g.nv;
    float acc = 0.0f, comp = 0.0f;
    if (col_ok) {
        RayAxis rx, ry, rz;
        load_ray(g, a, iu, iv, valid, rx, ry, rz);
        const size_t nz = (size_t)g.nz, row = (size_t)g.nx * g.nz;
        auto seg = [&](int i, int j, int k, float len) {
            const float term = len * Storage<T>::load(vol + (size_t)j * row + (size_t)i * nz + k);
            if (COMP) {          // Kahan-compensated running sum
                const float yk = term - comp;
                const float t = acc + yk;
                comp = (t - acc) - yk;
                acc = t;
            } else {
                acc += term;
            }
        };
        trace_column(g, rx, ry, rz, 0, g.nx, 0, g.ny, 0, g.nz, seg);
        if (valid) acc *= g.ray_len[(size_t)iv * g.nu + iu];
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int iu = blockIdx.x * FWD_COLS + warp;
    const int iv = blockIdx.y * FWD_ROWS + lane;
    const int a = blockIdx.z;
    int c = 0;
    if (iu < g.nu) {
        RayAxis rx, ry, rz;
        load_ray(g, a, iu, iv, iv < g.nv, rx, ry, rz);
        auto seg = [&](int, int, int, float len) { c += len > 0.0f; };
        trace_column(g, rx, ry, rz, 0, g.nx, 0, g.ny, 0, g.nz, seg);
    }
    const double s = block_sum<FWD_THREADS>((double)c, red);
    if (threadIdx.x == 0) atomicAdd(count, (unsigned long long)s);
}

static dim3 forward_grid(const DevGeom &g) {
    return dim3((g.nu + FWD_COLS - 1) / FWD_COLS, (g.nv + FWD_ROWS - 1) / FWD_ROWS, g.nangles);
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
// One CTA owns a brick of BX x BY x BZ voxels, accumulated in shared memory
// (z fastest).  For every angle each warp finds the detector window onto which
// the brick projects (its eight corners), cuts it into tasks of one detector
// column x 32 rows, and walks those rays through the brick with the forward
// traversal, adding len * |d'| * y to the voxels they meet.  Warps move from
// angle to angle independently.  After the last angle the brick is written
// once (fused epilogue, either volume layout), so no global atomics are needed.

constexpr int BWD_BX = 16, BWD_BY = 16, BWD_BZ = 32, BWD_THREADS = 256;

template <typename T, bool ZFAST>
__global__ void __launch_bounds__(BWD_THREADS)
backward_kernel(DevGeom g, const T *__restrict__ proj, T *__restrict__ vol, Epilogue epi) {
    __shared__ float sacc[BWD_BY * BWD_BX * BWD_BZ];
    __shared__ double red[BWD_THREADS / 32];
    if (epi.stop && *epi.stop) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = blockIdx.x * BWD_BX, by = blockIdx.y * BWD_BY, bz = blockIdx.z * BWD_BZ;
    const int ex = min(BWD_BX, g.nx - bx), ey = min(BWD_BY, g.ny - by), ez = min(BWD_BZ, g.nz - bz);
    for (int q = threadIdx.x; q < BWD_BY * BWD_BX * BWD_BZ; q += BWD_THREADS) sacc[q] = 0.0f;
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
            umin = fminf(umin, across * mag);
            umax = fmaxf(umax, across * mag);
            vmin = fminf(vmin, fminf(z0 * mag, z1 * mag));
            vmax = fmaxf(vmax, fmaxf(z0 * mag, z1 * mag));
        }
        const int iu0 = max(0, (int)ceilf(umin / g.du + cu - 0.01f));
        const int iu1 = min(g.nu - 1, (int)floorf(umax / g.du + cu + 0.01f));
        const int iv0 = max(0, (int)ceilf(vmin / g.dv + cv - 0.01f));
        const int iv1 = min(g.nv - 1, (int)floorf(vmax / g.dv + cv + 0.01f));
        if (iu0 > iu1 || iv0 > iv1) continue;
        const int nblk = (iv1 - iv0 + 32) / 32;
        const int ntask = (iu1 - iu0 + 1) * nblk;
        const T *pa = proj + (size_t)a * g.nv * g.nu;
        for (int task = warp; task < ntask; task += BWD_THREADS / 32) {
            const int iu = iu0 + task / nblk;
            const int iv = iv0 + (task % nblk) * 32 + lane;
            const bool row_ok = iv <= iv1;      // rows outside the window never enter the brick
            float w = 0.0f;
            if (row_ok) {
                const size_t pix = (size_t)iv * g.nu + iu;
                w = Storage<T>::load(pa + pix) * g.ray_len[pix];
            }
            if (!__any_sync(0xffffffffu, w != 0.0f)) continue;
            RayAxis rx, ry, rz;
            load_ray(g, a, iu, iv, row_ok, rx, ry, rz);
            auto seg = [&](int i, int j, int k, float len) {
                if (w != 0.0f && len > 0.0f)
                    atomicAdd(&sacc[((j - by) * BWD_BX + (i - bx)) * BWD_BZ + (k - bz)], len * w);
            };
            trace_column(g, rx, ry, rz, bx, bx + ex, by, by + ey, bz, bz + ez, seg);
        }
    }
    __syncthreads();

    const double acoef = epi_a(epi), bcoef = epi_b(epi);
    double sq = 0.0;
    for (int q = threadIdx.x; q < BWD_BY * BWD_BX * BWD_BZ; q += BWD_THREADS) {
        int i, j, k;
        if (ZFAST) {            // output x[j][i][k]: walk k fastest
            k = q % BWD_BZ;
            i = (q / BWD_BZ) % BWD_BX;
            j = q / (BWD_BZ * BWD_BX);
        } else {                // output x[k][j][i]: walk i fastest
            i = q % BWD_BX;
            j = (q / BWD_BX) % BWD_BY;
            k = q / (BWD_BX * BWD_BY);
        }
        if (i >= ex || j >= ey || k >= ez) continue;
        const int sidx = (j * BWD_BX + i) * BWD_BZ + k;
        const size_t v = ZFAST ? ((size_t)(by + j) * g.nx + (bx + i)) * g.nz + (bz + k)
                               : ((size_t)(bz + k) * g.ny + (by + j)) * g.nx + (bx + i);
        double out = acoef * (double)sacc[sidx];
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

template <bool ZF>
static void launch_backward_t(const DevGeom &g, const void *y, void *x, cbct_dtype t, const Epilogue &epi,
                              cudaStream_t s) {
    const dim3 grid = backward_grid(g);
    switch (t) {
    case CBCT_F32:
        backward_kernel<float, ZF><<<grid, BWD_THREADS, 0, s>>>(g, (const float *)y, (float *)x, epi);
        break;
    case CBCT_F16:
        backward_kernel<__half, ZF><<<grid, BWD_THREADS, 0, s>>>(g, (const __half *)y, (__half *)x, epi);
        break;
    case CBCT_BF16:
        backward_kernel<__nv_bfloat16, ZF><<<grid, BWD_THREADS, 0, s>>>(
            g, (const __nv_bfloat16 *)y, (__nv_bfloat16 *)x, epi);
        break;
    }
}

cbct_status launch_backward(const DevGeom &g, const void *y, void *x, cbct_dtype t, const Epilogue &epi,
                            cudaStream_t s, bool zfast) {
    if (zfast)
        launch_backward_t<true>(g, y, x, t, epi, s);
    else
        launch_backward_t<false>(g, y, x, t, epi, s);
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

// ------------------------------------------------------- volume re-layout
//
// Standard x[k][j][i] <-> z-fastest x[j][i][k]: for each j a (k, i) plane is
// transposed through a 32 x 33 shared tile (coalesced on both sides).

template <typename T, bool TO_ZFAST>
__global__ void __launch_bounds__(256) relayout_kernel(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny,
                                                       int nz) {
    __shared__ T tile[32][33];
    const int j = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    if (TO_ZFAST) {                 // src [k][j][i] -> dst [j][i][k]
        const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
        for (int r = ty; r < 32; r += 8) {
            const int k = k0 + r, i = i0 + tx;
            if (k < nz && i < nx) tile[r][tx] = src[((size_t)k * ny + j) * nx + i];
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r, k = k0 + tx;
            if (i < nx && k < nz) dst[((size_t)j * nx + i) * nz + k] = tile[tx][r];
        }
    } else {                        // src [j][i][k] -> dst [k][j][i]
        const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r, k = k0 + tx;
            if (i < nx && k < nz) tile[r][tx] = src[((size_t)j * nx + i) * nz + k];
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int k = k0 + r, i = i0 + tx;
            if (k < nz && i < nx) dst[((size_t)k * ny + j) * nx + i] = tile[tx][r];
        }
    }
}

template <typename T>
static void launch_relayout_t(const DevGeom &g, const void *src, void *dst, bool to_zfast, cudaStream_t s) {
    if (to_zfast) {
        const dim3 grid((g.nx + 31) / 32, (g.nz + 31) / 32, g.ny);
        relayout_kernel<T, true><<<grid, 256, 0, s>>>((const T *)src, (T *)dst, g.nx, g.ny, g.nz);
    } else {
        const dim3 grid((g.nz + 31) / 32, (g.nx + 31) / 32, g.ny);
        relayout_kernel<T, false><<<grid, 256, 0, s>>>((const T *)src, (T *)dst, g.nx, g.ny, g.nz);
    }
}

cbct_status launch_relayout(const DevGeom &g, const void *src, void *dst, cbct_dtype t, bool to_zfast,
                            cudaStream_t s) {
    switch (t) {
    case CBCT_F32: launch_relayout_t<float>(g, src, dst, to_zfast, s); break;
    case CBCT_F16: launch_relayout_t<__half>(g, src, dst, to_zfast, s); break;
    case CBCT_BF16: launch_relayout_t<__nv_bfloat16>(g, src, dst, to_zfast, s); break;
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
    cudaStream_t s = (cudaStream_t)stream;
    // the forward kernel reads the z-fastest layout: re-lay the caller's volume first
    void *tmp = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)cbct_geometry_num_voxels(g) * dtype_size(t), s));
    st = launch_relayout(g->dev, x, tmp, t, true, s);
    if (st == CBCT_OK) {
        Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
        st = launch_forward(g->dev, tmp, y, t, epi, s);
    }
    cudaFreeAsync(tmp, s);
    return st;
}

extern "C" cbct_status cbct_backproject(const cbct_geometry *g, const void *y, void *x, cbct_dtype t,
                                        cbct_stream stream) {
    cbct_status st = check_pair(g, y, x, t);
    if (st != CBCT_OK) return st;
    Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
    return launch_backward(g->dev, y, x, t, epi, (cudaStream_t)stream, false);
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
