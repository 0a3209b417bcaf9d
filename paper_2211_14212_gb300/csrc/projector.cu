// Cone-beam projectors for sm_103a: the Siddon forward projection y = A x
// (Sec. 1, Eq. 1: one ray per detector pixel) and its exact transpose
// x = A^T y, as plain grids of the tiles defined in projector_device.cuh
// (ray-column warps sharing x/y stepping; the transpose gathers per voxel).
//
// Launch shapes are per geometry: DevGeom::fwd_rows (rays per lane of the
// forward tile) and DevGeom::bwd_config (column patch and voxels per lane of
// the transpose tile), set to defaults at creation and chosen by
// cbct_geometry_autotune.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "projector_device.cuh"

namespace cbct {

// ------------------------------------------------------------- forward A x

// 4 rays per lane hold 80 registers (3 CTAs per SM); fewer fit in 64.
template <typename T, bool COMP, int R, bool VF>
__global__ void __launch_bounds__(FWD_THREADS, R >= 4 ? 3 : 4)
forward_kernel(DevGeom g, const T *__restrict__ vol, T *__restrict__ proj, Epilogue epi) {
    __shared__ double red[FWD_THREADS / 32];
    if (epi.stop && *epi.stop) return;
    auto partial_at = [&]() -> double * {
        const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        return epi.partial ? epi.partial + b * TILE_PARTIALS : nullptr;
    };
    forward_tile<T, COMP, R, VF>(g, vol, proj, epi, blockIdx.x, blockIdx.y, blockIdx.z, partial_at, red);
}

template <int R>
__global__ void __launch_bounds__(FWD_THREADS)
count_kernel(DevGeom g, unsigned long long *count) {
    __shared__ double red[FWD_THREADS / 32];
    const int warp = threadIdx.x >> 5;
    const int iu = blockIdx.x * FWD_COLS + warp;
    int c = 0;
    if (iu < g.nu) {
        RayAxis rx, ry, rz[R];
        load_rays<R>(g, blockIdx.z, iu, blockIdx.y * 32 * R, g.nv, rx, ry, rz);
        auto fetch = [](int) { return 0.0f; };
        auto seg = [&](int, float len, float) { c += len > 0.0f; };
        trace_columns<R>(g, rx, ry, rz, 0, g.nx, 0, g.ny, 0, g.nz, 0, g.nz, g.nx * g.nz, fetch, seg);
    }
    const double s = block_sum<FWD_THREADS>((double)c, red);
    if (threadIdx.x == 0) atomicAdd(count, (unsigned long long)s);
}

dim3 forward_grid(const DevGeom &g) {
    const int rows = 32 * g.fwd_rows;
    return dim3((g.nu + FWD_COLS - 1) / FWD_COLS, (g.nv + rows - 1) / rows, g.nangles);
}

int forward_num_blocks(const DevGeom &g) {
    dim3 gr = forward_grid(g);
    return (int)(gr.x * gr.y * gr.z);
}

template <int R, bool VF>
static void launch_forward_r(const DevGeom &g, const void *x, void *y, cbct_dtype t, const Epilogue &epi,
                             cudaStream_t s) {
    const dim3 grid = forward_grid(g);
    switch (t) {
    case CBCT_F32:
        forward_kernel<float, false, R, VF><<<grid, FWD_THREADS, 0, s>>>(g, (const float *)x, (float *)y, epi);
        break;
    case CBCT_F16:
        forward_kernel<__half, true, R, VF><<<grid, FWD_THREADS, 0, s>>>(g, (const __half *)x, (__half *)y, epi);
        break;
    case CBCT_BF16:
        forward_kernel<__nv_bfloat16, true, R, VF><<<grid, FWD_THREADS, 0, s>>>(
            g, (const __nv_bfloat16 *)x, (__nv_bfloat16 *)y, epi);
        break;
    }
}

template <bool VF>
static void launch_forward_v(const DevGeom &g, const void *x, void *y, cbct_dtype t, const Epilogue &epi,
                             cudaStream_t s) {
    switch (g.fwd_rows) {
    case 1: launch_forward_r<1, VF>(g, x, y, t, epi, s); break;
    case 4: launch_forward_r<4, VF>(g, x, y, t, epi, s); break;
    default: launch_forward_r<2, VF>(g, x, y, t, epi, s); break;
    }
}

cbct_status launch_forward(const DevGeom &g, const void *x, void *y, cbct_dtype t,
                           const Epilogue &epi, cudaStream_t s, bool vfast) {
    if (vfast)
        launch_forward_v<true>(g, x, y, t, epi, s);
    else
        launch_forward_v<false>(g, x, y, t, epi, s);
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

cbct_status launch_count(const DevGeom &g, unsigned long long *count_dev, cudaStream_t s) {
    const dim3 grid = forward_grid(g);
    switch (g.fwd_rows) {
    case 1: count_kernel<1><<<grid, FWD_THREADS, 0, s>>>(g, count_dev); break;
    case 4: count_kernel<4><<<grid, FWD_THREADS, 0, s>>>(g, count_dev); break;
    default: count_kernel<2><<<grid, FWD_THREADS, 0, s>>>(g, count_dev); break;
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

// ---------------------------------------------------------- transpose A^T y

// Transpose tile shapes: column patch CX x (8 / CX), 32 K voxels along z;
// configurations 0..3 and 8, 9 keep the slab intervals of their candidate
// rows in registers per angle (8, 9: 4 voxels per lane, 3 CTAs per SM).
BrickShape backward_shape(int config) {
    switch (config) {
    case 8: return BrickShape{2, 4, 128, 4};
    case 9: return BrickShape{4, 2, 128, 4};
    case 1: return BrickShape{4, 2, 64, 2};
    case 2: return BrickShape{8, 1, 32, 1};
    case 3: return BrickShape{2, 4, 64, 2};
    case 4: return BrickShape{4, 2, 128, 4};
    case 5: return BrickShape{2, 4, 128, 4};
    case 6: return BrickShape{4, 2, 256, 8};
    case 7: return BrickShape{2, 4, 256, 8};
    default: return BrickShape{4, 2, 32, 1};
    }
}

dim3 backward_grid(const DevGeom &g) {
    const BrickShape b = backward_shape(g.bwd_config);
    return dim3((g.nx + b.bx - 1) / b.bx, (g.ny + b.by - 1) / b.by, (g.nz + b.bz - 1) / b.bz);
}

int backward_num_blocks(const DevGeom &g) {
    dim3 gr = backward_grid(g);
    return (int)(gr.x * gr.y * gr.z);
}

int backward_passes(const DevGeom &g, const float *accum) {
    if (!accum || g.angle_block <= 0 || g.angle_block >= g.nangles) return 1;
    return (g.nangles + g.angle_block - 1) / g.angle_block;
}

// One launch per block of angles (DevGeom::angle_block) when `accum` (M FP32
// values) is given: each pass reads only its angles' projections, which then
// stay in L2 while every voxel tile of the pass gathers from them.
cbct_status launch_backward(const DevGeom &g, const float *y, void *x, cbct_dtype t, const Epilogue &epi,
                            cudaStream_t s, bool zfast, float *accum) {
    const int passes = backward_passes(g, accum);
    for (int p = 0; p < passes; ++p) {
        const int a0 = passes == 1 ? 0 : p * g.angle_block;
        const int a1 = passes == 1 ? g.nangles : min(g.nangles, a0 + g.angle_block);
        const float *acc_in = p > 0 ? accum : nullptr;
        float *acc_out = p + 1 < passes ? accum : nullptr;
        if (zfast)
            launch_backward_zfast(g, y, x, t, epi, s, a0, a1, acc_in, acc_out);
        else
            launch_backward_abi(g, y, x, t, epi, s, a0, a1, acc_in, acc_out);
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

// ------------------------------------------------------ z slab crossings
// zbox[k][iv] = (entry, exit) alpha of row iv's ray in z slab k, i.e. the two
// z plane crossings ordered; a ray in a z plane (I == 0) is inside slab pq
// for every alpha and outside every other slab.  The rows' z tables do not
// depend on the angle (circular orbit), so one table serves all angles.
__global__ void zbox_kernel(DevGeom g, float2 *__restrict__ zbox) {
    const size_t n = (size_t)g.nz * g.nv;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx / g.nv), iv = (int)(idx % g.nv);
        const float4 z = g.ray_z[iv];
        const float kf = (float)k;
        float2 r;
        if (z.y == 0.0f) {
            r = z.z == kf ? make_float2(-FLT_MAX, FLT_MAX) : make_float2(FLT_MAX, FLT_MAX);
        } else {
            const RayAxis rz{z.x, z.y, z.z};
            const float e0 = plane_alpha(kf - z.z, g.dz, rz);
            const float e1 = plane_alpha((kf + 1.0f) - z.z, g.dz, rz);
            r = make_float2(fminf(e0, e1), fmaxf(e0, e1));
        }
        zbox[idx] = r;
    }
}

cudaError_t launch_zbox(const DevGeom &g, float2 *zbox) {
    const size_t n = (size_t)g.nz * g.nv;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    zbox_kernel<<<blocks, 256, 0, 0>>>(g, zbox);
    return cudaGetLastError();
}

// ------------------------------------------- ray-length weighted inputs
// The transpose sums len * |d'| * y; its input w = |d'| * y (v-fastest) is
// formed once per product (here, or in the forward epilogue).

// v-fastest y[a][iu][iv] -> w[a][iu][iv]: one thread per detector pixel,
// looping over the angles (the length is loaded once).
template <typename T>
__global__ void __launch_bounds__(256) weight_kernel(const T *__restrict__ y, const float *__restrict__ len,
                                                     float *__restrict__ w, size_t nuv, int nangles) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nuv; i += (size_t)gridDim.x * blockDim.x) {
        const float l = len[i];
        for (int a = 0; a < nangles; ++a) w[(size_t)a * nuv + i] = l * Storage<T>::load(y + (size_t)a * nuv + i);
    }
}

cbct_status launch_weight(const DevGeom &g, const void *y, cbct_dtype t, float *w, cudaStream_t s) {
    const size_t nuv = (size_t)g.nu * g.nv;
    const int blocks = (int)std::min<size_t>((nuv + 255) / 256, 4096);
    const int na = g.nangles;
    switch (t) {
    case CBCT_F32: weight_kernel<float><<<blocks, 256, 0, s>>>((const float *)y, g.ray_len, w, nuv, na); break;
    case CBCT_F16: weight_kernel<__half><<<blocks, 256, 0, s>>>((const __half *)y, g.ray_len, w, nuv, na); break;
    case CBCT_BF16:
        weight_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16 *)y, g.ray_len, w, nuv, na);
        break;
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

// ABI y[a][iv][iu] (type T) -> w[a][iu][iv] = |d'| * y (FP32), through a
// 32 x 32 shared-memory tile so that both sides are coalesced.
template <typename T>
__global__ void __launch_bounds__(256) weighted_relayout_kernel(const T *__restrict__ src, const float *__restrict__ len,
                                                                float *__restrict__ dst, int nu, int nv) {
    __shared__ float tile[32][33];
    const size_t base = (size_t)blockIdx.z * nu * nv;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int u0 = blockIdx.x * 32, v0 = blockIdx.y * 32;
    for (int r = ty; r < 32; r += 8) {
        const int iv = v0 + r, iu = u0 + tx;
        if (iv < nv && iu < nu) tile[r][tx] = Storage<T>::load(src + base + (size_t)iv * nu + iu);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int iu = u0 + r, iv = v0 + tx;
        if (iu < nu && iv < nv) {
            const size_t o = (size_t)iu * nv + iv;
            dst[base + o] = len[o] * tile[tx][r];
        }
    }
}

cbct_status launch_weight_abi(const DevGeom &g, const void *y, cbct_dtype t, float *w, cudaStream_t s) {
    const dim3 grid((g.nu + 31) / 32, (g.nv + 31) / 32, g.nangles);
    switch (t) {
    case CBCT_F32:
        weighted_relayout_kernel<float><<<grid, 256, 0, s>>>((const float *)y, g.ray_len, w, g.nu, g.nv);
        break;
    case CBCT_F16:
        weighted_relayout_kernel<__half><<<grid, 256, 0, s>>>((const __half *)y, g.ray_len, w, g.nu, g.nv);
        break;
    case CBCT_BF16:
        weighted_relayout_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)y, g.ray_len, w, g.nu,
                                                                      g.nv);
        break;
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

// -------------------------------------------------- projection re-layout
//
// y[a][iv][iu] <-> y[a][iu][iv]: per angle a 2D transpose through a 32 x 33
// shared tile (coalesced on both sides).

template <typename T, bool TO_VFAST>
__global__ void __launch_bounds__(256) proj_relayout_kernel(const T *__restrict__ src, T *__restrict__ dst, int nu,
                                                            int nv) {
    __shared__ T tile[32][33];
    const size_t base = (size_t)blockIdx.z * nu * nv;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // rows/cols of the source plane: TO_VFAST: src [iv][iu]; else src [iu][iv]
    const int rows = TO_VFAST ? nv : nu, cols = TO_VFAST ? nu : nv;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int r = ty; r < 32; r += 8) {
        const int rr = r0 + r, cc = c0 + tx;
        if (rr < rows && cc < cols) tile[r][tx] = src[base + (size_t)rr * cols + cc];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int cc = c0 + r, rr = r0 + tx;
        if (cc < cols && rr < rows) dst[base + (size_t)cc * rows + rr] = tile[tx][r];
    }
}

template <typename T>
static void launch_proj_relayout_t(const DevGeom &g, const void *src, void *dst, bool to_vfast, cudaStream_t s) {
    const int rows = to_vfast ? g.nv : g.nu, cols = to_vfast ? g.nu : g.nv;
    const dim3 grid((cols + 31) / 32, (rows + 31) / 32, g.nangles);
    if (to_vfast)
        proj_relayout_kernel<T, true><<<grid, 256, 0, s>>>((const T *)src, (T *)dst, g.nu, g.nv);
    else
        proj_relayout_kernel<T, false><<<grid, 256, 0, s>>>((const T *)src, (T *)dst, g.nu, g.nv);
}

cbct_status launch_proj_relayout(const DevGeom &g, const void *src, void *dst, cbct_dtype t, bool to_vfast,
                                 cudaStream_t s) {
    switch (t) {
    case CBCT_F32: launch_proj_relayout_t<float>(g, src, dst, to_vfast, s); break;
    case CBCT_F16: launch_proj_relayout_t<__half>(g, src, dst, to_vfast, s); break;
    case CBCT_BF16: launch_proj_relayout_t<__nv_bfloat16>(g, src, dst, to_vfast, s); break;
    }
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

// ------------------------------------------------------- volume re-layout
//
// Standard x[k][j][i] <-> padded z-fastest (zf_col(i, j) + k): for each j a
// (k, i) plane is transposed through a 32 x 33 shared tile (coalesced on both
// sides).  Towards the padded layout the kernel also writes the zero pads of
// every column it covers and (block (0, 0, 0)) the guards at both ends.

template <typename T, bool TO_ZFAST>
__global__ void __launch_bounds__(256) relayout_kernel(DevGeom g, const T *__restrict__ src, T *__restrict__ dst) {
    __shared__ T tile[32][33];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int j = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    if (TO_ZFAST) {                 // src [k][j][i] -> dst padded [j][i][k]
        const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
        for (int r = ty; r < 32; r += 8) {
            const int k = k0 + r, i = i0 + tx;
            if (k < nz && i < nx) tile[r][tx] = src[((size_t)k * ny + j) * nx + i];
        }
        __syncthreads();
        const T zero = T(0.0f);
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r, k = k0 + tx;
            if (i < nx && k < nz) {
                const size_t c = (size_t)zf_col(g, i, j);
                dst[c + k] = tile[tx][r];
                if (k == 0) dst[c - 1] = zero;
                if (k == nz - 1) dst[c + nz] = zero;
            }
        }
        if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x < ZF_GUARD) {
            dst[threadIdx.x] = zero;
            dst[zf_len(g) - 1 - threadIdx.x] = zero;
        }
    } else {                        // src padded [j][i][k] -> dst [k][j][i]
        const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r, k = k0 + tx;
            if (i < nx && k < nz) tile[r][tx] = src[(size_t)zf_col(g, i, j) + k];
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
        relayout_kernel<T, true><<<grid, 256, 0, s>>>(g, (const T *)src, (T *)dst);
    } else {
        const dim3 grid((g.nz + 31) / 32, (g.nx + 31) / 32, g.ny);
        relayout_kernel<T, false><<<grid, 256, 0, s>>>(g, (const T *)src, (T *)dst);
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

// x = value in every voxel, 0 in every pad and guard (padded z-fastest, FP32).
__global__ void __launch_bounds__(256) fill_volume_kernel(DevGeom g, float *__restrict__ x, float value) {
    const int64_t n = zf_len(g);
    const int nzp = g.nz + 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e - ZF_GUARD;
        const int64_t k = c % nzp - 1;          // -1 and nz: pads
        const bool voxel = c >= 0 && c < n - 2 * ZF_GUARD && k >= 0 && k < g.nz;
        x[e] = voxel ? value : 0.0f;
    }
}

cbct_status launch_fill_volume(const DevGeom &g, float *x, float value, cudaStream_t s) {
    fill_volume_kernel<<<1024, 256, 0, s>>>(g, x, value);
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

}  // namespace cbct

using namespace cbct;

static cbct_status check_pair(const cbct_geometry *g, const void *a, const void *b, cbct_dtype t, const char *who) {
    if (!g || !a || !b) { set_error(std::string(who) + ": null geometry or buffer"); return CBCT_EINVAL; }
    if (t != CBCT_F32 && t != CBCT_F16 && t != CBCT_BF16) { set_error(std::string(who) + ": unknown dtype"); return CBCT_EINVAL; }
    return require_geometry_device(g, who);
}

extern "C" cbct_status cbct_project(const cbct_geometry *g, const void *x, void *y, cbct_dtype t,
                                    cbct_stream stream) {
    cbct_status st = check_pair(g, x, y, t, "cbct_project");
    if (st != CBCT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the forward kernel reads the padded z-fastest layout: re-lay the caller's volume first
    void *tmp = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)zf_len(g->dev) * dtype_size(t), s));
    st = launch_relayout(g->dev, x, tmp, t, true, s);
    if (st == CBCT_OK) {
        Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
        st = launch_forward(g->dev, tmp, y, t, epi, s, false);
    }
    cudaFreeAsync(tmp, s);
    return st;
}

extern "C" cbct_status cbct_backproject(const cbct_geometry *g, const void *y, void *x, cbct_dtype t,
                                        cbct_stream stream) {
    cbct_status st = check_pair(g, y, x, t, "cbct_backproject");
    if (st != CBCT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the transpose reads |d'| * y, v-fastest: re-lay and weight the caller's stack first
    float *tmp = nullptr;
    float *accum = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)cbct_geometry_num_rays(g) * sizeof(float), s));
    cudaError_t err = cudaSuccess;
    if (g->dev.angle_block < g->dev.nangles)     // summed in passes over blocks of angles
        err = cudaMallocAsync(&accum, (size_t)cbct_geometry_num_voxels(g) * sizeof(float), s);
    if (err != cudaSuccess) {
        cudaFreeAsync(tmp, s);
        return cuda_fail(err, "cbct_backproject");
    }
    st = launch_weight_abi(g->dev, y, t, tmp, s);
    if (st == CBCT_OK) {
        Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
        st = launch_backward(g->dev, tmp, x, t, epi, s, false, accum);
    }
    cudaFreeAsync(tmp, s);
    if (accum) cudaFreeAsync(accum, s);
    return st;
}

extern "C" cbct_status cbct_count_nnz(const cbct_geometry *g, int64_t *nnz, cbct_stream stream) {
    if (!g || !nnz) { set_error("cbct_count_nnz: null argument"); return CBCT_EINVAL; }
    const cbct_status dst = require_geometry_device(g, "cbct_count_nnz");
    if (dst != CBCT_OK) return dst;
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
