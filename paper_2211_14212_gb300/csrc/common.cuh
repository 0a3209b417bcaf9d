// Shared device-side definitions of the cone-beam library: the geometry as the
// kernels see it, storage-type conversions and error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>

#include "../../include/cbct.h"

namespace cbct {

// ---------------------------------------------------------------- geometry
//
// Every ray is parametrised by alpha along d' = (pixel - source), with alpha = 0
// at q, where the ray crosses the plane through the rotation axis parallel to
// the detector (so |alpha| < ~0.2 inside the volume; the source is at
// alpha = -dso/dsd, the pixel at 1 - dso/dsd).  For each axis a ray stores
// the index pq of the voxel plane nearest to q, the offset f = plane(pq) - q
// (|f| <= delta/2) and I = 1 / d'_axis.  The alpha at which it crosses plane p is
//     alpha(p) = ((p - pq) * delta + f) * I
// (x, y from ray_xy / ray_xyq [a][iu]; z from ray_z[iv]).  Measuring planes from
// the one nearest to q keeps every crossing exact to a few ulps of its distance
// from q, so rays meeting planes at glancing angles (rows near the mid-plane,
// columns near the centre at 0/90/180/270 degrees) keep their crossings in
// place.  I == 0 marks a ray exactly parallel to that axis' planes; pq then
// holds its (fixed) voxel index.  The length of the ray/voxel segment
// [alpha0, alpha1] is (alpha1 - alpha0) * ray_len[iu][iv].
//
// Forward and transposed kernels derive every x/y crossing from these tables
// with the same two rounded operations (plane_alpha); the transpose takes its
// z crossings from plane_alpha too (zbox), the forward projector from an
// equivalent one-FMA form measured from the same plane pq.  A^T is the
// transpose of A; in FP32 the two kernels' segment lengths agree to rounding
// (not bit for bit), which the dot-product tests bound.
struct DevGeom {
    int nx, ny, nz;
    int nu, nv, nangles;
    float dso, dsd;          // mm
    float du, dv;            // mm
    float bx0, by0, bz0;     // lower corner of the volume, mm
    float dx, dy, dz;        // voxel size, mm
    const float4 *ray_xy;    // [nangles][nu]: (fx, Ix, fy, Iy)
    const float2 *ray_xyq;   // [nangles][nu]: (pqx, pqy)
    const float4 *ray_z;     // [nv]: (fz, Iz, pqz, 0)
    const float *ray_len;    // [nu][nv]
    const float2 *trig;      // [nangles] (cos t, sin t), for footprint windows only
    const float2 *zbox;      // [nz][nv]: alpha interval (entry, exit) of row iv's ray in z slab k
    int zsingle;             // 1: every ray crosses at most one z plane inside any x/y voxel column
    int fwd_rows;            // forward tile: rays per lane (1, 2 or 4)
    int bwd_config;          // transpose tile: column patch / voxels per lane (backward_shape)
    int angle_block;         // transpose: angles per pass when summed in passes (launch_backward)
};

// Tile of the transpose: a bx x by patch of voxel columns (one warp each),
// bz = 32 r voxels along z (r per lane).
struct BrickShape {
    int bx, by, bz, r;
};

// ------------------------------------------------- internal volume layout
//
// Inside the library every volume-side vector is z-fastest with padded
// columns: voxel (i, j, k) sits at
//     ZF_GUARD + (j * nx + i) * (nz + 2) + 1 + k,
// each column carrying one zero below voxel 0 and one above voxel nz - 1, and
// the array starting and ending with ZF_GUARD zeros (zf_len elements in all).
// The forward projector then reads voxels k in [-2, nz + 1] of any column
// without a bounds test.  Vectors are zeroed when allocated; kernels that
// combine whole vectors elementwise keep the pads at zero, and the kernels
// that address voxels write the interior only.
constexpr int ZF_GUARD = 2;
__host__ __device__ __forceinline__ int64_t zf_len(const DevGeom &g) {
    return (int64_t)g.nx * g.ny * (g.nz + 2) + 2 * ZF_GUARD;
}
// index of voxel k = 0 of column (i, j)
__host__ __device__ __forceinline__ int64_t zf_col(const DevGeom &g, int i, int j) {
    return ZF_GUARD + 1 + ((int64_t)j * g.nx + i) * (g.nz + 2);
}

}  // namespace cbct

struct cbct_geometry {
    cbct::DevGeom dev;
    cbct_geometry_desc desc;     // angles_rad points at `angles`
    double *angles;              // host copy
    int device;                  // CUDA device the tables live on
    void *table_mem;             // one device allocation holding all tables
};

namespace cbct {

// ------------------------------------------------------------- storage types
template <typename T> struct Storage;
template <> struct Storage<float> {
    __device__ __forceinline__ static float load(const float *p) { return __ldg(p); }
    __device__ __forceinline__ static float ld_plain(const float *p) { return *p; }
    __device__ __forceinline__ static float round(float v) { return v; }
    __device__ __forceinline__ static void store(float *p, float v) { *p = v; }
};
template <> struct Storage<__half> {
    __device__ __forceinline__ static float load(const __half *p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static float ld_plain(const __half *p) { return __half2float(*p); }
    __device__ __forceinline__ static float round(float v) { return __half2float(__float2half_rn(v)); }
    __device__ __forceinline__ static void store(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    __device__ __forceinline__ static float load(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ __forceinline__ static float ld_plain(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ __forceinline__ static float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    __device__ __forceinline__ static void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

inline size_t dtype_size(cbct_dtype t) { return t == CBCT_F32 ? 4 : 2; }

// ------------------------------------------------- projector epilogue scalars
//
// The fused epilogues compute out = a * (A x) + b * out_old (or the A^T
// analogue).  a and b are FP64 values read from device memory (written by the
// previous solver kernel) or given directly; a null pointer means the
// immediate value.  out_old is read from `old` when set (an input buffer
// distinct from the output), else from the output buffer itself.  `partial`,
// when non-null, receives FP64 sums of squares of the stored outputs
// (TILE_PARTIALS per projector tile, one per warp), reduced later in a fixed
// order (deterministic norms).
struct Epilogue {
    const double *a_ptr;
    const double *b_ptr;
    double a_val, b_val;
    double *partial;
    const int *stop;         // when non-null and *stop != 0, the launch does nothing
    const void *old;         // where out_old is read (same storage type); null = the output itself
    float *weighted = nullptr;  // forward, v-fastest output only: when non-null, also receives
                             // |d'| * (stored output), the transpose's input (launch_backward)
};

__device__ __forceinline__ double epi_a(const Epilogue &e) { return e.a_ptr ? *e.a_ptr : e.a_val; }
__device__ __forceinline__ double epi_b(const Epilogue &e) { return e.b_ptr ? *e.b_ptr : e.b_val; }

// Projector tiles leave one FP64 norm partial per warp (8 per 256-thread
// tile), written without a block barrier; later kernels sum them in a fixed
// order.
constexpr int TILE_PARTIALS = 8;

// Sum of one double per lane of a warp, written by lane 0 to dst[warp].
__device__ __forceinline__ void warp_partial(double v, double *dst) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) dst[threadIdx.x >> 5] = v;
}

// Deterministic block reduction of one double per thread into thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *scratch /* NT/32 doubles */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < NT / 32; ++w) s += scratch[w];
    }
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------- host side
void set_error(const std::string &msg);
// CBCT_OK when the calling thread's current CUDA device is the one the
// geometry's tables were created on; CBCT_EINVAL (message names `who` and
// both devices) otherwise, CBCT_ECUDA when the current device cannot be read.
// Every entry point that launches work for a geometry checks this first: a
// launch on another device would read the tables and the caller's buffers
// through addresses that are not valid there.
cbct_status require_geometry_device(const cbct_geometry *g, const char *who);
cbct_status validate_geometry_desc(const cbct_geometry_desc *d);   // CBCT_EINVAL with a message
cbct_status cuda_fail(cudaError_t err, const char *what);

#define CBCT_CUDA_TRY(expr)                                     \
    do {                                                        \
        cudaError_t err__ = (expr);                             \
        if (err__ != cudaSuccess) return ::cbct::cuda_fail(err__, #expr); \
    } while (0)

// Kernel launchers (projector.cu).  All return CBCT_OK or a CUDA failure.
cbct_status launch_forward(const DevGeom &g, const void *x_zfast, void *y, cbct_dtype t,
                           const Epilogue &epi, cudaStream_t s, bool vfast);
// Layouts: the ABI uses x[k][j][i] and y[a][iv][iu].  The forward kernel reads
// volumes in the padded z-fastest layout above, and the transpose reads
// projections v-fastest, y[a][iu][iv]; the solvers keep their vectors in those
// layouts.
// launch_forward writes either projection layout, launch_backward either
// volume layout.
// The transpose reads its projections pre-weighted by the ray lengths |d'|,
// FP32, v-fastest: w[a][iu][iv] = |d'| * y (what the forward epilogue writes
// to Epilogue::weighted, or launch_weight / launch_weight_abi make).
// `accum` (optional, M FP32 values of scratch) lets the transpose run in passes
// over blocks of DevGeom::angle_block angles; null means one pass.
cbct_status launch_backward(const DevGeom &g, const float *w_vfast, void *x, cbct_dtype t,
                            const Epilogue &epi, cudaStream_t s, bool zfast, float *accum);
// One transpose launch over angles [a0, a1) (acc_in / acc_out as in
// backward_tile), output in the padded z-fastest or the ABI volume layout.
void launch_backward_zfast(const DevGeom &g, const float *w_vfast, void *x, cbct_dtype t, const Epilogue &epi,
                           cudaStream_t s, int a0, int a1, const float *acc_in, float *acc_out);
void launch_backward_abi(const DevGeom &g, const float *w_vfast, void *x, cbct_dtype t, const Epilogue &epi,
                         cudaStream_t s, int a0, int a1, const float *acc_in, float *acc_out);
// w[a][iu][iv] = |d'| * y for a v-fastest projection vector y[a][iu][iv] of type t.
cbct_status launch_weight(const DevGeom &g, const void *y_vfast, cbct_dtype t, float *w, cudaStream_t s);
// w[a][iu][iv] = |d'| * y for y in the ABI layout y[a][iv][iu].
cbct_status launch_weight_abi(const DevGeom &g, const void *y_abi, cbct_dtype t, float *w, cudaStream_t s);
int backward_passes(const DevGeom &g, const float *accum);
int default_angle_block(const DevGeom &g);
// Fills DevGeom::zbox (nz * nv entries) from the z tables; synchronous use at
// geometry creation (legacy default stream).
cudaError_t launch_zbox(const DevGeom &g, float2 *zbox);
// ABI x[k][j][i] <-> padded z-fastest (to_zfast also writes every pad and guard: zeros).
cbct_status launch_relayout(const DevGeom &g, const void *src, void *dst, cbct_dtype t, bool to_zfast,
                            cudaStream_t s);
// Zero pads and guards, `value` in every voxel of a padded z-fastest FP32 volume.
cbct_status launch_fill_volume(const DevGeom &g, float *x, float value, cudaStream_t s);
cbct_status launch_proj_relayout(const DevGeom &g, const void *src, void *dst, cbct_dtype t, bool to_vfast,
                                 cudaStream_t s);
cbct_status launch_count(const DevGeom &g, unsigned long long *count_dev, cudaStream_t s);
// Voxel-driven interpolating backprojector (an approximation of A^T), FP32,
// v-fastest projections in, either volume layout out (vdbp.cu).
cbct_status launch_voxel_backproject(const DevGeom &g, const float *y_vfast, float *x, bool zfast, cudaStream_t s);
int forward_num_blocks(const DevGeom &g);
int backward_num_blocks(const DevGeom &g);
// FP64 norm partials one launch leaves (TILE_PARTIALS per tile)
inline int forward_num_partials(const DevGeom &g) { return forward_num_blocks(g) * TILE_PARTIALS; }
inline int backward_num_partials(const DevGeom &g) { return backward_num_blocks(g) * TILE_PARTIALS; }
dim3 forward_grid(const DevGeom &g);
dim3 backward_grid(const DevGeom &g);
BrickShape backward_shape(int config);
constexpr int NUM_FWD_ROWS = 3, NUM_BWD_CONFIGS = 10;

}  // namespace cbct
