// Voxel-driven, interpolating backprojector: the usual fast approximation of
// A^T that is not its exact transpose, the kind of backprojector AB-/BA-GMRES
// are meant for (Sec. 2.1.4).  Every voxel centre is projected onto every
// detector and the projection is sampled there by bilinear interpolation
// (zero outside the detector), weighted by the expected sum of A's entries of
// the rays through the voxel,
//     w = dx dy dz mag^2 |d'| / (du dv DSD),   mag = DSD / (DSO - <c, s_hat>),
// with |d'| the source-to-pixel distance of the sampled point.
//
// Work layout as the exact transpose's gather: a warp owns one voxel column
// (i, j) and 32 K voxels along z (lane l: k0 + kk 32 + l); the column's
// projected u and magnification are the same for all its voxels (warp-uniform),
// only v = z mag is per lane, and the lanes' neighbouring rows make the
// v-fastest projection reads contiguous.
#include <cmath>

#include "common.cuh"

namespace cbct {

constexpr int VD_CX = 4, VD_CY = 2, VD_K = 2, VD_THREADS = 256;

template <bool ZFAST>
__global__ void __launch_bounds__(VD_THREADS)
voxel_backproject_kernel(DevGeom g, const float *__restrict__ proj, float *__restrict__ vol) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * VD_CX + (warp % VD_CX), j = blockIdx.y * VD_CY + (warp / VD_CX);
    const int k0 = blockIdx.z * 32 * VD_K;
    if (i >= g.nx || j >= g.ny) return;               // uniform across the warp
    const float xc = g.bx0 + (i + 0.5f) * g.dx, yc = g.by0 + (j + 0.5f) * g.dy;
    const float cu = 0.5f * (g.nu - 1), cv = 0.5f * (g.nv - 1);
    const float wvol = g.dx * g.dy * g.dz / (g.du * g.dv * g.dsd);
    float zc[VD_K], acc[VD_K];
#pragma unroll
    for (int kk = 0; kk < VD_K; ++kk) {
        zc[kk] = g.bz0 + (k0 + kk * 32 + lane + 0.5f) * g.dz;
        acc[kk] = 0.0f;
    }
    const size_t nuv = (size_t)g.nu * g.nv;
    for (int a = 0; a < g.nangles; ++a) {
        const float2 cs = g.trig[a];
        const float mag = g.dsd / (g.dso - (xc * cs.x + yc * cs.y));
        const float u = (-xc * cs.y + yc * cs.x) * mag;
        const float fu = u / g.du + cu;
        const float fu0 = floorf(fu);
        const int iu = (int)fu0;
        const float tu = fu - fu0;
        if (iu < -1 || iu >= g.nu) continue;           // the column projects off the detector
        const float *pa = proj + (size_t)a * nuv;
        const bool u0_ok = iu >= 0, u1_ok = iu + 1 < g.nu;
        const float *c0 = u0_ok ? pa + (size_t)iu * g.nv : pa;
        const float *c1 = u1_ok ? pa + (size_t)(iu + 1) * g.nv : pa;
        const float wmag = wvol * mag * mag;
#pragma unroll
        for (int kk = 0; kk < VD_K; ++kk) {
            const float v = zc[kk] * mag;
            const float fv = v / g.dv + cv;
            const float fv0 = floorf(fv);
            const int iv = (int)fv0;
            const float tv = fv - fv0;
            const bool v0_ok = iv >= 0 && iv < g.nv, v1_ok = iv + 1 >= 0 && iv + 1 < g.nv;
            const float y00 = (u0_ok && v0_ok) ? __ldg(c0 + iv) : 0.0f;
            const float y01 = (u0_ok && v1_ok) ? __ldg(c0 + iv + 1) : 0.0f;
            const float y10 = (u1_ok && v0_ok) ? __ldg(c1 + iv) : 0.0f;
            const float y11 = (u1_ok && v1_ok) ? __ldg(c1 + iv + 1) : 0.0f;
            const float val = (1.0f - tu) * ((1.0f - tv) * y00 + tv * y01) + tu * ((1.0f - tv) * y10 + tv * y11);
            const float dlen = sqrtf(g.dsd * g.dsd + u * u + v * v);
            acc[kk] = fmaf(wmag * dlen, val, acc[kk]);
        }
    }
#pragma unroll
    for (int kk = 0; kk < VD_K; ++kk) {
        const int k = k0 + kk * 32 + lane;
        if (k >= g.nz) continue;
        const size_t vi = ZFAST ? (size_t)(zf_col(g, i, j) + k) : ((size_t)k * g.ny + j) * g.nx + i;
        vol[vi] = acc[kk];
    }
}

cbct_status launch_voxel_backproject(const DevGeom &g, const float *y_vfast, float *x, bool zfast, cudaStream_t s) {
    const dim3 grid((g.nx + VD_CX - 1) / VD_CX, (g.ny + VD_CY - 1) / VD_CY, (g.nz + 32 * VD_K - 1) / (32 * VD_K));
    if (zfast)
        voxel_backproject_kernel<true><<<grid, VD_THREADS, 0, s>>>(g, y_vfast, x);
    else
        voxel_backproject_kernel<false><<<grid, VD_THREADS, 0, s>>>(g, y_vfast, x);
    CBCT_CUDA_TRY(cudaGetLastError());
    return CBCT_OK;
}

}  // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_backproject_voxel_driven(const cbct_geometry *g, const float *y, float *x,
                                                     cbct_stream stream) {
    if (!g || !y || !x) { set_error("cbct_backproject_voxel_driven: null argument"); return CBCT_EINVAL; }
    const cbct_status dst = require_geometry_device(g, "cbct_backproject_voxel_driven");
    if (dst != CBCT_OK) return dst;
    cudaStream_t s = (cudaStream_t)stream;
    float *tmp = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)cbct_geometry_num_rays(g) * sizeof(float), s));
    cbct_status st = launch_proj_relayout(g->dev, y, tmp, CBCT_F32, true, s);
    if (st == CBCT_OK) st = launch_voxel_backproject(g->dev, tmp, x, false, s);
    cudaFreeAsync(tmp, s);
    return st;
}
