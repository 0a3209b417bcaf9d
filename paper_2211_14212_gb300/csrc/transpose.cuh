// Grids of the transpose tile (x = A^T y, Sec. 1, Eq. 1 read column-wise):
// one kernel per launch configuration (DevGeom::bwd_config), storage type
// and output layout, instantiated by transpose_zfast.cu (padded z-fastest
// output, the solvers' layout) and transpose_abi.cu (x[k][j][i]), which
// compile in parallel.
//
// PASSES selects the kernel that sums a block of angles [a_begin, a_end)
// with FP32 running sums kept between passes (launch_backward); the
// single-pass kernel sums every angle and takes neither the angle range nor
// the running-sum buffers (fewer live registers through the angle loop).
#pragma once

#include "projector_device.cuh"

namespace cbct {

// Hoisted tiles of 2 or 4 voxels per lane and 8-voxel tiles run 3 CTAs per
// SM (80 registers): the 2-voxel tiles clip their detector columns across the
// lanes, which measured 36.6 ms at 256^3 this way against 39.0 ms at 4 CTAs.
template <typename T, bool ZFAST, int CX, int K, bool HOIST, bool PASSES>
__global__ void __launch_bounds__(BWD_THREADS, (K >= 8 || (HOIST && K >= 2)) ? 3 : 4)
backward_kernel(DevGeom g, const float *__restrict__ proj, T *__restrict__ vol, Epilogue epi, int a_begin, int a_end,
                const float *acc_in, float *acc_out) {
    __shared__ double red[BWD_THREADS / 32];
    if (epi.stop && *epi.stop) return;
    auto partial_at = [&]() -> double * {
        const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        return epi.partial ? epi.partial + b * TILE_PARTIALS : nullptr;
    };
    if (PASSES)
        backward_tile<T, ZFAST, CX, K, HOIST>(g, proj, vol, epi, blockIdx.x, blockIdx.y, blockIdx.z, a_begin, a_end,
                                              acc_in, acc_out, partial_at, red);
    else
        backward_tile<T, ZFAST, CX, K, HOIST>(g, proj, vol, epi, blockIdx.x, blockIdx.y, blockIdx.z, 0, g.nangles,
                                              nullptr, nullptr, partial_at, red);
}

template <typename T, bool ZF, bool PASSES>
void launch_backward_tp(const DevGeom &g, const float *y, void *x, const Epilogue &epi, cudaStream_t s, int a0,
                        int a1, const float *acc_in, float *acc_out) {
    const dim3 grid = backward_grid(g);
    T *xx = (T *)x;
#define CBCT_BWD(CX, K, HOIST)                                                                                  \
    backward_kernel<T, ZF, CX, K, HOIST, PASSES><<<grid, BWD_THREADS, 0, s>>>(g, y, xx, epi, a0, a1, acc_in, \
                                                                               acc_out)
    switch (g.bwd_config) {         // shapes as in backward_shape
    case 1: CBCT_BWD(4, 2, true); break;
    case 2: CBCT_BWD(8, 1, true); break;
    case 3: CBCT_BWD(2, 2, true); break;
    case 4: CBCT_BWD(4, 4, false); break;
    case 5: CBCT_BWD(2, 4, false); break;
    case 6: CBCT_BWD(4, 8, false); break;
    case 7: CBCT_BWD(2, 8, false); break;
    case 8: CBCT_BWD(2, 4, true); break;
    case 9: CBCT_BWD(4, 4, true); break;
    default: CBCT_BWD(4, 1, true); break;
    }
#undef CBCT_BWD
}

// One launch over angles [a0, a1) in storage type t; the single-pass kernel
// when the launch covers every angle with no running sums.
template <bool ZF>
void launch_backward_layout(const DevGeom &g, const float *y, void *x, cbct_dtype t, const Epilogue &epi,
                            cudaStream_t s, int a0, int a1, const float *acc_in, float *acc_out) {
    const bool passes = acc_in || acc_out || a0 != 0 || a1 != g.nangles;
    switch (t) {
    case CBCT_F32:
        passes ? launch_backward_tp<float, ZF, true>(g, y, x, epi, s, a0, a1, acc_in, acc_out)
               : launch_backward_tp<float, ZF, false>(g, y, x, epi, s, a0, a1, acc_in, acc_out);
        break;
    case CBCT_F16:
        passes ? launch_backward_tp<__half, ZF, true>(g, y, x, epi, s, a0, a1, acc_in, acc_out)
               : launch_backward_tp<__half, ZF, false>(g, y, x, epi, s, a0, a1, acc_in, acc_out);
        break;
    case CBCT_BF16:
        passes ? launch_backward_tp<__nv_bfloat16, ZF, true>(g, y, x, epi, s, a0, a1, acc_in, acc_out)
               : launch_backward_tp<__nv_bfloat16, ZF, false>(g, y, x, epi, s, a0, a1, acc_in, acc_out);
        break;
    }
}

}  // namespace cbct
