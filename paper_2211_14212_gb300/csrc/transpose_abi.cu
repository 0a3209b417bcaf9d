// Transpose grids writing the ABI volume layout x[k][j][i] (cbct_backproject).
#include "transpose.cuh"

namespace cbct {

void launch_backward_abi(const DevGeom &g, const float *y, void *x, cbct_dtype t, const Epilogue &epi,
                         cudaStream_t s, int a0, int a1, const float *acc_in, float *acc_out) {
    launch_backward_layout<false>(g, y, x, t, epi, s, a0, a1, acc_in, acc_out);
}

}  // namespace cbct
