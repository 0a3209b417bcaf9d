// Transpose grids writing the padded z-fastest volume (the solvers' layout).
#include "transpose.cuh"

namespace cbct {

void launch_backward_zfast(const DevGeom &g, const float *y, void *x, cbct_dtype t, const Epilogue &epi,
                           cudaStream_t s, int a0, int a1, const float *acc_in, float *acc_out) {
    launch_backward_layout<true>(g, y, x, t, epi, s, a0, a1, acc_in, acc_out);
}

}  // namespace cbct
