// Launch-shape autotuner: per geometry, the forward tile's rays per lane and
// the transpose tile's shape are chosen by timing every candidate on a
// strided subset of the scan's angles (the work per angle is what the shape
// changes; the angle count only scales it).
#include <algorithm>
#include <cfloat>
#include <vector>

#include "common.cuh"

namespace cbct {

static const int kFwdRows[NUM_FWD_ROWS] = {1, 2, 4};

__global__ void fill_kernel(float *p, size_t n, float v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// Median-free timing: one warm-up launch, then the best of `reps` launches.
template <typename F>
static cbct_status time_best(F &&launch, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double *ms) {
    cbct_status st = launch();
    if (st != CBCT_OK) return st;
    double best = DBL_MAX;
    for (int i = 0; i < reps; ++i) {
        CBCT_CUDA_TRY(cudaEventRecord(e0, s));
        st = launch();
        if (st != CBCT_OK) return st;
        CBCT_CUDA_TRY(cudaEventRecord(e1, s));
        CBCT_CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.0f;
        CBCT_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        if (t < best) best = t;
    }
    *ms = best;
    return CBCT_OK;
}

}  // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_geometry_set_launch(cbct_geometry *g, int fwd_rows, int bwd_config) {
    if (!g) { set_error("cbct_geometry_set_launch: null geometry"); return CBCT_EINVAL; }
    if (fwd_rows != 1 && fwd_rows != 2 && fwd_rows != 4) {
        set_error("cbct_geometry_set_launch: fwd_rows must be 1, 2 or 4");
        return CBCT_EINVAL;
    }
    if (bwd_config < 0 || bwd_config >= NUM_BWD_CONFIGS) {
        set_error("cbct_geometry_set_launch: unknown bwd_config");
        return CBCT_EINVAL;
    }
    g->dev.fwd_rows = fwd_rows;
    g->dev.bwd_config = bwd_config;
    return CBCT_OK;
}

extern "C" cbct_status cbct_geometry_get_launch(const cbct_geometry *g, int *fwd_rows, int *bwd_config) {
    if (!g || !fwd_rows || !bwd_config) { set_error("cbct_geometry_get_launch: null argument"); return CBCT_EINVAL; }
    *fwd_rows = g->dev.fwd_rows;
    *bwd_config = g->dev.bwd_config;
    return CBCT_OK;
}

extern "C" cbct_status cbct_geometry_set_angle_block(cbct_geometry *g, int angles) {
    if (!g) { set_error("cbct_geometry_set_angle_block: null geometry"); return CBCT_EINVAL; }
    if (angles < 0) { set_error("cbct_geometry_set_angle_block: angles must be >= 0"); return CBCT_EINVAL; }
    g->dev.angle_block = angles == 0 ? default_angle_block(g->dev) : std::min(angles, g->dev.nangles);
    return CBCT_OK;
}

extern "C" cbct_status cbct_geometry_get_angle_block(const cbct_geometry *g, int *angles) {
    if (!g || !angles) { set_error("cbct_geometry_get_angle_block: null argument"); return CBCT_EINVAL; }
    *angles = g->dev.angle_block;
    return CBCT_OK;
}

extern "C" cbct_status cbct_geometry_autotune(cbct_geometry *g, int max_angles, double *times_ms,
                                              cbct_stream stream) {
    if (!g) { set_error("cbct_geometry_autotune: null geometry"); return CBCT_EINVAL; }
    const cbct_status dst = require_geometry_device(g, "cbct_geometry_autotune");
    if (dst != CBCT_OK) return dst;
    cudaStream_t s = (cudaStream_t)stream;
    const int na = g->desc.nangles;
    int keep = max_angles > 0 && max_angles < na ? max_angles : na;
    // A stack that fits in L2 would time the transpose's gathers from L2:
    // keep at least twice L2's worth of projections.
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess) {
        const size_t per_angle = (size_t)g->desc.nu * g->desc.nv * sizeof(float);
        keep = (int)std::max<size_t>(keep, std::min<size_t>(na, (2 * (size_t)l2 + per_angle - 1) / per_angle));
    }
    std::vector<double> sub((size_t)keep);
    for (int i = 0; i < keep; ++i) sub[i] = g->desc.angles_rad[(size_t)i * na / keep];
    cbct_geometry_desc d = g->desc;
    d.nangles = keep;
    d.angles_rad = sub.data();
    cbct_geometry *t = nullptr;
    cbct_status st = cbct_geometry_create(&d, &t);
    if (st != CBCT_OK) return st;

    const size_t m = (size_t)zf_len(g->dev);            // padded z-fastest volume
    const size_t n = (size_t)keep * g->dev.nv * g->dev.nu;
    float *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double tf[NUM_FWD_ROWS], tb[NUM_BWD_CONFIGS];
    cudaError_t err = cudaMallocAsync(&x, m * sizeof(float), s);
    if (err == cudaSuccess) err = cudaMallocAsync(&y, n * sizeof(float), s);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err != cudaSuccess) st = cuda_fail(err, "cbct_geometry_autotune");
    if (st == CBCT_OK) {
        st = launch_fill_volume(t->dev, x, 1.0f, s);
        fill_kernel<<<1024, 256, 0, s>>>(y, n, 1.0f);
        const Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
        for (int c = 0; c < NUM_FWD_ROWS && st == CBCT_OK; ++c) {
            t->dev.fwd_rows = kFwdRows[c];
            st = time_best([&] { return launch_forward(t->dev, x, y, CBCT_F32, epi, s, true); }, 2, s, e0, e1, &tf[c]);
        }
        for (int c = 0; c < NUM_BWD_CONFIGS && st == CBCT_OK; ++c) {
            t->dev.bwd_config = c;
            st = time_best([&] { return launch_backward(t->dev, y, x, CBCT_F32, epi, s, true, nullptr); }, 2, s, e0, e1,
                           &tb[c]);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (x) cudaFreeAsync(x, s);
    if (y) cudaFreeAsync(y, s);
    cudaStreamSynchronize(s);
    cbct_geometry_destroy(t);
    if (st != CBCT_OK) return st;
    int bf = 0, bb = 0;
    for (int c = 1; c < NUM_FWD_ROWS; ++c)
        if (tf[c] < tf[bf]) bf = c;
    for (int c = 1; c < NUM_BWD_CONFIGS; ++c)
        if (tb[c] < tb[bb]) bb = c;
    g->dev.fwd_rows = kFwdRows[bf];
    g->dev.bwd_config = bb;
    if (times_ms) {
        for (int c = 0; c < NUM_FWD_ROWS; ++c) times_ms[c] = tf[c];
        for (int c = 0; c < NUM_BWD_CONFIGS; ++c) times_ms[NUM_FWD_ROWS + c] = tb[c];
    }
    return CBCT_OK;
}
