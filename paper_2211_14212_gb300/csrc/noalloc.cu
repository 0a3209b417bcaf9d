// cbct_project_static: the forward projection y = A x of cbct_project for
// callers that cannot allocate device memory.  cbct_project re-lays the
// caller's volume x[k][j][i] into a padded z-fastest temporary (nx ny (nz + 2)
// + 4 elements) that it allocates on the stream; here that temporary is a
// fixed array in the library's own device memory, so the call allocates
// nothing.
#include <mutex>

#include "common.cuh"

namespace cbct {

// Largest re-laid volume the static scratch holds: 66 MiB of the padded
// layout, e.g. a 256^3 FP32 volume (67.6 MB padded) or 256^2 x 512 FP16/BF16.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)66 << 20;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static std::mutex g_scratch_mutex;
static void *g_scratch_ptr[MAX_DEVICES];

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device also loads the module there).
static cbct_status scratch_for_current_device(void **out) {
    int dev = 0;
    CBCT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("cbct_project_static: device ordinal out of range");
        return CBCT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_static_scratch);
        if (err != cudaSuccess) return cuda_fail(err, "cbct_project_static: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CBCT_OK;
}

}  // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_project_static(const cbct_geometry *g, const void *x, void *y, cbct_dtype t,
                                           cbct_stream stream) {
    if (!g || !x || !y) { set_error("cbct_project_static: null geometry or buffer"); return CBCT_EINVAL; }
    if (t != CBCT_F32 && t != CBCT_F16 && t != CBCT_BF16) {
        set_error("cbct_project_static: unknown dtype");
        return CBCT_EINVAL;
    }
    const size_t bytes = (size_t)zf_len(g->dev) * dtype_size(t);
    if (bytes > STATIC_SCRATCH_BYTES) {
        set_error("cbct_project_static: the volume's padded copy (nx ny (nz + 2) + 4 elements) needs more "
                  "than the 66 MiB of static scratch (a 256^3 FP32 volume fits)");
        return CBCT_EINVAL;
    }
    cbct_status st0 = require_geometry_device(g, "cbct_project_static");
    if (st0 != CBCT_OK) return st0;
    void *scratch = nullptr;
    cbct_status st = scratch_for_current_device(&scratch);
    if (st != CBCT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // The re-layout writes every voxel, pad and guard of the padded copy before
    // the forward kernel reads any, so nothing left by an earlier call is used
    // and nothing has to be cleared.
    st = launch_relayout(g->dev, x, scratch, t, true, s);
    if (st != CBCT_OK) return st;
    const Epilogue epi{nullptr, nullptr, 1.0, 0.0, nullptr, nullptr, nullptr};
    return launch_forward(g->dev, scratch, y, t, epi, s, false);
}
