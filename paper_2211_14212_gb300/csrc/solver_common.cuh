// Building blocks shared by the Krylov solver drivers: deterministic FP64
// reductions, Givens rotations, storage scaling, workspace and iteration
// replay (optionally as a CUDA graph).
#pragma once

#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace cbct {

constexpr int VEC_THREADS = 256;
constexpr int VEC_BLOCKS = 152 * 4;     // fixed grid: fixed partial layout, deterministic sums
constexpr int RED_THREADS = 256;

// Sum of n partials in a fixed order, result valid in thread 0: thread t
// keeps four running sums (of the partials t + (4 q + r) RED_THREADS,
// r = 0..3, so that four loads are in flight), the rest goes to the first,
// the four are added pairwise, then the block tree.  Launch with RED_THREADS
// threads.
__device__ __forceinline__ double reduce_partials(const double *p, int n, double *scratch) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * RED_THREADS < n; i += 4 * RED_THREADS) {
        s0 += p[i];
        s1 += p[i + RED_THREADS];
        s2 += p[i + 2 * RED_THREADS];
        s3 += p[i + 3 * RED_THREADS];
    }
    for (; i < n; i += RED_THREADS) s0 += p[i];
    return block_sum<RED_THREADS>((s0 + s1) + (s2 + s3), scratch);
}

// Fixed-order fold of many norm partials into FOLD_BLOCKS block sums (block b
// takes a contiguous range), so that the single-block scalar step that
// follows reads few values; used when a projector leaves more than
// FOLD_MIN partials.  Launch FOLD_BLOCKS blocks of RED_THREADS threads.
constexpr int FOLD_BLOCKS = 152, FOLD_MIN = 16384;
template <int NT>
__global__ void __launch_bounds__(NT) k_fold_partials(const double *p, int n, double *out) {
    static_assert(NT == RED_THREADS, "reduce_partials runs on RED_THREADS threads");
    __shared__ double red[NT / 32];
    const int chunk = (n + gridDim.x - 1) / gridDim.x;
    const int b0 = min(n, (int)blockIdx.x * chunk), b1 = min(n, b0 + chunk);
    const double sum = reduce_partials(p + b0, b1 - b0, red);
    if (threadIdx.x == 0) out[blockIdx.x] = sum;
}

// Givens rotation (c, s, r): [c s; -s c] [a; b] = [r; 0], r = hypot(a, b) >= 0.
struct Rot { double c, s, r; };
__device__ __forceinline__ Rot givens(double a, double b) {
    const double r = hypot(a, b);
    if (r == 0.0) return Rot{1.0, 0.0, 0.0};
    return Rot{a / r, b / r, r};
}

// Storage scale for a vector about to be written: FP16 storage keeps the
// entries near unit RMS (stored = scale x true vector, scale a power of two
// predicted from the previous norm) so that they stay clear of FP16
// subnormals and overflow; FP32/BF16 keep scale 1.
__device__ __forceinline__ double storage_scale(int scaled, double sqrt_len, double norm_pred) {
    if (!scaled || !(norm_pred > 0.0) || !isfinite(norm_pred)) return 1.0;
    double e = rint(log2(sqrt_len / norm_pred));
    e = fmax(-60.0, fmin(60.0, e));
    return exp2(e);
}

__device__ __forceinline__ bool good(double v) { return v > 0.0 && isfinite(v); }

// -------------------------------------------------------------- vector kernels
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_sumsq(const T *__restrict__ x, int64_t n, double *partial) {
    __shared__ double red[VEC_THREADS / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        const double v = (double)Storage<T>::ld_plain(x + i);
        s += v * v;
    }
    s = block_sum<VEC_THREADS>(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// dst = coef * src, converting FP32 -> storage type.
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_scale_to(const float *__restrict__ src, T *__restrict__ dst, int64_t n, const double *coef, const int *stop) {
    if (stop && *stop) return;
    const float c = (float)*coef;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS)
        Storage<T>::store(dst + i, c * src[i]);
}

// v = coef * v in place.
static __global__ void __launch_bounds__(VEC_THREADS)
k_scale_inplace(float *v, int64_t n, const double *coef, const int *stop) {
    if (stop && *stop) return;
    const float c = (float)*coef;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS)
        v[i] *= c;
}

// Combine a basis: x[m] = sum_j coef[j] * basis_j[m], basis_j = basis + j * n.
// When `stop` is given the launch does nothing once *stop is set (the
// coefficients of an unfinished step are not valid then).
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_combine(const T *__restrict__ basis, const double *__restrict__ coef, int k, int64_t n, float *__restrict__ x,
          const int *stop = nullptr) {
    if (stop && *stop) return;
    for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n; i += (int64_t)VEC_BLOCKS * VEC_THREADS) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc += coef[j] * (double)Storage<T>::ld_plain(basis + (size_t)j * n + i);
        x[i] = (float)acc;
    }
}

// --------------------------------------------------------------- host helpers

// Stream-ordered workspace: every allocation is freed on the stream at scope exit.
struct Workspace {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Workspace(cudaStream_t st) : s(st) {}
    ~Workspace() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, count * sizeof(T) + 16, s);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = (T *)q;
        return e;
    }
    // `count` volume-side vectors in the padded z-fastest layout, back to
    // back, all zero (pads and guards included).
    template <typename T>
    cudaError_t alloc_volumes(T **p, const DevGeom &g, size_t count = 1) {
        const size_t len = (size_t)zf_len(g) * count;
        cudaError_t e = alloc(p, len);
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, len * sizeof(T), s);
        return e;
    }
};

inline bool is_device_pointer(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Launch accounting of one solver call: kernel counts and, in profiling
// mode, a CUDA event pair around every projector launch.
struct Tracker {
    bool profile = false;
    cudaStream_t s = nullptr;
    int64_t launches = 0, fwd = 0, bwd = 0;
    std::vector<cudaEvent_t> ev[2];         // [0] forward, [1] backward: start, end, start, end, ...
    ~Tracker() {
        for (auto &v : ev)
            for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
    cbct_status mark(int kind) {
        if (!profile) return CBCT_OK;
        cudaEvent_t e;
        CBCT_CUDA_TRY(cudaEventCreate(&e));
        ev[kind].push_back(e);
        CBCT_CUDA_TRY(cudaEventRecord(e, s));
        return CBCT_OK;
    }
    // counts only (events are owned by this tracker)
    Tracker snapshot() const {
        Tracker t;
        t.launches = launches;
        t.fwd = fwd;
        t.bwd = bwd;
        return t;
    }
    // a graph captured the launches made since `before` once and replayed them `replays` times
    void scale_since(const Tracker &before, int replays) {
        if (replays <= 1) return;
        launches = before.launches + (launches - before.launches) * replays;
        fwd = before.fwd + (fwd - before.fwd) * replays;
        bwd = before.bwd + (bwd - before.bwd) * replays;
    }
    // after the stream has been synchronised
    void fill(cbct_solve_report *rep) {
        if (!rep) return;
        rep->kernel_launches = launches;
        rep->forward_launches = fwd;
        rep->backward_launches = bwd;
        double ms[2] = {0.0, 0.0};
        for (int k = 0; k < 2; ++k)
            for (size_t i = 0; i + 1 < ev[k].size(); i += 2) {
                float t = 0.0f;
                if (cudaEventElapsedTime(&t, ev[k][i], ev[k][i + 1]) == cudaSuccess) ms[k] += t;
            }
        rep->forward_ms = ms[0];
        rep->backward_ms = ms[1];
    }
};

// Enqueue one iteration `iters` times; with use_graph (and a capturable
// stream), capture it once as a CUDA graph and replay the graph.  *replays
// is set to the number of graph launches (0 without a graph).
template <typename F>
cbct_status run_iterations(int iters, bool use_graph, cudaStream_t s, F &&enqueue_one, int *replays) {
    *replays = 0;
    if (iters <= 0) return CBCT_OK;
    if (!use_graph || s == nullptr || iters < 2) {
        for (int i = 0; i < iters; ++i) {
            cbct_status st = enqueue_one();
            if (st != CBCT_OK) return st;
        }
        return CBCT_OK;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CBCT_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cbct_status st = enqueue_one();
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != CBCT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    for (int i = 0; i < iters && e == cudaSuccess; ++i) {
        e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) ++*replays;
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
    return CBCT_OK;
}

// ------------------------------------------------- solver input / output
//
// The solvers keep b v-fastest and the iterate z-fastest; host buffers are
// staged through device memory.

struct SolveIO {
    const float *b_dev;   // b re-laid v-fastest, y[a][iu][iv], like the projection-side vectors
    float *x_dev;         // caller layout x[k][j][i] (device; staging buffer for host x)
    float *xz;            // the iterate in the solvers' padded z-fastest layout
    bool x_is_host;
    float *x_host;
};

inline cbct_status check_solve_args(const cbct_geometry *g, const float *b, float *x, const cbct_solve_opts *o) {
    if (!g || !b || !x || !o) { set_error("solver: null argument"); return CBCT_EINVAL; }
    if (o->iters < 1) { set_error("solver: iters must be >= 1"); return CBCT_EINVAL; }
    if (o->storage != CBCT_F32 && o->storage != CBCT_F16 && o->storage != CBCT_BF16) {
        set_error("solver: unknown storage type");
        return CBCT_EINVAL;
    }
    if (!(o->lambda >= 0.0) || !std::isfinite(o->lambda)) { set_error("solver: lambda must be finite and >= 0"); return CBCT_EINVAL; }
    if (o->explicit_residual && !(o->stop_tol >= 0.0 && o->stop_tol < 1.0)) {
        set_error("solver: stop_tol must be in [0, 1)");
        return CBCT_EINVAL;
    }
    return require_geometry_device(g, "solver");
}

// Stage host b / x through device memory when needed.
inline cbct_status setup_io(const cbct_geometry *g, const float *b, float *x, Workspace &ws, SolveIO &io) {
    const int64_t n = cbct_geometry_num_rays(g), m = cbct_geometry_num_voxels(g);
    io.x_dev = x;
    io.x_is_host = false;
    io.x_host = nullptr;
    const float *bsrc = b;
    if (!is_device_pointer(b)) {
        float *bd = nullptr;
        CBCT_CUDA_TRY(ws.alloc(&bd, (size_t)n));
        CBCT_CUDA_TRY(cudaMemcpyAsync(bd, b, sizeof(float) * n, cudaMemcpyHostToDevice, ws.s));
        bsrc = bd;
    }
    float *bv = nullptr;
    CBCT_CUDA_TRY(ws.alloc(&bv, (size_t)n));
    cbct_status st = launch_proj_relayout(g->dev, bsrc, bv, CBCT_F32, true, ws.s);
    if (st != CBCT_OK) return st;
    io.b_dev = bv;
    if (!is_device_pointer(x)) {
        float *xd = nullptr;
        CBCT_CUDA_TRY(ws.alloc(&xd, (size_t)m));
        io.x_dev = xd;
        io.x_is_host = true;
        io.x_host = x;
    }
    CBCT_CUDA_TRY(ws.alloc_volumes(&io.xz, g->dev));
    return CBCT_OK;
}

// x (caller layout) <- the z-fastest iterate; then to the host if x is a host buffer.
inline cbct_status finish_io(const cbct_geometry *g, SolveIO &io, cudaStream_t s) {
    cbct_status st = launch_relayout(g->dev, io.xz, io.x_dev, CBCT_F32, false, s);
    if (st != CBCT_OK) return st;
    if (io.x_is_host)
        CBCT_CUDA_TRY(cudaMemcpyAsync(io.x_host, io.x_dev, sizeof(float) * cbct_geometry_num_voxels(g),
                                      cudaMemcpyDeviceToHost, s));
    return CBCT_OK;
}

inline void copy_report(cbct_solve_report *rep, int done, const std::vector<double> &h, int iters) {
    if (!rep) return;
    rep->iters_done = done;
    const int c = done < iters ? done : iters;
    if (rep->resid_norm) std::memcpy(rep->resid_norm, h.data(), sizeof(double) * c);
    if (rep->normal_resid_norm) std::memcpy(rep->normal_resid_norm, h.data() + iters, sizeof(double) * c);
    if (rep->lambda_k) std::memcpy(rep->lambda_k, h.data() + 2 * iters, sizeof(double) * c);
}

}  // namespace cbct
