// Continuous-batching reconstruction server.
//
// Requests (a scan, its measured projections b, LSQR or LSMR, an iteration
// count, optional Tikhonov damping) are admitted into slots while the device
// memory they need fits a budget.  A step of the server advances a set of
// slots by one Krylov iteration with persistent multi-instance kernels: one
// forward launch walks the forward tiles of all slots in the step, one
// transpose launch walks all their tiles, one launch per scalar step handles
// all of them (one block each) and one launch updates all their vectors.  The
// schedule picks the set: the oldest slots until the step's forward tiles
// fill the GPU (FIFO), the shortest remaining work first (SRPT), the highest
// response ratio (RATIO), or every slot (SHARE).  Admission (tables, upload
// of b, the solver's start) and read-out (x to the host, freeing) run on
// their own threads and streams while the steps go on.  The launch
// topology of a step does not depend on the set (fixed persistent grids, a
// device slot table), so one captured CUDA graph is replayed for every step.
//
// Each slot computes what the single-request solver computes: the same tiles,
// the same per-ray and per-voxel summation order, the same scalar steps
// (gk.cuh); only the blockwise norm partials can be grouped differently when
// the single-request solver runs other launch shapes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gk.cuh"
#include "projector_device.cuh"

namespace cbct {

constexpr int SRV_MAX_SLOTS = 64;
constexpr int SRV_FWD_ROWS = 4;                       // forward tile: 4 rays per lane
constexpr int64_t SRV_SAT_TILES = 2048;                // forward tiles (8 columns x 128 rows) that fill a step
constexpr int SRV_SRPT_AGE_CAP = 64;                   // SRPT: steps a slot may be passed over before it goes first
constexpr int SRV_CX = 2, SRV_BK = 2;                  // transpose tile: 2 x 4 columns x 64 (configuration 3)
constexpr int SRV_BWD_CONFIG = 3;

struct SlotDev {
    DevGeom g;
    float *U, *Uw, *V, *w, *x, *h2;     // Uw = |d'| U, the transpose's input
    GkState *st;
    double *pf, *pb, *hist_r, *hist_n;
    const double *qf, *qb;  // the partials the scalar steps read: pf / pb, or their folds
    int nqf, nqb;
    int method, cap;
    int fgx, fgy;          // forward tile grid (x: columns / 8, y: row groups); z: angles
    int bgx, bgy;          // brick grid (x, y); z: bricks along z
    int64_t m;             // length of a volume-side vector (padded z-fastest layout)
};

struct SlotTable {
    int n;                                  // slots in use (entries 0..n-1)
    int fwd_start[SRV_MAX_SLOTS + 1];       // prefix sums of forward tiles
    int bwd_start[SRV_MAX_SLOTS + 1];       // prefix sums of bricks
    SlotDev s[SRV_MAX_SLOTS];
};

struct SlotStatus {
    int iter, stop, status, pad;
};

// Largest s in [0, n) with start[s] <= item (start is non-decreasing).
__device__ __forceinline__ int find_slot(const int *start, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Tiles are claimed one at a time from a counter (reset at the start of every
// step), so that blocks that drew cheap tiles (columns that miss the volume,
// voxel columns near the corners) take more: a persistent grid walking a fixed
// stride leaves SMs idle at the end of each kernel.
__device__ __forceinline__ int claim_tile(unsigned *counter, int *slot_sh) {
    __syncthreads();                       // every thread is done with the previous tile
    if (threadIdx.x == 0) *slot_sh = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *slot_sh;
}

// The tile kernels copy the claimed tile's DevGeom into shared memory, one
// int per thread (its fields then need no registers of their own).
static_assert(sizeof(DevGeom) % sizeof(int) == 0 && sizeof(DevGeom) / sizeof(int) <= FWD_THREADS &&
                  sizeof(DevGeom) / sizeof(int) <= BWD_THREADS,
              "DevGeom is copied one int per thread");

// U <- fa * A V + fb * U for every slot (forward tiles of all slots).
__global__ void __launch_bounds__(FWD_THREADS, 3) srv_forward(const SlotTable *tab, unsigned *counter) {
    __shared__ double red[FWD_THREADS / 32];
    __shared__ int item_sh;
    __shared__ DevGeom g_sh;               // the claimed tile's geometry
    const int n = tab->n;
    const int total = tab->fwd_start[n];
    for (int item = claim_tile(counter, &item_sh); item < total; item = claim_tile(counter, &item_sh)) {
        const int s = find_slot(tab->fwd_start, n, item);
        const SlotDev &sd = tab->s[s];
        if (sd.st->stop) continue;
        if (threadIdx.x < sizeof(DevGeom) / sizeof(int)) ((int *)&g_sh)[threadIdx.x] = ((const int *)&sd.g)[threadIdx.x];
        __syncthreads();
        const int local = item - tab->fwd_start[s];
        const int tx = local % sd.fgx, ty = (local / sd.fgx) % sd.fgy, a = local / (sd.fgx * sd.fgy);
        const Epilogue epi{&sd.st->fa, &sd.st->fb, 0.0, 0.0, nullptr, nullptr, nullptr, sd.Uw};
        forward_tile<float, false, SRV_FWD_ROWS, true>(g_sh, sd.V, sd.U, epi, tx, ty, a,
                                                       [&]() { return sd.pf + (size_t)local * TILE_PARTIALS; }, red);
    }
}

// V <- ba * A^T U + bb * V for every slot (transpose tiles of all slots, z-fastest volumes).
__global__ void __launch_bounds__(BWD_THREADS, 4) srv_backward(const SlotTable *tab, unsigned *counter) {
    __shared__ double red[BWD_THREADS / 32];
    __shared__ int item_sh;
    __shared__ DevGeom g_sh;               // the claimed tile's geometry
    const int n = tab->n;
    const int total = tab->bwd_start[n];
    for (int item = claim_tile(counter, &item_sh); item < total; item = claim_tile(counter, &item_sh)) {
        const int s = find_slot(tab->bwd_start, n, item);
        const SlotDev &sd = tab->s[s];
        if (sd.st->stop) continue;
        if (threadIdx.x < sizeof(DevGeom) / sizeof(int)) ((int *)&g_sh)[threadIdx.x] = ((const int *)&sd.g)[threadIdx.x];
        __syncthreads();
        const int local = item - tab->bwd_start[s];
        const int tbx = local % sd.bgx, tby = (local / sd.bgx) % sd.bgy, tbz = local / (sd.bgx * sd.bgy);
        const Epilogue epi{&sd.st->ba, &sd.st->bb, 0.0, 0.0, nullptr, nullptr, nullptr};
        backward_tile<float, true, SRV_CX, SRV_BK, true, 2>(g_sh, sd.Uw, sd.V, epi, tbx, tby, tbz, 0, g_sh.nangles,
                                                         nullptr, nullptr,
                                                         [&]() { return sd.pb + (size_t)local * TILE_PARTIALS; }, red);
    }
}

// Scalar steps, one block per slot, same fixed-order reductions as the solvers.
__global__ void __launch_bounds__(RED_THREADS) srv_after_forward(const SlotTable *tab) {
    __shared__ double red[RED_THREADS / 32];
    const int s = blockIdx.x;
    if (s >= tab->n) return;
    const SlotDev &sd = tab->s[s];
    if (sd.st->stop) return;
    const double ss = reduce_partials(sd.qf, sd.nqf, red);
    if (threadIdx.x == 0) gk_after_forward_step(sd.st, ss, nullptr);
}

__global__ void __launch_bounds__(RED_THREADS) srv_after_backward(const SlotTable *tab) {
    __shared__ double red[RED_THREADS / 32];
    const int s = blockIdx.x;
    if (s >= tab->n) return;
    const SlotDev &sd = tab->s[s];
    if (sd.st->stop) return;
    const double ss = reduce_partials(sd.qb, sd.nqb, red);
    if (threadIdx.x == 0)
        gk_after_backward_step(sd.st, ss, sd.method, sd.hist_r, sd.hist_n, nullptr, nullptr, sd.cap);
}

// Vector recurrences of every slot (grid-stride over each slot's voxels).
__global__ void __launch_bounds__(VEC_THREADS) srv_update(const SlotTable *tab) {
    const int n = tab->n;
    const int64_t stride = (int64_t)gridDim.x * VEC_THREADS;
    for (int s = 0; s < n; ++s) {
        const SlotDev &sd = tab->s[s];
        const GkState *st = sd.st;
        if (st->stop) continue;
        const float k1 = (float)st->k1, k2 = (float)st->k2, k3 = (float)st->k3, k4 = (float)st->k4;
        for (int64_t i = (int64_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < sd.m; i += stride) {
            if (sd.method == M_LSQR) lsqr_elem(sd.V[i], sd.x[i], sd.w[i], k1, k2, k3);
            else lsmr_elem(sd.V[i], sd.x[i], sd.w[i], sd.h2[i], k1, k2, k3, k4);
        }
    }
}

__global__ void srv_status(const SlotTable *tab, SlotStatus *out) {
    const int s = threadIdx.x;
    if (s >= tab->n) return;
    const GkState *st = tab->s[s].st;
    out[s] = SlotStatus{st->iter, st->stop, st->status, 0};
}

// ====================================================================== host

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Request {
    uint64_t id = 0;
    cbct_geometry_desc desc{};
    std::vector<double> angles;
    std::vector<float> b;
    int method = M_LSQR;
    int iters = 0;
    double damp = 0.0;
    size_t bytes = 0;
    // results
    bool admitted = false;
    bool done = false;
    cbct_status status = CBCT_OK;
    std::string error;
    std::vector<float> x;
    std::vector<double> hist_r, hist_n;
    int iters_done = 0;
    double t_submit = 0, t_admit = 0, t_finish = 0;
};

struct Slot {
    std::shared_ptr<Request> req;
    cbct_geometry *geom = nullptr;
    float *U = nullptr, *Uw = nullptr, *V = nullptr, *w = nullptr, *x = nullptr, *h2 = nullptr, *b = nullptr;
    GkState *st = nullptr;
    double *pf = nullptr, *pb = nullptr, *hist = nullptr;
    double *pfold = nullptr;          // 2 x FOLD_BLOCKS folded partials (steps of this slot alone)
    int nf = 0, nb = 0, steps = 0;
    int passed_over = 0;              // consecutive steps this slot was left out of (SRPT aging)
    bool aged = false;                // passed over SRV_SRPT_AGE_CAP steps in a row: first until it finishes
    double work_iter = 0.0;           // cost model of one iteration: rays x (nx + ny)
    cudaEvent_t ready = nullptr;      // recorded on the admission stream once the set-up is queued
    cudaGraphExec_t solo_graph = nullptr;   // captured step of this slot alone (enqueue_step)
};

// Forward tiles and bricks of a scan under the server's launch shapes.
void grids(const cbct_geometry_desc &d, int &fgx, int &fgy, int &bgx, int &bgy, int &bgz) {
    fgx = (d.nu + FWD_COLS - 1) / FWD_COLS;
    fgy = (d.nv + 32 * SRV_FWD_ROWS - 1) / (32 * SRV_FWD_ROWS);
    bgx = (d.nx + SRV_CX - 1) / SRV_CX;
    bgy = (d.ny + (8 / SRV_CX) - 1) / (8 / SRV_CX);
    bgz = (d.nz + 32 * SRV_BK - 1) / (32 * SRV_BK);
}

// Device memory a request holds at its peak (ray tables, Krylov vectors,
// staging of b, partial sums, state and histories), rounded up per buffer.
size_t request_bytes(const cbct_geometry_desc &d, int method, int iters) {
    auto al = [](size_t b) { return (b + 1023) & ~(size_t)1023; };
    // m: a volume-side vector in the padded z-fastest layout
    const size_t n = (size_t)d.nangles * d.nv * d.nu, m = (size_t)d.nx * d.ny * (d.nz + 2) + 2 * ZF_GUARD;
    int fgx, fgy, bgx, bgy, bgz;
    grids(d, fgx, fgy, bgx, bgy, bgz);
    const size_t nf = (size_t)fgx * fgy * d.nangles, nb = (size_t)bgx * bgy * bgz;
    size_t t = al((size_t)d.nangles * d.nu * 24) + al((size_t)d.nv * 16) + al(n / d.nangles * 4) + al(d.nangles * 8);
    t += al((size_t)d.nz * d.nv * 8);                       // z slab table
    t += 3 * al(n * 4);                                     // U, |d'| U and the staged b
    t += al(m * 4) * (method == M_LSMR ? 4 : 3);            // V, w, x (+ hbar)
    t += al(nf * 8 * TILE_PARTIALS) + al(nb * 8 * TILE_PARTIALS) + al(2 * FOLD_BLOCKS * 8) + al(sizeof(GkState)) +
         al((size_t)2 * iters * 8);
    t += al(m * 4);                                         // re-layout of x when the result is read out
    return t;
}

}  // namespace

// Three library threads share the work of a server, so that the steps never
// wait for host-side work:
//   admission   takes waiting requests in submission order while the budget
//               and the slot count allow, builds the scan's tables, uploads b
//               and queues the solver's start (b / ||b||, the first A^T) on
//               its own stream, then hands the slot to the step thread with
//               an event that orders the step stream after the set-up;
//   steps       advances the admitted slots one Krylov iteration per step
//               (one captured graph replayed) and hands finished slots on;
//   read-out    copies each finished result to the host on its own stream,
//               frees the slot's memory and wakes the waiters.
// Geometries of finished slots are destroyed only while no slot is active
// (their tables are a few MB), because freeing device memory waits for the
// whole device and would hold up the set-up of the next request (measured:
// freeing them right after queuing a step raised the median latency of the
// serving stream by 9 %).
struct ServerImpl {
    size_t budget = 0, in_use = 0;
    int max_slots = 1, use_graph = 1, device = 0, schedule = CBCT_SCHED_FIFO;
    double work_rate = 0.0;           // cost-model units per second, running estimate from timed steps
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_admit, cv_ready, cv_finish, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::map<uint64_t, std::shared_ptr<Request>> requests;
    std::vector<Slot> ready;          // set up, not yet stepped (guarded by mu)
    std::deque<Slot> finishing;       // stepped to the end, not yet read out (guarded by mu)
    std::vector<cbct_geometry *> graveyard;   // geometries of read-out slots (guarded by mu)
    int in_flight = 0;                // admitted and not yet finished stepping (guarded by mu)
    int active_slots = 0;             // slots the step thread holds (guarded by mu)
    uint64_t next_id = 1;
    bool stopping = false, steps_stopped = false;
    std::thread admitter, worker, reader;
    cudaStream_t s = nullptr, s_admit = nullptr, s_read = nullptr;
    // step-thread owned
    SlotTable *tab_host = nullptr, *tab_dev = nullptr;
    SlotStatus *stat_host = nullptr, *stat_dev = nullptr;
    unsigned *counters = nullptr;     // tile counters of the forward and transpose kernels
    std::vector<Slot> slots;
    std::vector<int> step_slots;      // slots advanced by the current step, in slot-table order
    bool table_dirty = true;
    cudaGraphExec_t step_graph = nullptr;
    int fwd_grid = 0, bwd_grid = 0, vec_grid = 0;
    int64_t steps_run = 0, graph_replays = 0;

    void run_admission();
    void run_steps();
    void run_readout();
    std::vector<int> pick_step_slots() const;
    cbct_status setup_slot(Slot &sl);
    void release_slot(Slot &sl, cudaStream_t st, bool keep_geometry);
    cbct_status finish_slot(Slot &sl);
    cbct_status enqueue_step();
    // the current step advances one slot whose tiles fill the GPU alone
    bool solo_step() const { return step_slots.size() == 1 && slots[step_slots[0]].nf >= SRV_SAT_TILES; }
    void complete(const std::shared_ptr<Request> &r, cbct_status st, const std::string &msg);
    void publish(const std::shared_ptr<Request> &r, cbct_status st, const std::string &msg);
    void return_budget(const std::shared_ptr<Request> &r);
};

// -------------------------------------------------------------- slot life

// On the admission thread and stream.
cbct_status ServerImpl::setup_slot(Slot &sl) {
    Request &r = *sl.req;
    r.desc.angles_rad = r.angles.data();
    cbct_status st = cbct_geometry_create(&r.desc, &sl.geom);
    if (st != CBCT_OK) return st;
    sl.geom->dev.fwd_rows = SRV_FWD_ROWS;
    sl.geom->dev.bwd_config = SRV_BWD_CONFIG;
    const DevGeom &g = sl.geom->dev;
    // m: a volume-side vector in the padded z-fastest layout (pads zeroed below)
    const int64_t n = cbct_geometry_num_rays(sl.geom), m = zf_len(g);
    sl.nf = forward_num_blocks(g);
    sl.nb = backward_num_blocks(g);
    sl.work_iter = (double)n * (g.nx + g.ny);
    cudaStream_t sa = s_admit;
    auto A = [&](auto **p, size_t cnt) {
        return cudaMallocAsync((void **)p, cnt * sizeof(**p) + 16, sa);
    };
    cudaError_t e = A(&sl.U, (size_t)n);
    if (e == cudaSuccess) e = A(&sl.Uw, (size_t)n);
    if (e == cudaSuccess) e = A(&sl.b, (size_t)n);
    if (e == cudaSuccess) e = A(&sl.V, (size_t)m);
    if (e == cudaSuccess) e = A(&sl.w, (size_t)m);
    if (e == cudaSuccess) e = A(&sl.x, (size_t)m);
    if (e == cudaSuccess && r.method == M_LSMR) e = A(&sl.h2, (size_t)m);
    if (e == cudaSuccess) e = A(&sl.pf, (size_t)std::max(sl.nf * TILE_PARTIALS, VEC_BLOCKS));
    if (e == cudaSuccess) e = A(&sl.pb, (size_t)sl.nb * TILE_PARTIALS);
    if (e == cudaSuccess) e = A(&sl.pfold, (size_t)2 * FOLD_BLOCKS);
    if (e == cudaSuccess) e = A(&sl.st, (size_t)1);
    if (e == cudaSuccess) e = A(&sl.hist, (size_t)2 * r.iters);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.b, r.b.data(), sizeof(float) * n, cudaMemcpyHostToDevice, sa);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.x, 0, sizeof(float) * m, sa);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.V, 0, sizeof(float) * m, sa);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.w, 0, sizeof(float) * m, sa);
    if (e == cudaSuccess && sl.h2) e = cudaMemsetAsync(sl.h2, 0, sizeof(float) * m, sa);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.hist, 0, sizeof(double) * 2 * r.iters, sa);
    GkState init;
    std::memset(&init, 0, sizeof init);
    init.damp = r.damp;
    init.sqrt_n = std::sqrt((double)n);
    init.sqrt_m = std::sqrt((double)cbct_geometry_num_voxels(sl.geom));
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.st, &init, sizeof init, cudaMemcpyHostToDevice, sa);
    if (e != cudaSuccess) return cuda_fail(e, "server: slot allocation");
    // beta_1 u_1 = b, alpha_1 v_1 = A^T u_1: the same start as the single-request solver
    k_sumsq<float><<<VEC_BLOCKS, VEC_THREADS, 0, sa>>>(sl.b, n, sl.pf);
    gk_begin<<<1, RED_THREADS, 0, sa>>>(sl.st, sl.pf, VEC_BLOCKS);
    // U = su * b, v-fastest
    st = launch_proj_relayout(g, sl.b, sl.U, CBCT_F32, true, sa);
    if (st != CBCT_OK) return st;
    k_scale_inplace<<<VEC_BLOCKS, VEC_THREADS, 0, sa>>>(sl.U, n, &sl.st->c0, &sl.st->stop);
    st = launch_weight(g, sl.U, CBCT_F32, sl.Uw, sa);
    if (st != CBCT_OK) return st;
    Epilogue eb{&sl.st->ba, &sl.st->bb, 0.0, 0.0, sl.pb, &sl.st->stop, nullptr};
    st = launch_backward(g, sl.Uw, sl.V, CBCT_F32, eb, sa, true, nullptr);
    if (st != CBCT_OK) return st;
    gk_begin2<<<1, RED_THREADS, 0, sa>>>(sl.st, sl.pb, sl.nb * TILE_PARTIALS, r.method);
    k_start_dirs<float><<<VEC_BLOCKS, VEC_THREADS, 0, sa>>>(sl.V, sl.w, r.method == M_LSMR ? sl.h2 : nullptr, nullptr,
                                                            m, sl.st);
    CBCT_CUDA_TRY(cudaGetLastError());
    CBCT_CUDA_TRY(cudaFreeAsync(sl.b, sa));
    sl.b = nullptr;
    CBCT_CUDA_TRY(cudaEventCreateWithFlags(&sl.ready, cudaEventDisableTiming));
    CBCT_CUDA_TRY(cudaEventRecord(sl.ready, sa));
    return CBCT_OK;
}

// Frees the slot's buffers on stream `st`; the geometry is destroyed at once
// or (keep_geometry) left in the graveyard for a quiet moment.
void ServerImpl::release_slot(Slot &sl, cudaStream_t st, bool keep_geometry) {
    for (void *p : {(void *)sl.U, (void *)sl.Uw, (void *)sl.b, (void *)sl.V, (void *)sl.w, (void *)sl.x, (void *)sl.h2,
                    (void *)sl.pf, (void *)sl.pb, (void *)sl.pfold, (void *)sl.st, (void *)sl.hist})
        if (p) cudaFreeAsync(p, st);
    sl.U = sl.Uw = sl.b = sl.V = sl.w = sl.x = sl.h2 = nullptr;
    sl.pf = sl.pb = sl.pfold = sl.hist = nullptr;
    sl.st = nullptr;
    if (sl.ready) {
        cudaEventDestroy(sl.ready);
        sl.ready = nullptr;
    }
    if (sl.solo_graph) {
        cudaGraphExecDestroy(sl.solo_graph);
        sl.solo_graph = nullptr;
    }
    if (sl.geom) {
        cudaStreamSynchronize(st);
        if (keep_geometry) {
            std::lock_guard<std::mutex> lk(mu);
            graveyard.push_back(sl.geom);
        } else {
            cbct_geometry_destroy(sl.geom);
        }
        sl.geom = nullptr;
    }
}

// On the read-out thread and stream: x (caller layout), histories and final state.
cbct_status ServerImpl::finish_slot(Slot &sl) {
    Request &r = *sl.req;
    const int64_t m = cbct_geometry_num_voxels(sl.geom);
    cudaStream_t sr = s_read;
    float *tmp = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync(&tmp, sizeof(float) * m, sr));
    cbct_status st = launch_relayout(sl.geom->dev, sl.x, tmp, CBCT_F32, false, sr);
    r.x.assign((size_t)m, 0.0f);
    r.hist_r.assign((size_t)r.iters, 0.0);
    r.hist_n.assign((size_t)r.iters, 0.0);
    GkState fin;
    cudaError_t e = cudaSuccess;
    if (st == CBCT_OK) e = cudaMemcpyAsync(r.x.data(), tmp, sizeof(float) * m, cudaMemcpyDeviceToHost, sr);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r.hist_r.data(), sl.hist, sizeof(double) * r.iters, cudaMemcpyDeviceToHost, sr);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r.hist_n.data(), sl.hist + r.iters, sizeof(double) * r.iters, cudaMemcpyDeviceToHost, sr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fin, sl.st, sizeof fin, cudaMemcpyDeviceToHost, sr);
    cudaFreeAsync(tmp, sr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sr);
    if (st != CBCT_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "server: read-out");
    r.iters_done = fin.iter;
    r.status = (cbct_status)fin.status;
    if (r.status == CBCT_EBREAKDOWN) r.error = "Krylov breakdown: a norm became zero or non-finite";
    return CBCT_OK;
}

// Marks a request done (its memory already released) and wakes waiters and admission.
void ServerImpl::complete(const std::shared_ptr<Request> &r, cbct_status st, const std::string &msg) {
    publish(r, st, msg);
    return_budget(r);
}

// Marks a request done and wakes its waiters (its memory may still be held).
void ServerImpl::publish(const std::shared_ptr<Request> &r, cbct_status st, const std::string &msg) {
    {
        std::lock_guard<std::mutex> lk(mu);
        if (st != CBCT_OK) r->status = st;
        if (!msg.empty()) r->error = msg;
        r->done = true;
        r->t_finish = now_s(t0);
    }
    cv_done.notify_all();
}

// Gives a request's memory back to the budget (its buffers already freed) and wakes admission.
void ServerImpl::return_budget(const std::shared_ptr<Request> &r) {
    {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= r->bytes;
    }
    cv_admit.notify_one();
}

// One Krylov iteration of every slot, then the per-slot status to the host.
// A step of one slot whose tiles fill the GPU alone runs the single-request
// projector kernels instead of the multi-slot ones (the geometry in kernel
// parameters, no tile claiming); both walk the same tiles in the same order
// and leave the norm partials in the same places, so the results agree
// bit for bit.  That step is captured once per slot.
cbct_status ServerImpl::enqueue_step() {
    Slot *solo = solo_step() ? &slots[step_slots[0]] : nullptr;
    auto launch_all = [&]() -> cudaError_t {
        if (solo) {
            const DevGeom &g = solo->geom->dev;
            const Epilogue ef{&solo->st->fa, &solo->st->fb, 0.0, 0.0, solo->pf, &solo->st->stop, nullptr, solo->Uw};
            const Epilogue eb{&solo->st->ba, &solo->st->bb, 0.0, 0.0, solo->pb, &solo->st->stop, nullptr};
            if (launch_forward(g, solo->V, solo->U, CBCT_F32, ef, s, true) != CBCT_OK) return cudaErrorLaunchFailure;
            if (solo->nf * TILE_PARTIALS > FOLD_MIN)
                k_fold_partials<RED_THREADS><<<FOLD_BLOCKS, RED_THREADS, 0, s>>>(solo->pf, solo->nf * TILE_PARTIALS,
                                                                                solo->pfold);
            srv_after_forward<<<1, RED_THREADS, 0, s>>>(tab_dev);
            if (launch_backward(g, solo->Uw, solo->V, CBCT_F32, eb, s, true, nullptr) != CBCT_OK)
                return cudaErrorLaunchFailure;
            if (solo->nb * TILE_PARTIALS > FOLD_MIN)
                k_fold_partials<RED_THREADS><<<FOLD_BLOCKS, RED_THREADS, 0, s>>>(solo->pb, solo->nb * TILE_PARTIALS,
                                                                                solo->pfold + FOLD_BLOCKS);
            srv_after_backward<<<1, RED_THREADS, 0, s>>>(tab_dev);
        } else {
            cudaError_t e0 = cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned), s);
            if (e0 != cudaSuccess) return e0;
            srv_forward<<<fwd_grid, FWD_THREADS, 0, s>>>(tab_dev, counters);
            srv_after_forward<<<SRV_MAX_SLOTS, RED_THREADS, 0, s>>>(tab_dev);
            srv_backward<<<bwd_grid, BWD_THREADS, 0, s>>>(tab_dev, counters + 1);
            srv_after_backward<<<SRV_MAX_SLOTS, RED_THREADS, 0, s>>>(tab_dev);
        }
        srv_update<<<vec_grid, VEC_THREADS, 0, s>>>(tab_dev);
        srv_status<<<1, SRV_MAX_SLOTS, 0, s>>>(tab_dev, stat_dev);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(stat_host, stat_dev, sizeof(SlotStatus) * SRV_MAX_SLOTS, cudaMemcpyDeviceToHost, s);
        return e;
    };
    cudaGraphExec_t &exec = solo ? solo->solo_graph : step_graph;
    if (use_graph && !exec) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = launch_all();
            e = cudaStreamEndCapture(s, &graph);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {             // fall back to plain launches
            (void)cudaGetLastError();
            exec = nullptr;
            use_graph = 0;
        }
    }
    if (use_graph && exec) {
        CBCT_CUDA_TRY(cudaGraphLaunch(exec, s));
        ++graph_replays;
        return CBCT_OK;
    }
    CBCT_CUDA_TRY(launch_all());
    return CBCT_OK;
}

// ---------------------------------------------------------------- schedules

// FIFO: the slots in submission order; SRPT: the least remaining work
// (iterations left x cost of one), ties by request id, except that slots
// passed over for SRV_SRPT_AGE_CAP consecutive steps go first from then on
// (oldest first), so a long request cannot wait for ever behind a stream of
// short ones; RATIO: the highest
// response ratio (time since submission + remaining time) / remaining time,
// the remaining time from the cost model and the measured work rate.  All
// three take slots in that order as long as the step's forward tiles stay
// within SRV_SAT_TILES (the first slot always runs).  SHARE: every slot.
// Returned in increasing slot index.
std::vector<int> ServerImpl::pick_step_slots() const {
    std::vector<int> all(slots.size());
    for (size_t i = 0; i < slots.size(); ++i) all[i] = (int)i;
    if (schedule == CBCT_SCHED_SHARE) return all;
    auto remaining = [&](int i) { return (slots[i].req->iters - slots[i].steps) * slots[i].work_iter; };
    std::vector<double> key(slots.size());
    const double now = now_s(t0);
    for (size_t i = 0; i < slots.size(); ++i) {
        const double rem = remaining((int)i);
        if (schedule == CBCT_SCHED_FIFO) {
            key[i] = (double)slots[i].req->id;
        } else if (schedule == CBCT_SCHED_SRPT && slots[i].aged) {
            key[i] = -1e300 + (double)slots[i].req->id;        // aged: ahead of every fresh slot, oldest first
        } else if (schedule == CBCT_SCHED_RATIO && work_rate > 0.0) {
            const double rem_s = std::max(rem / work_rate, 1e-6);
            key[i] = -(now - slots[i].req->t_submit + rem_s) / rem_s;       // higher ratio first
        } else {
            key[i] = rem;
        }
    }
    std::sort(all.begin(), all.end(), [&](int a, int b) {
        return key[a] != key[b] ? key[a] < key[b] : slots[a].req->id < slots[b].req->id;
    });
    std::vector<int> pick;
    int64_t tiles = 0;
    for (int i : all) {
        // a step's duration is its total work: never let a request join (and
        // slow down) a step that the ones before it in the order already fill
        if (!pick.empty() && tiles + slots[i].nf > SRV_SAT_TILES) break;
        pick.push_back(i);
        tiles += slots[i].nf;
    }
    std::sort(pick.begin(), pick.end());
    return pick;
}

// ------------------------------------------------------------------ threads

void ServerImpl::run_admission() {
    cudaSetDevice(device);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_admit.wait(lk, [&] {
                return stopping || (!pending.empty() && in_flight < max_slots &&
                                    in_use + pending.front()->bytes <= budget);
            });
            if (stopping) break;
            r = pending.front();
            pending.pop_front();
            in_use += r->bytes;
            ++in_flight;
            r->t_admit = now_s(t0);
            r->admitted = true;
        }
        Slot sl;
        sl.req = r;
        cbct_status st = setup_slot(sl);
        if (st != CBCT_OK) {
            const std::string msg = cbct_last_error();
            release_slot(sl, s_admit, false);
            {
                std::lock_guard<std::mutex> lk(mu);
                --in_flight;
            }
            complete(r, st, msg);
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            ready.push_back(sl);
        }
        cv_ready.notify_one();
    }
}

void ServerImpl::run_steps() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<Slot> incoming;
        std::vector<cbct_geometry *> dead;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (slots.empty()) cv_ready.wait(lk, [&] { return stopping || !ready.empty(); });
            if (stopping) break;
            incoming.swap(ready);
            active_slots = (int)(slots.size() + incoming.size());
            if (slots.empty() && finishing.empty()) dead.swap(graveyard);     // a quiet moment
        }
        for (cbct_geometry *g : dead) cbct_geometry_destroy(g);
        for (Slot &sl : incoming) {
            cudaStreamWaitEvent(s, sl.ready, 0);          // the step stream follows the slot's set-up
            slots.push_back(sl);
            table_dirty = true;
        }
        if (slots.empty()) continue;
        {
            std::vector<int> pick = pick_step_slots();
            std::vector<char> in_step(slots.size(), 0);
            for (int i : pick) in_step[i] = 1;
            for (size_t i = 0; i < slots.size(); ++i) {
                slots[i].passed_over = in_step[i] ? 0 : slots[i].passed_over + 1;
                if (slots[i].passed_over >= SRV_SRPT_AGE_CAP) slots[i].aged = true;
            }
            if (pick != step_slots) {
                step_slots.swap(pick);
                table_dirty = true;
            }
        }
        if (table_dirty) {
            SlotTable &t = *tab_host;
            t.n = (int)step_slots.size();
            t.fwd_start[0] = t.bwd_start[0] = 0;
            for (int i = 0; i < t.n; ++i) {
                const Slot &sl = slots[step_slots[i]];
                SlotDev &d = t.s[i];
                d.g = sl.geom->dev;
                d.U = sl.U; d.Uw = sl.Uw; d.V = sl.V; d.w = sl.w; d.x = sl.x; d.h2 = sl.h2;
                d.st = sl.st;
                d.pf = sl.pf; d.pb = sl.pb;
                // a step of this slot alone folds its partials first (enqueue_step)
                const bool fold_f = solo_step() && sl.nf * TILE_PARTIALS > FOLD_MIN;
                const bool fold_b = solo_step() && sl.nb * TILE_PARTIALS > FOLD_MIN;
                d.qf = fold_f ? sl.pfold : sl.pf;
                d.nqf = fold_f ? FOLD_BLOCKS : sl.nf * TILE_PARTIALS;
                d.qb = fold_b ? sl.pfold + FOLD_BLOCKS : sl.pb;
                d.nqb = fold_b ? FOLD_BLOCKS : sl.nb * TILE_PARTIALS;
                d.hist_r = sl.hist; d.hist_n = sl.hist + sl.req->iters;
                d.method = sl.req->method;
                d.cap = sl.req->iters;
                const dim3 fg = forward_grid(d.g), bg = backward_grid(d.g);
                d.fgx = fg.x; d.fgy = fg.y; d.bgx = bg.x; d.bgy = bg.y;
                d.m = zf_len(d.g);
                t.fwd_start[i + 1] = t.fwd_start[i] + sl.nf;
                t.bwd_start[i + 1] = t.bwd_start[i] + sl.nb;
            }
            cudaError_t e = cudaMemcpyAsync(tab_dev, tab_host, sizeof(SlotTable), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) table_dirty = false;
        }
        // Steps queued before the host looks at the status again: under FIFO a
        // slot that fills the GPU alone stays the only one picked until it
        // finishes (nothing older waits and nothing fits beside it), so all
        // its remaining iterations are queued at once (a slot that stops
        // early turns the rest into no-ops); otherwise one.
        int run = 1;
        if (schedule == CBCT_SCHED_FIFO && solo_step())
            run = std::max(1, slots[step_slots[0]].req->iters - slots[step_slots[0]].steps);
        const double t_step = now_s(t0);
        cbct_status st = table_dirty ? cuda_fail(cudaGetLastError(), "server: slot table") : CBCT_OK;
        for (int q = 0; q < run && st == CBCT_OK; ++q) st = enqueue_step();
        cudaError_t e = cudaStreamSynchronize(s);
        {   // running estimate of the work rate (cost-model units per second)
            double w = 0.0;
            for (int i : step_slots) w += slots[i].work_iter * run;
            const double dt = now_s(t0) - t_step;
            if (dt > 0.0 && w > 0.0) work_rate = work_rate > 0.0 ? 0.8 * work_rate + 0.2 * (w / dt) : w / dt;
        }
        if (st != CBCT_OK || e != cudaSuccess) {
            if (e != cudaSuccess) st = cuda_fail(e, "server: step");
            const std::string msg = cbct_last_error();
            std::vector<Slot> failed;
            failed.swap(slots);
            step_slots.clear();
            table_dirty = true;
            for (Slot &sl : failed) {
                std::shared_ptr<Request> r = sl.req;
                release_slot(sl, s, false);
                {
                    std::lock_guard<std::mutex> lk(mu);
                    --in_flight;
                }
                complete(r, st, msg);
            }
            continue;
        }
        steps_run += run;
        // table entries are in increasing slot index: walk them backwards so that
        // erasing a finished slot leaves the remaining indices valid
        std::vector<Slot> done_now;
        for (int ti = (int)step_slots.size() - 1; ti >= 0; --ti) {
            const int i = step_slots[ti];
            Slot &sl = slots[i];
            sl.steps += run;
            if (!stat_host[ti].stop && sl.steps < sl.req->iters) continue;
            done_now.push_back(sl);
            slots.erase(slots.begin() + i);
        }
        if (!done_now.empty()) {
            step_slots.clear();              // slot indices shifted: the next step re-picks
            table_dirty = true;
            {
                std::lock_guard<std::mutex> lk(mu);
                in_flight -= (int)done_now.size();
                active_slots = (int)slots.size();
                for (Slot &sl : done_now) finishing.push_back(sl);
            }
            cv_finish.notify_one();
            cv_admit.notify_one();           // a slot is free (its memory follows at read-out)
        }
    }
    for (Slot &sl : slots) {
        std::shared_ptr<Request> r = sl.req;
        release_slot(sl, s, false);
        complete(r, CBCT_EINVAL, "server destroyed before the request finished");
    }
    slots.clear();
    cudaStreamSynchronize(s);
}

void ServerImpl::run_readout() {
    cudaSetDevice(device);
    for (;;) {
        Slot sl;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_finish.wait(lk, [&] { return steps_stopped || !finishing.empty(); });
            if (finishing.empty()) break;        // steps stopped and nothing left to read out
            sl = finishing.front();
            finishing.pop_front();
        }
        cbct_status fs = finish_slot(sl);
        const std::string msg = fs == CBCT_OK ? std::string() : std::string(cbct_last_error());
        std::shared_ptr<Request> r = sl.req;
        publish(r, fs, msg);                     // the result is on the host: the waiter may go on
        release_slot(sl, s_read, true);
        return_budget(r);
    }
}

}  // namespace cbct

using namespace cbct;

struct cbct_server {
    ServerImpl impl;
};

static void free_server_resources(ServerImpl &S) {
    if (S.tab_host) cudaFreeHost(S.tab_host);
    if (S.tab_dev) cudaFree(S.tab_dev);
    if (S.stat_host) cudaFreeHost(S.stat_host);
    if (S.stat_dev) cudaFree(S.stat_dev);
    if (S.counters) cudaFree(S.counters);
    for (cudaStream_t st : {S.s, S.s_admit, S.s_read})
        if (st) cudaStreamDestroy(st);
}

extern "C" cbct_status cbct_server_create(const cbct_server_opts *o, cbct_server **out) {
    if (!o || !out) { set_error("cbct_server_create: null argument"); return CBCT_EINVAL; }
    *out = nullptr;
    if (o->hbm_budget_bytes == 0 || o->max_slots < 1 || o->max_slots > SRV_MAX_SLOTS) {
        set_error("cbct_server_create: need hbm_budget_bytes > 0 and 1 <= max_slots <= 64");
        return CBCT_EINVAL;
    }
    if (o->schedule != CBCT_SCHED_SRPT && o->schedule != CBCT_SCHED_SHARE && o->schedule != CBCT_SCHED_RATIO &&
        o->schedule != CBCT_SCHED_FIFO) {
        set_error("cbct_server_create: unknown schedule");
        return CBCT_EINVAL;
    }
    cbct_server *srv = new (std::nothrow) cbct_server();
    if (!srv) { set_error("cbct_server_create: out of host memory"); return CBCT_ENOMEM; }
    ServerImpl &S = srv->impl;
    S.budget = o->hbm_budget_bytes;
    S.max_slots = o->max_slots;
    S.use_graph = o->use_graph != 0;
    S.schedule = o->schedule;
    S.t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&S.device);
    int sms = 0, occ_f = 0, occ_b = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S.device);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, srv_forward, FWD_THREADS, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, srv_backward, BWD_THREADS, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S.s_admit, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S.s_read, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&S.tab_host, sizeof(SlotTable));
    if (e == cudaSuccess) e = cudaMalloc(&S.tab_dev, sizeof(SlotTable));
    if (e == cudaSuccess) e = cudaMallocHost(&S.stat_host, sizeof(SlotStatus) * SRV_MAX_SLOTS);
    if (e == cudaSuccess) e = cudaMalloc(&S.stat_dev, sizeof(SlotStatus) * SRV_MAX_SLOTS);
    if (e == cudaSuccess) e = cudaMalloc(&S.counters, 2 * sizeof(unsigned));
    if (e != cudaSuccess) {
        cbct_status st = cuda_fail(e, "cbct_server_create");
        free_server_resources(S);
        delete srv;
        return st;
    }
    std::memset(S.tab_host, 0, sizeof(SlotTable));
    S.fwd_grid = sms * std::max(occ_f, 1);
    S.bwd_grid = sms * std::max(occ_b, 1);
    S.vec_grid = sms * 4;
    try {
        S.reader = std::thread([&S] { S.run_readout(); });
        S.worker = std::thread([&S] { S.run_steps(); });
        S.admitter = std::thread([&S] { S.run_admission(); });
    } catch (...) {
        set_error("cbct_server_create: cannot start the server threads");
        {
            std::lock_guard<std::mutex> lk(S.mu);
            S.stopping = S.steps_stopped = true;
        }
        S.cv_admit.notify_all();
        S.cv_ready.notify_all();
        S.cv_finish.notify_all();
        for (std::thread *t : {&S.admitter, &S.worker, &S.reader})
            if (t->joinable()) t->join();
        free_server_resources(S);
        delete srv;
        return CBCT_ENOMEM;
    }
    *out = srv;
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_request_bytes(const cbct_geometry_desc *desc, cbct_solver solver, int iters,
                                                 size_t *bytes) {
    if (!desc || !bytes) { set_error("cbct_server_request_bytes: null argument"); return CBCT_EINVAL; }
    if (solver != CBCT_SOLVER_LSQR && solver != CBCT_SOLVER_LSMR) {
        set_error("cbct_server_request_bytes: solver must be LSQR or LSMR");
        return CBCT_EINVAL;
    }
    if (iters < 1) { set_error("cbct_server_request_bytes: need iters >= 1"); return CBCT_EINVAL; }
    const cbct_status st = validate_geometry_desc(desc);
    if (st != CBCT_OK) return st;
    *bytes = request_bytes(*desc, solver == CBCT_SOLVER_LSQR ? M_LSQR : M_LSMR, iters);
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_submit(cbct_server *srv, const cbct_geometry_desc *desc, const float *b_host,
                                          cbct_solver solver, const cbct_solve_opts *o, uint64_t *id) {
    if (!srv || !desc || !b_host || !o || !id) { set_error("cbct_server_submit: null argument"); return CBCT_EINVAL; }
    if (solver != CBCT_SOLVER_LSQR && solver != CBCT_SOLVER_LSMR) {
        set_error("cbct_server_submit: solver must be LSQR or LSMR");
        return CBCT_EINVAL;
    }
    if (o->iters < 1 || o->storage != CBCT_F32 || !(o->lambda >= 0.0) || !std::isfinite(o->lambda)) {
        set_error("cbct_server_submit: need iters >= 1, FP32 storage and a finite lambda >= 0");
        return CBCT_EINVAL;
    }
    cbct_status st = validate_geometry_desc(desc);
    if (st != CBCT_OK) return st;
    ServerImpl &S = srv->impl;
    const int method = solver == CBCT_SOLVER_LSQR ? M_LSQR : M_LSMR;
    const size_t bytes = request_bytes(*desc, method, o->iters);
    if (bytes > S.budget) {
        set_error("cbct_server_submit: the request needs more device memory than the server's budget");
        return CBCT_EBUDGET;
    }
    std::shared_ptr<Request> r;
    try {
        r = std::make_shared<Request>();
        r->desc = *desc;
        r->angles.assign(desc->angles_rad, desc->angles_rad + desc->nangles);
        const size_t n = (size_t)desc->nangles * desc->nv * desc->nu;
        r->b.assign(b_host, b_host + n);
    } catch (...) {
        set_error("cbct_server_submit: out of host memory");
        return CBCT_ENOMEM;
    }
    r->method = method;
    r->iters = o->iters;
    r->damp = o->lambda;
    r->bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        r->t_submit = now_s(S.t0);
        r->id = S.next_id++;
        S.requests[r->id] = r;
        S.pending.push_back(r);
        *id = r->id;
    }
    S.cv_admit.notify_one();
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_poll(cbct_server *srv, uint64_t id, int *done) {
    if (!srv || !done) { set_error("cbct_server_poll: null argument"); return CBCT_EINVAL; }
    std::lock_guard<std::mutex> lk(srv->impl.mu);
    auto it = srv->impl.requests.find(id);
    if (it == srv->impl.requests.end()) { set_error("cbct_server_poll: unknown request"); return CBCT_ENOTFOUND; }
    *done = it->second->done ? 1 : 0;
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_wait(cbct_server *srv, uint64_t id, double timeout_s, float *x_host,
                                        cbct_solve_report *rep, cbct_request_times *times) {
    if (!srv) { set_error("cbct_server_wait: null server"); return CBCT_EINVAL; }
    ServerImpl &S = srv->impl;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.requests.find(id);
    if (it == S.requests.end()) { set_error("cbct_server_wait: unknown request"); return CBCT_ENOTFOUND; }
    std::shared_ptr<Request> r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_s < 0.0) {
        S.cv_done.wait(lk, ready);
    } else if (!S.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        set_error("cbct_server_wait: request not finished within the time-out");
        return CBCT_ETIMEOUT;
    }
    if (x_host && !r->x.empty()) std::memcpy(x_host, r->x.data(), sizeof(float) * r->x.size());
    if (rep) {
        rep->iters_done = r->iters_done;
        const int c = std::min(r->iters_done, r->iters);
        if (rep->resid_norm && c > 0) std::memcpy(rep->resid_norm, r->hist_r.data(), sizeof(double) * c);
        if (rep->normal_resid_norm && c > 0) std::memcpy(rep->normal_resid_norm, r->hist_n.data(), sizeof(double) * c);
        rep->kernel_launches = rep->forward_launches = rep->backward_launches = 0;
        rep->forward_ms = rep->backward_ms = 0.0;
    }
    if (times) *times = cbct_request_times{r->t_submit, r->t_admit, r->t_finish};
    const cbct_status st = r->status;
    if (st != CBCT_OK) set_error(r->error);
    S.requests.erase(it);
    return st;
}

extern "C" cbct_status cbct_server_get_stats(cbct_server *srv, cbct_server_stats *out) {
    if (!srv || !out) { set_error("cbct_server_get_stats: null argument"); return CBCT_EINVAL; }
    ServerImpl &S = srv->impl;
    std::lock_guard<std::mutex> lk(S.mu);
    out->steps = S.steps_run;
    out->graph_replays = S.graph_replays;
    out->bytes_in_use = S.in_use;
    out->pending = (int)S.pending.size();
    int active = 0;
    for (auto &kv : S.requests)
        if (!kv.second->done && kv.second->admitted) ++active;
    out->active = active;
    return CBCT_OK;
}

extern "C" void cbct_server_destroy(cbct_server *srv) {
    if (!srv) return;
    ServerImpl &S = srv->impl;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stopping = true;
    }
    S.cv_admit.notify_all();
    S.cv_ready.notify_all();
    if (S.admitter.joinable()) S.admitter.join();
    if (S.worker.joinable()) S.worker.join();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.steps_stopped = true;
    }
    S.cv_finish.notify_all();
    if (S.reader.joinable()) S.reader.join();
    for (Slot &sl : S.ready) {                 // set up but never stepped
        std::shared_ptr<Request> r = sl.req;
        S.release_slot(sl, S.s_admit, false);
        S.complete(r, CBCT_EINVAL, "server destroyed before the request finished");
    }
    S.ready.clear();
    for (cbct_geometry *g : S.graveyard) cbct_geometry_destroy(g);
    S.graveyard.clear();
    if (S.step_graph) cudaGraphExecDestroy(S.step_graph);
    for (cudaStream_t st : {S.s, S.s_admit, S.s_read}) cudaStreamSynchronize(st);
    free_server_resources(S);
    delete srv;
}
