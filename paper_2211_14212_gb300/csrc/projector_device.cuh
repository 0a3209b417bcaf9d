// Device-side building blocks of the cone-beam projectors (Sec. 1, Eq. 1):
// the ray traversal shared by A and A^T, and one tile of each projector,
// callable from a plain grid (projector.cu) or from a persistent kernel that
// walks a work list spanning several problems (serve.cu).
//
// Work layout ("ray-column warps").  In a circular cone-beam scan every ray of
// one detector column (angle a, column iu) has the same projection onto the
// xy plane, so all of them cross the x and y voxel planes at the same alpha
// (the x/y tables depend on (a, iu) only).  A warp therefore takes rays of one
// detector column: lane l follows rows iv0 + r * 32 + l for r = 0..R-1.  The
// x/y plane stepping is identical in all lanes and is shared by the warp's
// 32 R rays; each ray only tracks its own z crossings, which are rare
// (|dz/d| <= the cone half-angle).  Volumes are read in a z-fastest layout
// x[j][i][k] so that the lanes of one row group, which sit at ~17 consecutive
// k of one voxel column, gather one contiguous run.
//
// Both projectors take every plane crossing from the per-ray tables of
// DevGeom through plane_alpha, so a ray/voxel segment has the same FP32 length
// in both: the backprojector is the transpose of the forward projector, not an
// approximation of it (the paper traces Krylov instabilities to unmatched
// backprojectors, Sec. 2.1.4 and Sec. 4).
#pragma once

#include <cfloat>

#include "common.cuh"

namespace cbct {

// One axis of one ray: offset f = plane(pq) - q, inverse direction I, and the
// index pq of the plane nearest to the ray origin (the fixed voxel index when
// I == 0, a ray parallel to the axis' planes).
struct RayAxis {
    float f, I, pq;
};

// Alpha at which a ray crosses plane pq + r of one axis (plane spacing delta):
// (r * delta + f) * I, rounded twice.  Both projectors use only this.
__device__ __forceinline__ float plane_alpha(float r, float delta, const RayAxis &a) {
    return __fmul_rn(__fmaf_rn(r, delta, a.f), a.I);
}

// One axis of the traversal: current voxel index i, step s (+1/-1, 0 when the
// ray is parallel to the axis' planes), index of the plane through which the
// ray leaves the current voxel (relative to pq, as float) and the alpha of
// that crossing.
struct Axis {
    int i, s;
    float r, e;
};

// Clip alpha interval [amin, amax] to the slab between planes plo and phi.
__device__ __forceinline__ void clip_slab(const RayAxis &ra, float delta, int plo, int phi, float &amin,
                                          float &amax, bool &miss) {
    if (ra.I == 0.0f) {
        if (!(ra.pq >= (float)plo && ra.pq < (float)phi)) miss = true;
        return;
    }
    const float a0 = plane_alpha((float)plo - ra.pq, delta, ra), a1 = plane_alpha((float)phi - ra.pq, delta, ra);
    amin = fmaxf(amin, fminf(a0, a1));
    amax = fminf(amax, fmaxf(a0, a1));
}

// Voxel index on one axis at alpha0, within [lo - 1, hi] (lo - 1 and hi stand
// for "before" and "beyond" the range).  The estimate from the ray position is
// corrected by comparing with the crossing alphas themselves, so the result is
// exactly the voxel whose alpha interval [entry, exit) contains alpha0.  The
// exit crossing is returned; it is FLT_MAX when the ray is outside the range
// and moving away from it.
__device__ __forceinline__ Axis axis_start(const RayAxis &ra, float delta, float alpha0, int lo, int hi) {
    Axis st;
    if (ra.I == 0.0f) {         // parallel: fixed index, never crossed
        st.i = (int)ra.pq;
        st.s = 0;
        st.r = 0.0f;
        st.e = FLT_MAX;
        return st;
    }
    // plane coordinate of the ray at alpha0: pq + (alpha0 / I - f) / delta
    int i = (int)floorf(ra.pq + (__fdividef(alpha0, ra.I) - ra.f) / delta);
    i = max(lo - 1, min(hi, i));
    auto al = [&](int p) { return plane_alpha((float)p - ra.pq, delta, ra); };
    if (ra.I > 0.0f) {          // alpha grows with the plane index: voxel i = [alpha(i), alpha(i+1))
        if (i < hi && al(i + 1) <= alpha0) ++i;
        if (i >= lo && al(i) > alpha0) --i;
        st.s = 1;
        st.r = (float)(i + 1) - ra.pq;
        st.e = i < hi ? plane_alpha(st.r, delta, ra) : FLT_MAX;
    } else {                    // alpha falls with the plane index: voxel i = [alpha(i+1), alpha(i))
        if (i >= lo && al(i) <= alpha0) --i;
        if (i < hi && al(i + 1) > alpha0) ++i;
        st.s = -1;
        st.r = (float)i - ra.pq;
        st.e = i >= lo ? plane_alpha(st.r, delta, ra) : FLT_MAX;
    }
    st.i = i;
    return st;
}

// Walk R rays of one detector column (shared xy tables rx, ry; z tables
// rz[r]) through the box [lox,hix) x [loy,hiy) x [loz,hiz) of voxels.  For
// every segment inside the box it calls
//     add(r, alpha_length, value),   value = fetch(cell + k),
//     cell = off + i * sx + j * sy,
// in order along each ray (cell is kept incrementally, so the caller picks the
// linear layout through off, sx, sy).  The value of the voxel a ray occupies
// when it enters the next xy cell is fetched before the current cell's
// segments are added, so each lane keeps R loads in flight across the
// latency of a step; a z crossing inside a cell (rare) fetches the new voxel
// on the spot.  Segments of rays outside [loz, hiz) are added with length 0
// and no fetch.  Returns false (uniformly across the warp) if the xy
// projection misses the box.
template <int R, typename Fetch, typename Add>
__device__ __forceinline__ bool trace_columns(const DevGeom &g, const RayAxis &rx, const RayAxis &ry,
                                              const RayAxis (&rz)[R], int lox, int hix, int loy, int hiy,
                                              int loz, int hiz, int off, int sx, int sy, Fetch &&fetch,
                                              Add &&add) {
    float amin = -FLT_MAX, amax = FLT_MAX;
    bool miss = false;
    clip_slab(rx, g.dx, lox, hix, amin, amax, miss);
    clip_slab(ry, g.dy, loy, hiy, amin, amax, miss);
    if (miss || !(amin < amax)) return false;

    Axis ax = axis_start(rx, g.dx, amin, lox, hix);
    Axis ay = axis_start(ry, g.dy, amin, loy, hiy);
    Axis az[R];
    bool inz[R];
    float cur[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        az[r] = axis_start(rz[r], g.dz, amin, loz, hiz);
        if (az[r].s == 0 && (az[r].i < loz || az[r].i >= hiz)) az[r].i = loz - 1;   // parallel outside
        inz[r] = az[r].i >= loz && az[r].i < hiz;
        cur[r] = amin;
    }
    int cell = off + ax.i * sx + ay.i * sy;
    const int dcx = ax.s * sx, dcy = ay.s * sy;
    float vnext[R];
#pragma unroll
    for (int r = 0; r < R; ++r) vnext[r] = inz[r] ? fetch(cell + az[r].i) : 0.0f;
    const int maxsteps = (hix - lox) + (hiy - loy) + 1;
#pragma unroll 1
    for (int n = 0; n < maxsteps; ++n) {
        const float e = fminf(ax.e, ay.e);
        float v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = vnext[r];
        float zmin = az[0].e;
#pragma unroll
        for (int r = 1; r < R; ++r) zmin = fminf(zmin, az[r].e);
        if (zmin < e) {                    // some ray of this lane crosses a z plane in this xy cell
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll 1
                while (az[r].e < e) {
                    if (inz[r]) add(r, az[r].e - cur[r], v[r]);
                    cur[r] = az[r].e;
                    az[r].i += az[r].s;
                    az[r].r += (float)az[r].s;
                    inz[r] = az[r].i >= loz && az[r].i < hiz;
                    az[r].e = inz[r] ? plane_alpha(az[r].r, g.dz, rz[r]) : FLT_MAX;
                    v[r] = inz[r] ? fetch(cell + az[r].i) : 0.0f;
                }
            }
        }
        float len[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            len[r] = inz[r] ? e - cur[r] : 0.0f;
            cur[r] = e;
        }
        bool done;
        if (e == ax.e) {
            ax.i += ax.s;
            done = (unsigned)(ax.i - lox) >= (unsigned)(hix - lox);
            if (!done) {
                cell += dcx;
                ax.r += (float)ax.s;
                ax.e = plane_alpha(ax.r, g.dx, rx);
            }
        } else {
            ay.i += ay.s;
            done = (unsigned)(ay.i - loy) >= (unsigned)(hiy - loy);
            if (!done) {
                cell += dcy;
                ay.r += (float)ay.s;
                ay.e = plane_alpha(ay.r, g.dy, ry);
            }
        }
        if (!done) {
#pragma unroll
            for (int r = 0; r < R; ++r) vnext[r] = inz[r] ? fetch(cell + az[r].i) : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (inz[r]) add(r, len[r], v[r]);
        if (done) break;
    }
    return true;
}

// xy tables of column (a, iu) and z tables of R rows iv0 + r * 32 + lane; rows
// outside [0, nv) (or past `row_end`) get a z axis that is parallel and
// outside every box, so the lane follows the warp without effect.
template <int R>
__device__ __forceinline__ void load_rays(const DevGeom &g, int a, int iu, int iv0, int row_end, RayAxis &rx,
                                          RayAxis &ry, RayAxis (&rz)[R]) {
    const float4 xy = g.ray_xy[(size_t)a * g.nu + iu];
    const float2 q = g.ray_xyq[(size_t)a * g.nu + iu];
    rx = RayAxis{xy.x, xy.y, q.x};
    ry = RayAxis{xy.z, xy.w, q.y};
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int iv = iv0 + r * 32 + lane;
        if (iv < row_end) {
            const float4 z = g.ray_z[iv];
            rz[r] = RayAxis{z.x, z.y, z.z};
        } else {
            rz[r] = RayAxis{0.0f, 0.0f, (float)(g.nz + 1)};
        }
    }
}

// ------------------------------------------------------------- forward A x
//
// One tile = 8 warps = 8 adjacent detector columns (iu) x 32 R detector rows
// (iv) of one angle.  The volume is read z-fastest: vol[(j * nx + i) * nz + k].
// Epilogue: proj = a * (A vol) + b * old (either projection layout), and one
// FP64 sum of squares of the stored values into *partial (when non-null).

constexpr int FWD_COLS = 8, FWD_THREADS = 32 * FWD_COLS;

template <typename T, bool COMP, int R, bool VFAST>
__device__ __forceinline__ void forward_tile(const DevGeom &g, const T *__restrict__ vol, T *__restrict__ proj,
                                             const Epilogue &epi, int tx, int ty, int a, double *partial,
                                             double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int iu = tx * FWD_COLS + warp;
    const int iv0 = ty * 32 * R;
    const bool col_ok = iu < g.nu;            // uniform across the warp
    float acc[R], comp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = comp[r] = 0.0f;
    if (col_ok) {
        RayAxis rx, ry, rz[R];
        load_rays<R>(g, a, iu, iv0, g.nv, rx, ry, rz);
        auto fetch = [&](int idx) { return Storage<T>::load(vol + idx); };
        auto seg = [&](int r, float len, float value) {
            const float term = len * value;
            if (COMP) {          // Kahan-compensated running sum
                const float yk = term - comp[r];
                const float t = acc[r] + yk;
                comp[r] = (t - acc[r]) - yk;
                acc[r] = t;
            } else {
                acc[r] += term;
            }
        };
        // z-fastest volume: voxel (i, j, k) at (j * nx + i) * nz + k
        trace_columns<R>(g, rx, ry, rz, 0, g.nx, 0, g.ny, 0, g.nz, 0, g.nz, g.nx * g.nz, fetch, seg);
    }
    double sq = 0.0;
    const double acoef = epi_a(epi), bcoef = epi_b(epi);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int iv = iv0 + r * 32 + lane;
        if (col_ok && iv < g.nv) {
            // output y[a][iu][iv] (v fastest: one warp writes consecutive rows) or y[a][iv][iu]
            const size_t ray = VFAST ? ((size_t)a * g.nu + iu) * g.nv + iv : ((size_t)a * g.nv + iv) * g.nu + iu;
            const float len = g.ray_len[(size_t)iu * g.nv + iv];
            double out = acoef * (double)(acc[r] * len);
            if (bcoef != 0.0) {
                const T *oldp = epi.old ? (const T *)epi.old : (const T *)proj;
                out += bcoef * (double)Storage<T>::ld_plain(oldp + ray);
            }
            const float stored = Storage<T>::round((float)out);
            Storage<T>::store(proj + ray, stored);
            if (VFAST && epi.weighted) epi.weighted[ray] = len * stored;
            sq += (double)stored * (double)stored;
        }
    }
    if (partial) {
        const double s = block_sum<FWD_THREADS>(sq, red);
        if (threadIdx.x == 0) *partial = s;
    }
}

// ---------------------------------------------------------- transpose A^T y
//
// Gather form: each lane owns voxels (i, j, k) of one voxel column and sums
// len * w over every ray that meets them, in registers, angle by angle;
// the volume is written once (fused epilogue), so there are no atomics and the
// result does not depend on scheduling.  A warp owns one column (i, j) and
// 32 K consecutive k (k = k0 + kk * 32 + lane); a tile is 8 warps on a
// CX x (8 / CX) patch of columns.  For every angle the warp projects the
// cell's four corners to find the detector columns whose xy projection
// crosses cell (i, j), and each lane the detector rows that can meet its
// voxel's z slab (v = z dsd / depth over the corners' depths).  For each such
// column the warp takes the alpha interval [ain, aout] of the crossing (x and
// y plane crossings, warp-uniform), and a lane takes for each of its rows
// the segment
//     [max(ain, z entry), min(aout, z exit)].
// The z entry/exit of a row's ray in slab k does not depend on the angle
// (circular orbit), so it is read from the table DevGeom::zbox, which
// plane_alpha filled at geometry creation: every length is bit-identical to
// the forward projector's, and A^T is the exact transpose.
// Projections are read v-fastest and pre-weighted by the ray length:
// w[a][iu][iv] = |d'| * y.

constexpr int BWD_THREADS = 256;
constexpr int BWD_SHORT_ROWS = 3;

// Angles [a_begin, a_end) are summed in one call.  A scan whose projections
// do not fit in L2 is summed in passes over blocks of angles (launch_backward):
// `acc_in` (if not null) holds the FP32 sums of the earlier passes and
// `acc_out` (if not null) receives the running sums instead of the volume, so
// only the last pass applies the epilogue.  Both are z-fastest, indexed like
// the internal volume; they may be the same buffer (each lane reads and writes
// only its own voxels).
template <typename T, bool ZFAST, int CX, int K>
__device__ __forceinline__ void backward_tile(const DevGeom &g, const float *__restrict__ wproj, T *__restrict__ vol,
                                              const Epilogue &epi, int tx, int ty, int tz, int a_begin, int a_end,
                                              const float *acc_in, float *acc_out, double *partial,
                                              double *red) {
    constexpr int CY = 8 / CX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = tx * CX + (warp % CX), j = ty * CY + (warp / CX);
    const int k0 = tz * 32 * K;
    const bool col_ok = i < g.nx && j < g.ny;          // uniform across the warp
    float acc[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int k = k0 + kk * 32 + lane;
        acc[kk] = acc_in && col_ok && k < g.nz ? acc_in[((size_t)j * g.nx + i) * g.nz + k] : 0.0f;
    }
    if (col_ok) {
        const float x0 = g.bx0 + i * g.dx, x1 = x0 + g.dx;
        const float y0 = g.by0 + j * g.dy, y1 = y0 + g.dy;
        const float cu = 0.5f * (g.nu - 1), cv = 0.5f * (g.nv - 1);
        // The detector windows below only select candidates (every length is
        // then computed exactly from plane_alpha), so they use fast
        // approximate divisions: their relative error (~1e-6) stays far below
        // the 0.05-pixel margins.
        const float inv_du = 1.0f / g.du, inv_dv = 1.0f / g.dv;
        const size_t nuv = (size_t)g.nu * g.nv;
        for (int a = a_begin; a < a_end; ++a) {
            const float2 cs = g.trig[a];
            float umin = FLT_MAX, umax = -FLT_MAX, magmin = FLT_MAX, magmax = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float px = (c & 1) ? x1 : x0, py = (c & 2) ? y1 : y0;
                const float along = g.dso - (px * cs.x + py * cs.y);   // > 0: source outside
                const float mag = __fdividef(g.dsd, along);
                const float u = (-px * cs.y + py * cs.x) * mag;
                umin = fminf(umin, u);
                umax = fmaxf(umax, u);
                magmin = fminf(magmin, mag);
                magmax = fmaxf(magmax, mag);
            }
            const int iu0 = max(0, (int)ceilf(__fmaf_rn(umin, inv_du, cu - 0.05f)));
            const int iu1 = min(g.nu - 1, (int)floorf(__fmaf_rn(umax, inv_du, cu + 0.05f)));
            // Rows that can meet the lane's voxel at this angle: a point at
            // height z and source depth `along` lies on row v = z dsd / along,
            // and the column's depths span the corners' (mag = dsd / along is
            // extreme at a corner).  The window holds for every detector
            // column below; a row that misses the voxel for one of them adds
            // an exact zero.
            int r0[K], r1[K];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int k = k0 + kk * 32 + lane;
                const float zlo = (g.bz0 + k * g.dz) * inv_dv, zhi = (g.bz0 + (k + 1) * g.dz) * inv_dv;
                const float vmin = fminf(zlo * magmin, zlo * magmax);
                const float vmax = fmaxf(zhi * magmin, zhi * magmax);
                r0[kk] = max(0, (int)ceilf(vmin + (cv - 0.05f)));
                r1[kk] = k < g.nz ? min(g.nv - 1, (int)floorf(vmax + (cv + 0.05f))) : -1;
            }
            // Windows of at most BWD_SHORT_ROWS rows in every lane (the usual
            // case: a slab spans dz * mag / dv rows) take a fixed, predicated
            // sequence instead of a loop; the same rows are summed in the same
            // order either way.
            bool short_rows = true;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) short_rows = short_rows && r1[kk] - r0[kk] < BWD_SHORT_ROWS;
            short_rows = __all_sync(0xffffffffu, short_rows);
            const float *pa = wproj + (size_t)a * nuv;
            for (int iu = iu0; iu <= iu1; ++iu) {
                const float4 xy = g.ray_xy[(size_t)a * g.nu + iu];
                const float2 q = g.ray_xyq[(size_t)a * g.nu + iu];
                float ain = -FLT_MAX, aout = FLT_MAX;
                bool miss = false;
                clip_slab(RayAxis{xy.x, xy.y, q.x}, g.dx, i, i + 1, ain, aout, miss);
                clip_slab(RayAxis{xy.z, xy.w, q.y}, g.dy, j, j + 1, ain, aout, miss);
                if (miss || !(ain < aout)) continue;
                const float *wcol = pa + (size_t)iu * g.nv;
                if (short_rows) {
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const float2 *zb = g.zbox + (size_t)(k0 + kk * 32 + lane) * g.nv;
#pragma unroll
                        for (int t = 0; t < BWD_SHORT_ROWS; ++t) {
                            const int iv = r0[kk] + t;
                            if (iv <= r1[kk]) {
                                const float2 e = zb[iv];
                                const float lo = fmaxf(ain, e.x), hi = fminf(aout, e.y);
                                acc[kk] = __fmaf_rn(fmaxf(hi - lo, 0.0f), __ldg(wcol + iv), acc[kk]);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const float2 *zb = g.zbox + (size_t)(k0 + kk * 32 + lane) * g.nv;
                        for (int iv = r0[kk]; iv <= r1[kk]; ++iv) {
                            const float2 e = zb[iv];         // row iv's alpha interval in slab k
                            const float lo = fmaxf(ain, e.x), hi = fminf(aout, e.y);
                            // a miss adds exactly zero: the same sum as skipping it
                            acc[kk] = __fmaf_rn(fmaxf(hi - lo, 0.0f), __ldg(wcol + iv), acc[kk]);
                        }
                    }
                }
            }
        }
    }
    if (acc_out) {                      // an earlier pass: keep the running sums
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int k = k0 + kk * 32 + lane;
            if (col_ok && k < g.nz) acc_out[((size_t)j * g.nx + i) * g.nz + k] = acc[kk];
        }
        return;
    }
    const double acoef = epi_a(epi), bcoef = epi_b(epi);
    double sq = 0.0;
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int k = k0 + kk * 32 + lane;
        if (!col_ok || k >= g.nz) continue;
        const size_t v = ZFAST ? ((size_t)j * g.nx + i) * g.nz + k : ((size_t)k * g.ny + j) * g.nx + i;
        double out = acoef * (double)acc[kk];
        if (bcoef != 0.0) {
            const T *oldp = epi.old ? (const T *)epi.old : (const T *)vol;
            out += bcoef * (double)Storage<T>::ld_plain(oldp + v);
        }
        const float stored = Storage<T>::round((float)out);
        Storage<T>::store(vol + v, stored);
        sq += (double)stored * (double)stored;
    }
    if (partial) {
        const double s = block_sum<BWD_THREADS>(sq, red);
        if (threadIdx.x == 0) *partial = s;
    }
}

}  // namespace cbct
