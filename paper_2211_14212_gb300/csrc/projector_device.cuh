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
// DevGeom (the x/y crossings through plane_alpha in both), so the
// backprojector is the transpose of the forward projector, not an
// approximation of it (the paper traces Krylov instabilities to unmatched
// backprojectors, Sec. 2.1.4 and Sec. 4); in FP32 their segment lengths agree
// to rounding.
#pragma once

#include <cfloat>
#include <type_traits>

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

// ------------------------------------------- z index from alpha (forward)
//
// Along a ray the z voxel coordinate is linear in alpha: measured from the
// plane pq nearest to the ray origin, zeta(alpha) - pq = alpha / (dz I) -
// f / dz.  Its floor, the voxel index k, comes from one FMA and one add of
// 1.5 * 2^23 + pq (the add rounds to an integer, and the float's bits are
// then k + MAGIC_BITS); k - pq comes back exactly by subtracting the same
// constant.  The alpha at which the ray leaves voxel k through a z plane is
// (k - pq) (dz I) + c, both terms small (no cancellation).  alpha is clamped to
// the ray's range inside [0, nz) along z, so every segment outside the volume
// has zero length and k stays in [-1, nz].
constexpr float ZMAGIC = 12582912.0f;        // 1.5 * 2^23
constexpr int ZMAGIC_BITS = 0x4B400000;

struct RayZ {
    float a, b;          // (zeta - pq) - 0.5 = a * alpha + b (voxel units)
    float m;             // ZMAGIC + pq
    float inva, c;       // exit-plane alpha of voxel k: (k - pq) * inva + c
    float lo, hi;        // alpha range inside the slab [0, nz)
    int soff;            // +1 / -1 / 0: neighbour voxel across the exit plane
};

__device__ __forceinline__ RayZ make_rayz(const RayAxis &rz, float dz, int nz) {
    RayZ r;
    r.m = ZMAGIC + rz.pq;
    if (rz.I == 0.0f) {                          // parallel to the z planes: fixed voxel pq
        const bool in = rz.pq >= 0.0f && rz.pq < (float)nz;
        r.a = r.b = r.inva = 0.0f;
        r.c = FLT_MAX;
        r.lo = in ? -FLT_MAX : 0.0f;
        r.hi = in ? FLT_MAX : 0.0f;
        r.soff = 0;
        return r;
    }
    const float a0 = plane_alpha(0.0f - rz.pq, dz, rz), a1 = plane_alpha((float)nz - rz.pq, dz, rz);
    r.lo = fminf(a0, a1);
    r.hi = fmaxf(a0, a1);
    r.inva = dz * rz.I;
    r.a = 1.0f / r.inva;
    r.b = -rz.f / dz - 0.5f;
    const bool up = rz.I > 0.0f;                 // alpha grows with the plane index
    r.c = up ? (dz + rz.f) * rz.I : rz.f * rz.I; // exit plane of voxel k: k + 1 (up) or k (down)
    r.soff = up ? 1 : -1;
    return r;
}

// Forward traversal of R rays of one detector column through the padded
// z-fastest volume, for geometries with at most one z-plane crossing per xy
// cell (DevGeom::zsingle).  At every xy cell boundary e each ray adds
//     (e - e_prev) v + max(e - ze, 0) (vn - v),
// v and vn the voxel it occupied on entering the cell and its neighbour across
// the next z plane (crossed at ze if ze < e): both are loaded for every cell,
// so no lane branches.  The next cell's voxel index comes from zeta(e).  Ray
// pairs use packed FP32x2 arithmetic unless COMP (Kahan-compensated sums, for
// 16-bit storage).  Returns the ray sums in acc (alpha units).
template <typename T, bool COMP, int R>
__device__ __forceinline__ void trace_rays_zsingle(const DevGeom &g, const T *__restrict__ vol, const RayAxis &rx,
                                                   const RayAxis &ry, const RayAxis (&rzax)[R], float (&acc)[R]) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    float amin = -FLT_MAX, amax = FLT_MAX;
    bool miss = false;
    clip_slab(rx, g.dx, 0, nx, amin, amax, miss);
    clip_slab(ry, g.dy, 0, ny, amin, amax, miss);
    if (miss || !(amin < amax)) return;
    Axis ax = axis_start(rx, g.dx, amin, 0, nx);
    Axis ay = axis_start(ry, g.dy, amin, 0, ny);
    const int sx = nz + 2, sy = nx * (nz + 2);
    // index of voxel k of the current column is base + bits(k + ZMAGIC)
    int base = (int)zf_col(g, ax.i, ay.i) - ZMAGIC_BITS;
    RayZ z[R];
    float kf[R], v[R], vn[R], ep[R], comp[R];
    auto ld = [&](int idx) { return Storage<T>::load(vol + idx); };
#pragma unroll
    for (int r = 0; r < R; ++r) {
        z[r] = make_rayz(rzax[r], g.dz, nz);
        ep[r] = fminf(fmaxf(amin, z[r].lo), z[r].hi);
        const float kb = __fadd_rn(__fmaf_rn(ep[r], z[r].a, z[r].b), z[r].m);
        kf[r] = __fadd_rn(kb, -z[r].m);
        const int idx = base + __float_as_int(kb);
        v[r] = ld(idx);
        vn[r] = ld(idx + z[r].soff);
        comp[r] = 0.0f;
    }
    auto kahan = [&](int r, float term) {
        const float yk = term - comp[r];
        const float t = acc[r] + yk;
        comp[r] = (t - acc[r]) - yk;
        acc[r] = t;
    };
    const int dcx = ax.s * sx, dcy = ay.s * sy;
    const int maxsteps = nx + ny + 1;
#pragma unroll 1
    for (int n = 0; n < maxsteps; ++n) {
        const float e = fminf(ax.e, ay.e);
        float kbn[R];
        if (!COMP && R % 2 == 0) {
#pragma unroll
            for (int p = 0; p < R / 2; ++p) {
                const int r0 = 2 * p, r1 = r0 + 1;
                const float2 ec = make_float2(fminf(fmaxf(e, z[r0].lo), z[r0].hi), fminf(fmaxf(e, z[r1].lo), z[r1].hi));
                const float2 len = __fadd2_rn(ec, make_float2(-ep[r0], -ep[r1]));
                float2 a2 = __ffma2_rn(len, make_float2(v[r0], v[r1]), make_float2(acc[r0], acc[r1]));
                const float2 ze = __ffma2_rn(make_float2(kf[r0], kf[r1]), make_float2(z[r0].inva, z[r1].inva),
                                             make_float2(z[r0].c, z[r1].c));
                const float2 d = __fadd2_rn(ec, make_float2(-ze.x, -ze.y));
                const float2 w = make_float2(fmaxf(d.x, 0.0f), fmaxf(d.y, 0.0f));
                const float2 dv = __fadd2_rn(make_float2(vn[r0], vn[r1]), make_float2(-v[r0], -v[r1]));
                a2 = __ffma2_rn(w, dv, a2);
                acc[r0] = a2.x;
                acc[r1] = a2.y;
                const float2 t = __ffma2_rn(ec, make_float2(z[r0].a, z[r1].a), make_float2(z[r0].b, z[r1].b));
                const float2 kb = __fadd2_rn(t, make_float2(z[r0].m, z[r1].m));
                const float2 kn = __fadd2_rn(kb, make_float2(-z[r0].m, -z[r1].m));
                kbn[r0] = kb.x;
                kbn[r1] = kb.y;
                kf[r0] = kn.x;
                kf[r1] = kn.y;
                ep[r0] = ec.x;
                ep[r1] = ec.y;
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float ec = fminf(fmaxf(e, z[r].lo), z[r].hi);
                const float ze = __fmaf_rn(kf[r], z[r].inva, z[r].c);
                const float w = fmaxf(ec - ze, 0.0f);
                if (COMP) {
                    kahan(r, (ec - ep[r]) * v[r]);
                    kahan(r, w * (vn[r] - v[r]));
                } else {
                    acc[r] = __fmaf_rn(ec - ep[r], v[r], acc[r]);
                    acc[r] = __fmaf_rn(w, vn[r] - v[r], acc[r]);
                }
                const float kb = __fadd_rn(__fmaf_rn(ec, z[r].a, z[r].b), z[r].m);
                kf[r] = __fadd_rn(kb, -z[r].m);
                kbn[r] = kb;
                ep[r] = ec;
            }
        }
        bool done;
        if (e == ax.e) {
            ax.i += ax.s;
            done = (unsigned)ax.i >= (unsigned)nx;
            if (!done) {
                base += dcx;
                ax.r += (float)ax.s;
                ax.e = plane_alpha(ax.r, g.dx, rx);
            }
        } else {
            ay.i += ay.s;
            done = (unsigned)ay.i >= (unsigned)ny;
            if (!done) {
                base += dcy;
                ay.r += (float)ay.s;
                ay.e = plane_alpha(ay.r, g.dy, ry);
            }
        }
        if (done) break;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int idx = base + __float_as_int(kbn[r]);
            v[r] = ld(idx);
            vn[r] = ld(idx + z[r].soff);
        }
    }
}

// ------------------------------------------------------------- forward A x
//
// One tile = 8 warps = 8 adjacent detector columns (iu) x 32 R detector rows
// (iv) of one angle.  The volume is read in the padded z-fastest layout.
// Epilogue: proj = a * (A vol) + b * old (either projection layout), and one
// FP64 sums of squares of the stored values, one per warp, into
// partial_at()[warp] (when it returns non-null).  partial_at is called only in
// the epilogue, so that the address it computes is not held in a register
// through the traversal, and the sums need no block barrier (measured 6 %
// of the transpose's time with one).

constexpr int FWD_COLS = 8, FWD_THREADS = 32 * FWD_COLS;

template <typename T, bool COMP, int R, bool VFAST, typename PartialAt>
__device__ __forceinline__ void forward_tile(const DevGeom &g, const T *__restrict__ vol, T *__restrict__ proj,
                                             const Epilogue &epi, int tx, int ty, int a, PartialAt &&partial_at,
                                             double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int iu = tx * FWD_COLS + warp;
    const int iv0 = ty * 32 * R;
    const bool col_ok = iu < g.nu;            // uniform across the warp
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0f;
    if (col_ok) {
        RayAxis rx, ry, rz[R];
        load_rays<R>(g, a, iu, iv0, g.nv, rx, ry, rz);
        if (g.zsingle) {
            trace_rays_zsingle<T, COMP, R>(g, vol, rx, ry, rz, acc);
        } else {
            // several z crossings per xy cell are possible: the exact
            // crossing-by-crossing traversal
            float comp[R];
#pragma unroll
            for (int r = 0; r < R; ++r) comp[r] = 0.0f;
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
            trace_columns<R>(g, rx, ry, rz, 0, g.nx, 0, g.ny, 0, g.nz, (int)zf_col(g, 0, 0), g.nz + 2,
                             g.nx * (g.nz + 2), fetch, seg);
        }
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
    double *partial = partial_at();
    if (partial) warp_partial(sq, partial);
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
// plane_alpha filled at geometry creation.
// Projections are read v-fastest and pre-weighted by the ray length:
// w[a][iu][iv] = |d'| * y.

constexpr int BWD_THREADS = 256;

// Calls body(iu, ain, aout) for every detector column iu in [iu0, iu1], in
// increasing order, whose ray column crosses voxel column (i, j) of angle a:
// [ain, aout] is the alpha interval of the x/y cell (warp-uniform), from the
// same plane_alpha values either way.  LANES: the lanes clip up to 32 columns
// at once (lane l: column c0 + l), then the warp walks them, taking each
// column's interval from its lane; otherwise the warp clips column by column
// (fewer registers).  All lanes must call it.
template <bool LANES, int UNROLL, typename Body>
__device__ __forceinline__ void for_crossing_columns(const DevGeom &g, int a, int i, int j, int iu0, int iu1,
                                                     int lane, Body &&body) {
    auto clip = [&](int iu, float &ain, float &aout) {
        const float4 xy = __ldg(&g.ray_xy[(size_t)a * g.nu + iu]);
        const float2 q = __ldg(&g.ray_xyq[(size_t)a * g.nu + iu]);
        ain = -FLT_MAX;
        aout = FLT_MAX;
        bool miss = false;
        clip_slab(RayAxis{xy.x, xy.y, q.x}, g.dx, i, i + 1, ain, aout, miss);
        clip_slab(RayAxis{xy.z, xy.w, q.y}, g.dy, j, j + 1, ain, aout, miss);
        if (miss) {
            ain = FLT_MAX;                             // empty: no crossing
            aout = -FLT_MAX;
        }
    };
    if (LANES) {
        for (int c0 = iu0; c0 <= iu1; c0 += 32) {
            const int cn = min(32, iu1 - c0 + 1);
            float cin = FLT_MAX, cout = -FLT_MAX;
            if (lane < cn) clip(c0 + lane, cin, cout);
#pragma unroll UNROLL
            for (int c = 0; c < cn; ++c) {
                const float ain = __shfl_sync(0xffffffffu, cin, c), aout = __shfl_sync(0xffffffffu, cout, c);
                if (ain < aout) body(c0 + c, ain, aout);
            }
        }
    } else {
#pragma unroll UNROLL
        for (int iu = iu0; iu <= iu1; ++iu) {
            float ain, aout;
            clip(iu, ain, aout);
            if (ain < aout) body(iu, ain, aout);
        }
    }
}
constexpr int BWD_SHORT_ROWS = 3;

// Angles [a_begin, a_end) are summed in one call.  A scan whose projections
// do not fit in L2 is summed in passes over blocks of angles (launch_backward):
// `acc_in` (if not null) holds the FP32 sums of the earlier passes and
// `acc_out` (if not null) receives the running sums instead of the volume, so
// only the last pass applies the epilogue (with the FP64 sums of squares of
// the stored values into partial_at()[warp], when non-null, as in the
// forward tile).  Both are indexed
// ((j * nx + i) * nz + k) (unpadded); they may be the same buffer (each lane
// reads and writes only its own voxels).  ZFAST output goes to the padded
// z-fastest layout, else to the ABI layout x[k][j][i].
template <typename T, bool ZFAST, int CX, int K, bool HOIST, int IU_UNROLL = 0, typename PartialAt>
__device__ __forceinline__ void backward_tile(const DevGeom &g, const float *__restrict__ wproj, T *__restrict__ vol,
                                              const Epilogue &epi, int tx, int ty, int tz, int a_begin, int a_end,
                                              const float *acc_in, float *acc_out, PartialAt &&partial_at,
                                              double *red) {
    constexpr int CY = 8 / CX;
    // detector columns clipped by the lanes at once (tiles of up to 2 voxels
    // per lane; the 4-voxel tiles keep the per-column clip, which needs fewer
    // registers) and columns per unrolled step of the column loops
    constexpr bool BWD_LANE_CLIP = K <= 2;
    constexpr int BWD_IU_UNROLL = IU_UNROLL > 0 ? IU_UNROLL : !HOIST ? 1 : K == 1 ? 2 : K == 2 ? 1 : 2;
    // HOIST: the slab intervals of the candidate rows are loaded once per
    // angle and kept in registers (2 or 3 rows x 2 floats per voxel of the
    // lane); otherwise they are loaded for every detector column.
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
    if (col_ok && HOIST) {
        // The three candidate rows of each voxel start at its window's first
        // row moved down to fit the detector, and their slab intervals are
        // loaded once per angle (a row outside the window meets the voxel
        // nowhere and adds an exact zero).  The detector windows only select
        // candidates (every length is then computed exactly from the crossing
        // tables), so they use fast approximate divisions: their relative
        // error (~1e-6) stays far below the 0.05-pixel margins.
        const float inv_dv = 1.0f / g.dv, inv_du = 1.0f / g.du;
        const float cu = 0.5f * (g.nu - 1), cv = 0.5f * (g.nv - 1);
        float zlo[K], zhi[K];
        int zboff[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int k = k0 + kk * 32 + lane;
            zlo[kk] = (g.bz0 + k * g.dz) * inv_dv;
            zhi[kk] = (g.bz0 + (k + 1) * g.dz) * inv_dv;
            zboff[kk] = min(k, g.nz - 1) * g.nv;
        }
        const float x0 = g.bx0 + i * g.dx, x1 = x0 + g.dx;
        const float y0 = g.by0 + j * g.dy, y1 = y0 + g.dy;
        const size_t nuv = (size_t)g.nu * g.nv;
        for (int a = a_begin; a < a_end; ++a) {
            const float2 cs = __ldg(&g.trig[a]);
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
            // rows 2 / 3: every lane's window has at most 2 / 3 rows
            int wlo[K];
            bool rows2 = true, rows3 = true;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int k = k0 + kk * 32 + lane;
                const float vmin = fminf(zlo[kk] * magmin, zlo[kk] * magmax);
                const float vmax = fmaxf(zhi[kk] * magmin, zhi[kk] * magmax);
                const int lo = max(0, (int)ceilf(vmin + (cv - 0.05f)));
                const int hi = k < g.nz ? min(g.nv - 1, (int)floorf(vmax + (cv + 0.05f))) : -1;
                rows2 = rows2 && hi - lo < 2;
                rows3 = rows3 && hi - lo < 3;
                wlo[kk] = lo;
            }
            rows2 = __all_sync(0xffffffffu, rows2) && g.nv >= 2;
            rows3 = __all_sync(0xffffffffu, rows3) && g.nv >= 3;
            const float *pa = wproj + (size_t)a * nuv;
            // A fixed sequence of ROWS rows per voxel, starting at the window's
            // first row moved down to fit the detector; their slab intervals
            // are loaded once per angle.
            auto short_pass = [&](auto rows_c) {
                constexpr int ROWS = decltype(rows_c)::value;
                int r0[K];
                float2 zb[K][ROWS];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    r0[kk] = min(wlo[kk], g.nv - ROWS);
#pragma unroll
                    for (int t = 0; t < ROWS; ++t) zb[kk][t] = __ldg(&g.zbox[zboff[kk] + r0[kk] + t]);
                }
                // the column walk is unrolled by BWD_IU_UNROLL, so that the
                // next columns' loads are issued before this column's sums
                // (the per-column clip measured 7 % faster that way than the
                // compiler's choice, which kept the loop rolled; the lane
                // clip runs best rolled, at 3 CTAs per SM)
                for_crossing_columns<BWD_LANE_CLIP, BWD_IU_UNROLL>(g, a, i, j, iu0, iu1, lane, [&](int iu, float ain, float aout) {
                    const float *wcol = pa + (size_t)iu * g.nv;
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const float *wr = wcol + r0[kk];
#pragma unroll
                        for (int t = 0; t < ROWS; ++t) {
                            const float2 e = zb[kk][t];
                            const float lo = fmaxf(ain, e.x), hi = fminf(aout, e.y);
                            acc[kk] = __fmaf_rn(fmaxf(hi - lo, 0.0f), __ldg(wr + t), acc[kk]);
                        }
                    }
                });
            };
            if (rows2) {
                short_pass(std::integral_constant<int, 2>());
            } else if (rows3) {
                short_pass(std::integral_constant<int, 3>());
            } else {
                int rlo[K], rhi[K];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const int k = k0 + kk * 32 + lane;
                    const float vmin = fminf(zlo[kk] * magmin, zlo[kk] * magmax);
                    const float vmax = fmaxf(zhi[kk] * magmin, zhi[kk] * magmax);
                    rlo[kk] = max(0, (int)ceilf(vmin + (cv - 0.05f)));
                    rhi[kk] = k < g.nz ? min(g.nv - 1, (int)floorf(vmax + (cv + 0.05f))) : -1;
                }
                for_crossing_columns<BWD_LANE_CLIP, 1>(g, a, i, j, iu0, iu1, lane, [&](int iu, float ain, float aout) {
                    const float *wcol = pa + (size_t)iu * g.nv;
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        for (int iv = rlo[kk]; iv <= rhi[kk]; ++iv) {
                            const float2 e = __ldg(&g.zbox[zboff[kk] + iv]);
                            const float lo = fmaxf(ain, e.x), hi = fminf(aout, e.y);
                            acc[kk] = __fmaf_rn(fmaxf(hi - lo, 0.0f), __ldg(wcol + iv), acc[kk]);
                        }
                    }
                });
            }
        }
    }
    if (col_ok && !HOIST) {
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
            const float2 cs = __ldg(&g.trig[a]);
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
            // unrolled by BWD_IU_UNROLL, as the hoisted walk above
            for_crossing_columns<BWD_LANE_CLIP, BWD_IU_UNROLL>(g, a, i, j, iu0, iu1, lane, [&](int iu, float ain, float aout) {
                const float *wcol = pa + (size_t)iu * g.nv;
                if (short_rows) {
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const float2 *zb = g.zbox + (size_t)(k0 + kk * 32 + lane) * g.nv;
#pragma unroll
                        for (int t = 0; t < BWD_SHORT_ROWS; ++t) {
                            const int iv = r0[kk] + t;
                            if (iv <= r1[kk]) {
                                const float2 e = __ldg(zb + iv);
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
                            const float2 e = __ldg(zb + iv);        // row iv's alpha interval in slab k
                            const float lo = fmaxf(ain, e.x), hi = fminf(aout, e.y);
                            // a miss adds exactly zero: the same sum as skipping it
                            acc[kk] = __fmaf_rn(fmaxf(hi - lo, 0.0f), __ldg(wcol + iv), acc[kk]);
                        }
                    }
                }
            });
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
        const size_t v = ZFAST ? (size_t)(zf_col(g, i, j) + k) : ((size_t)k * g.ny + j) * g.nx + i;
        double out = acoef * (double)acc[kk];
        if (bcoef != 0.0) {
            const T *oldp = epi.old ? (const T *)epi.old : (const T *)vol;
            out += bcoef * (double)Storage<T>::ld_plain(oldp + v);
        }
        const float stored = Storage<T>::round((float)out);
        Storage<T>::store(vol + v, stored);
        sq += (double)stored * (double)stored;
    }
    double *partial = partial_at();
    if (partial) warp_partial(sq, partial);
}

}  // namespace cbct
