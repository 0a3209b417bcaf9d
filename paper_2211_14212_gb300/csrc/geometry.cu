// Geometry handle: validation, FP64 construction of the per-ray alpha tables,
// and the error plumbing shared by every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace cbct {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

cbct_status cuda_fail(cudaError_t err, const char *what) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s", (int)err, cudaGetErrorString(err), what);
    set_error(buf);
    (void)cudaGetLastError();   // clear a sticky launch error so the next call is not blamed
    return err == cudaErrorMemoryAllocation ? CBCT_ENOMEM : CBCT_ECUDA;
}

static cbct_status invalid(const char *msg) {
    set_error(msg);
    return CBCT_EINVAL;
}

cbct_status require_geometry_device(const cbct_geometry *g, const char *who) {
    int dev = -1;
    const cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, who);
    if (dev != g->device) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s: the geometry lives on CUDA device %d but the current device is %d", who,
                 g->device, dev);
        set_error(buf);
        return CBCT_EINVAL;
    }
    return CBCT_OK;
}

// Per-ray constants of one axis: the index pq of the plane nearest to the ray
// origin q, the offset f = plane(pq) - q (mm) and I = 1 / d (d = direction
// component along the axis).  Exactly parallel rays keep a fixed voxel index
// (half-open voxels: floor), stored in pq with I = 0.
static void axis_map(double q, double d, double b0, double delta, int n, float *f, float *I, float *pq) {
    if (d == 0.0) {
        *I = 0.0f;
        *f = 0.0f;
        double idx = std::floor((q - b0) / delta);
        if (idx < -1.0) idx = -1.0;
        if (idx > (double)n) idx = (double)n;
        *pq = (float)idx;
        return;
    }
    const double p = std::nearbyint((q - b0) / delta);
    *pq = (float)p;
    *f = (float)((b0 + p * delta) - q);
    *I = (float)(1.0 / d);
}

}  // namespace cbct

using namespace cbct;

extern "C" const char *cbct_last_error(void) { return g_last_error.c_str(); }

namespace cbct {

cbct_status validate_geometry_desc(const cbct_geometry_desc *d) {
    if (!d) return invalid("geometry: null description");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nu < 1 || d->nv < 1 || d->nangles < 1)
        return invalid("geometry: every count must be >= 1");
    if (!(d->dx > 0 && d->dy > 0 && d->dz > 0 && d->du > 0 && d->dv > 0))
        return invalid("geometry: voxel and pixel sizes must be > 0");
    if (!(d->dso > 0 && d->dsd > d->dso))
        return invalid("geometry: need 0 < dso < dsd");
    if (!d->angles_rad) return invalid("geometry: angles_rad is null");
    const double hx = 0.5 * d->nx * d->dx, hy = 0.5 * d->ny * d->dy;
    const double rcyl = std::sqrt(hx * hx + hy * hy);
    if (!(d->dso > rcyl) || !(d->dsd - d->dso > rcyl))
        return invalid("geometry: source and detector must lie outside the volume's circumscribed cylinder");
    // index ranges: voxels addressed with int32, rays with int64
    if ((int64_t)d->nx * d->ny * d->nz >= (int64_t)1 << 31)
        return invalid("geometry: more than 2^31-1 voxels");
    // the internal padded z-fastest layout (nz + 2 per column, 4 guards) is addressed with int32
    if ((int64_t)d->nx * d->ny * (d->nz + 2) + 4 >= (int64_t)1 << 31)
        return invalid("geometry: the padded volume layout needs more than 2^31-1 elements");
    if ((int64_t)d->nu * d->nv >= (int64_t)1 << 31)
        return invalid("geometry: more than 2^31-1 pixels per projection");
    if (d->nangles > 65535 || d->nv > 65535 * 4)
        return invalid("geometry: more than 65535 angles");
    for (int a = 0; a < d->nangles; ++a)
        if (!std::isfinite(d->angles_rad[a])) return invalid("geometry: non-finite angle");
    return CBCT_OK;
}

}  // namespace cbct

// Transpose passes: one by default.  Summing in passes over blocks of angles
// keeps each pass's projections in L2, but at 256^3 / 512^2 / 360 angles the
// gathers already hit L1/L2 (91 % L2 hits in one pass) and blocks of 12..120
// angles measured 0..4 % slower, so passes are left to the caller
// (cbct_geometry_set_angle_block).
namespace cbct {
int default_angle_block(const DevGeom &g) { return g.nangles; }
}  // namespace cbct

extern "C" cbct_status cbct_geometry_create(const cbct_geometry_desc *d, cbct_geometry **out) {
    if (!d || !out) return invalid("cbct_geometry_create: null argument");
    *out = nullptr;
    cbct_status vst = validate_geometry_desc(d);
    if (vst != CBCT_OK) return vst;

    const int nx = d->nx, ny = d->ny, nz = d->nz, nu = d->nu, nv = d->nv, na = d->nangles;
    const double dsd = d->dsd, m = d->dso / d->dsd;
    const double bx0 = -0.5 * nx * d->dx, by0 = -0.5 * ny * d->dy, bz0 = -0.5 * nz * d->dz;

    std::vector<float4> xy((size_t)na * nu);
    std::vector<float2> xyq((size_t)na * nu);
    std::vector<float4> zt(nv);
    std::vector<float> len((size_t)nv * nu);
    std::vector<float2> trig(na);
    for (int a = 0; a < na; ++a) {
        const double ct = std::cos(d->angles_rad[a]), st = std::sin(d->angles_rad[a]);
        trig[a] = make_float2((float)ct, (float)st);
        for (int iu = 0; iu < nu; ++iu) {
            const double u = (iu - 0.5 * (nu - 1)) * d->du;
            // rotated frame: source (dso, 0), pixel (dso - dsd, u); world = R(t) * frame
            const double dxw = -dsd * ct - u * st, dyw = -dsd * st + u * ct;
            const double qx = -u * m * st, qy = u * m * ct;
            float4 e;
            float2 q;
            axis_map(qx, dxw, bx0, d->dx, nx, &e.x, &e.y, &q.x);
            axis_map(qy, dyw, by0, d->dy, ny, &e.z, &e.w, &q.y);
            xy[(size_t)a * nu + iu] = e;
            xyq[(size_t)a * nu + iu] = q;
        }
    }
    for (int iv = 0; iv < nv; ++iv) {
        const double v = (iv - 0.5 * (nv - 1)) * d->dv;
        float4 e = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        axis_map(v * m, v, bz0, d->dz, nz, &e.x, &e.y, &e.z);
        zt[iv] = e;
        for (int iu = 0; iu < nu; ++iu) {
            const double u = (iu - 0.5 * (nu - 1)) * d->du;
            len[(size_t)iu * nv + iv] = (float)std::sqrt(dsd * dsd + u * u + v * v);
        }
    }

    cbct_geometry *g = new (std::nothrow) cbct_geometry();
    if (!g) { set_error("cbct_geometry_create: out of host memory"); return CBCT_ENOMEM; }
    g->angles = new (std::nothrow) double[na];
    if (!g->angles) { delete g; set_error("cbct_geometry_create: out of host memory"); return CBCT_ENOMEM; }
    std::memcpy(g->angles, d->angles_rad, sizeof(double) * na);
    g->desc = *d;
    g->desc.angles_rad = g->angles;

    auto align = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t s_xy = align(xy.size() * sizeof(float4)), s_q = align(xyq.size() * sizeof(float2));
    const size_t s_z = align(zt.size() * sizeof(float4));
    const size_t s_len = align(len.size() * sizeof(float)), s_tr = align(trig.size() * sizeof(float2));
    const size_t s_zb = align((size_t)nz * nv * sizeof(float2));
    const size_t o_q = s_xy, o_z = o_q + s_q, o_len = o_z + s_z, o_tr = o_len + s_len, o_zb = o_tr + s_tr;
    cudaError_t err = cudaGetDevice(&g->device);
    char *mem = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&mem, o_zb + s_zb);
    if (err == cudaSuccess) err = cudaMemcpy(mem, xy.data(), xy.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(mem + o_q, xyq.data(), xyq.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(mem + o_z, zt.data(), zt.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(mem + o_len, len.data(), len.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(mem + o_tr, trig.data(), trig.size() * sizeof(float2), cudaMemcpyHostToDevice);
    g->table_mem = mem;
    DevGeom &dg = g->dev;
    dg.nx = nx; dg.ny = ny; dg.nz = nz; dg.nu = nu; dg.nv = nv; dg.nangles = na;
    dg.dso = (float)d->dso; dg.dsd = (float)d->dsd; dg.du = (float)d->du; dg.dv = (float)d->dv;
    dg.bx0 = (float)bx0; dg.by0 = (float)by0; dg.bz0 = (float)bz0;
    dg.dx = (float)d->dx; dg.dy = (float)d->dy; dg.dz = (float)d->dz;
    dg.ray_xy = reinterpret_cast<const float4 *>(mem);
    dg.ray_xyq = reinterpret_cast<const float2 *>(mem + o_q);
    dg.ray_z = reinterpret_cast<const float4 *>(mem + o_z);
    dg.ray_len = reinterpret_cast<const float *>(mem + o_len);
    dg.trig = reinterpret_cast<const float2 *>(mem + o_tr);
    dg.zbox = reinterpret_cast<const float2 *>(mem + o_zb);
    // the z slab crossings are computed on the device by the projectors' own
    // plane_alpha (the same two roundings as every x/y crossing)
    if (err == cudaSuccess) err = launch_zbox(dg, reinterpret_cast<float2 *>(mem + o_zb));
    if (err == cudaSuccess) err = cudaStreamSynchronize(0);
    if (err != cudaSuccess) {
        if (mem) cudaFree(mem);
        delete[] g->angles;
        delete g;
        return cuda_fail(err, "cbct_geometry_create");
    }
    dg.fwd_rows = nv >= 128 ? 4 : nv >= 64 ? 2 : 1;   // forward tile: rows per lane by detector height
    // At most one z-plane crossing per x/y voxel column along every ray: a
    // ray's x/y path inside one column is at most the column's diagonal, and
    // its z slope is at most max|v| / DSD (the pixel farthest from the
    // mid-plane, seen from the source).  The forward projector's fast
    // traversal relies on it (2 % margin for rounding).
    {
        const double vmax = 0.5 * (nv - 1) * d->dv;
        const double zrise = std::sqrt(d->dx * d->dx + d->dy * d->dy) * vmax / d->dsd;
        dg.zsingle = zrise < 0.98 * d->dz ? 1 : 0;
    }
    dg.bwd_config = nz >= 64 ? 3 : 0;   // 2 / 1 voxels per lane by column depth
    dg.angle_block = default_angle_block(dg);
    *out = g;
    return CBCT_OK;
}

extern "C" void cbct_geometry_destroy(cbct_geometry *g) {
    if (!g) return;
    if (g->table_mem) cudaFree(g->table_mem);
    delete[] g->angles;
    delete g;
}

extern "C" int cbct_geometry_device(const cbct_geometry *g) { return g ? g->device : -1; }

extern "C" int64_t cbct_geometry_num_voxels(const cbct_geometry *g) {
    return g ? (int64_t)g->dev.nx * g->dev.ny * g->dev.nz : -1;
}

extern "C" int64_t cbct_geometry_num_rays(const cbct_geometry *g) {
    return g ? (int64_t)g->dev.nangles * g->dev.nv * g->dev.nu : -1;
}
