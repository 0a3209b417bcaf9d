/*
 * Oracle: FP64 cone-beam system matrix A and its transpose, computed on the CPU
 * straight from the definition.  TEST INFRASTRUCTURE ONLY: it is built and run
 * by the tests, by the CPU baseline of the benchmark and by the smoke check,
 * never by the library's product path.  It shares no code with the GPU path.
 *
 * Definition (Sec. 1, Eq. 1; Sec. 2, Eq. 2): A in R^{N x M}, N = detector
 * pixels x projection angles, M = voxels.  Entry A[i][j] = l_ij is the length
 * of ray i (the segment from the source to the centre of pixel i) inside voxel
 * j, a half-open box.  The paper leaves the projector to its toolbox; the
 * entries here are that length, which a Siddon ray tracer reaches exactly.
 *
 * Geometry conventions (the paper is silent; these are the repository's):
 *   source          s = (dso cos t, dso sin t, 0)
 *   detector centre c = -(dsd - dso) (cos t, sin t, 0)
 *   detector axes   e_u = (-sin t, cos t, 0), e_v = (0, 0, 1)
 *   pixel centre    c + (iu - (nu-1)/2) du e_u + (iv - (nv-1)/2) dv e_v
 *   voxel (i,j,k)   [x0 + i dx, x0 + (i+1) dx) x ..., x0 = -nx dx / 2
 *   storage         x[k][j][i], y[a][iv][iu]; ray index (a*nv + iv)*nu + iu
 *
 * Ray segments (merged-alpha form): parametrise the ray as s + a (p - s),
 * a in [0, 1]; clip to the volume box by the slab method; collect every plane
 * crossing strictly inside the clipped interval; sort; each consecutive pair
 * (a_m, a_m+1) with a_m+1 > a_m is one segment of length (a_m+1 - a_m) |p - s|.
 * Its voxel is the one the ray is in after the crossings it has passed: on an
 * axis the ray crosses, the index follows from how many of that axis' plane
 * crossings lie at or before the segment's midpoint (Siddon's index rule; the
 * same voxel as the one containing the midpoint, but decided by comparing
 * crossing parameters, so it stays exact for rays lying within rounding
 * distance of a plane); on an axis the ray runs parallel to, the index is that
 * of its fixed coordinate in the half-open voxels.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int nu, nv;
    double du, dv;
    double dso, dsd;
    int nangles;
    const double *angles;
} og_geom;

static void ray_endpoints(const og_geom *g, int64_t ray, double s[3], double p[3])
{
    int64_t per_angle = (int64_t)g->nu * g->nv;
    int a = (int)(ray / per_angle);
    int64_t rem = ray % per_angle;
    int iv = (int)(rem / g->nu);
    int iu = (int)(rem % g->nu);
    double t = g->angles[a];
    double ct = cos(t), st = sin(t);
    double u = (iu - 0.5 * (g->nu - 1)) * g->du;
    double v = (iv - 0.5 * (g->nv - 1)) * g->dv;
    s[0] = g->dso * ct;
    s[1] = g->dso * st;
    s[2] = 0.0;
    p[0] = -(g->dsd - g->dso) * ct - u * st;
    p[1] = -(g->dsd - g->dso) * st + u * ct;
    p[2] = v;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Capacity needed for the alpha list of one ray, plus the three per-axis crossing lists. */
static int64_t alpha_capacity(const og_geom *g)
{
    return 2 * ((int64_t)g->nx + g->ny + g->nz + 3) + 2;
}

/* Number of entries of the monotone list a[0..n) that are <= x (increasing or decreasing list). */
static int count_le(const double *a, int n, int increasing, double x)
{
    int lo = 0, hi = n;              /* binary search for the boundary */
    if (increasing) {                /* entries <= x form a prefix */
        while (lo < hi) { int mid = (lo + hi) / 2; if (a[mid] <= x) lo = mid + 1; else hi = mid; }
        return lo;
    }
    while (lo < hi) { int mid = (lo + hi) / 2; if (a[mid] <= x) hi = mid; else lo = mid + 1; }
    return n - lo;                   /* entries <= x form a suffix */
}

/*
 * Segments of one ray: writes voxel indices (k*ny + j)*nx + i and lengths of
 * every positive-length piece, in order from the source.  `alpha` is scratch of
 * alpha_capacity() doubles.  Returns the number of segments.
 */
static int ray_segments(const og_geom *g, int64_t ray, int64_t *idx, double *len, double *alpha)
{
    double s[3], p[3], d[3];
    ray_endpoints(g, ray, s, p);
    const int n[3] = {g->nx, g->ny, g->nz};
    const double del[3] = {g->dx, g->dy, g->dz};
    double b0[3];
    for (int c = 0; c < 3; ++c) {
        d[c] = p[c] - s[c];
        b0[c] = -0.5 * n[c] * del[c];
    }
    double length = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);

    /* slab method on the whole volume box, restricted to the segment [0, 1] */
    double lo = 0.0, hi = 1.0;
    for (int c = 0; c < 3; ++c) {
        double b1 = b0[c] + n[c] * del[c];
        if (d[c] != 0.0) {
            double a0 = (b0[c] - s[c]) / d[c];
            double a1 = (b1 - s[c]) / d[c];
            if (a0 > a1) { double tmp = a0; a0 = a1; a1 = tmp; }
            if (a0 > lo) lo = a0;
            if (a1 < hi) hi = a1;
        } else if (!(s[c] >= b0[c] && s[c] < b1)) {
            return 0;               /* parallel to this slab and outside it */
        }
    }
    if (!(lo < hi)) return 0;

    /* crossing parameter of every plane of every axis the ray is not parallel to */
    double *cross[3];
    double *tail = alpha + (g->nx + g->ny + g->nz + 3) + 2;
    for (int c = 0; c < 3; ++c) {
        cross[c] = tail;
        if (d[c] != 0.0) {
            for (int q = 0; q <= n[c]; ++q) cross[c][q] = (b0[c] + q * del[c] - s[c]) / d[c];
            tail += n[c] + 1;
        }
    }

    int m = 0;
    alpha[m++] = lo;
    alpha[m++] = hi;
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.0) continue;
        for (int q = 0; q <= n[c]; ++q) {
            double a = cross[c][q];
            if (a > lo && a < hi) alpha[m++] = a;
        }
    }
    qsort(alpha, (size_t)m, sizeof(double), cmp_double);

    int count = 0;
    for (int q = 0; q + 1 < m; ++q) {
        double a0 = alpha[q], a1 = alpha[q + 1];
        if (!(a1 > a0)) continue;
        double mid = 0.5 * (a0 + a1);
        int64_t ijk[3];
        int inside = 1;
        for (int c = 0; c < 3; ++c) {
            if (d[c] != 0.0) {
                /* planes crossed so far: increasing coordinate -> voxel (crossed - 1),
                   decreasing coordinate -> voxel n - crossed */
                int crossed = count_le(cross[c], n[c] + 1, d[c] > 0.0, mid);
                ijk[c] = d[c] > 0.0 ? crossed - 1 : n[c] - crossed;
            } else {
                ijk[c] = (int64_t)floor((s[c] - b0[c]) / del[c]);
            }
            if (ijk[c] < 0 || ijk[c] >= n[c]) inside = 0;
        }
        if (!inside) continue;
        idx[count] = (ijk[2] * n[1] + ijk[1]) * n[0] + ijk[0];
        len[count] = (a1 - a0) * length;
        ++count;
    }
    return count;
}

int64_t oracle_num_rays(const og_geom *g)
{
    return (int64_t)g->nangles * g->nv * g->nu;
}

int64_t oracle_max_segments(const og_geom *g)
{
    return alpha_capacity(g);
}

/* Segment list of one ray (for tests).  Returns the count, or -1 if cap is too small. */
int oracle_ray_segments(const og_geom *g, int64_t ray, int64_t *idx, double *len, int cap)
{
    int64_t need = alpha_capacity(g);
    if (cap < need) return -1;
    double *alpha = (double *)malloc(sizeof(double) * need);
    int c = ray_segments(g, ray, idx, len, alpha);
    free(alpha);
    return c;
}

/* y[r] = sum_j l_rj x[j] for the listed rays (all rays when rays == NULL). */
void oracle_project_rays(const og_geom *g, const double *x, const int64_t *rays, int64_t count,
                         double *y, int nthreads)
{
    int64_t cap = alpha_capacity(g);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *alpha = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            int64_t r = rays ? rays[q] : q;
            int c = ray_segments(g, r, idx, len, alpha);
            double acc = 0.0;
            for (int m = 0; m < c; ++m) acc += len[m] * x[idx[m]];
            y[q] = acc;
        }
        free(idx);
        free(len);
        free(alpha);
    }
}

/* y = A x over all rays. */
void oracle_project(const og_geom *g, const double *x, double *y, int nthreads)
{
    oracle_project_rays(g, x, NULL, oracle_num_rays(g), y, nthreads);
}

/* Scatter x[j] += l_ij y[i] for rays [r0, r1) in order. */
static void scatter_rays(const og_geom *g, const double *y, int64_t r0, int64_t r1, double *x)
{
    int64_t cap = alpha_capacity(g);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * cap);
    double *len = (double *)malloc(sizeof(double) * cap);
    double *alpha = (double *)malloc(sizeof(double) * cap);
    for (int64_t r = r0; r < r1; ++r) {
        if (y[r] == 0.0) continue;
        int c = ray_segments(g, r, idx, len, alpha);
        for (int m = 0; m < c; ++m) x[idx[m]] += len[m] * y[r];
    }
    free(idx);
    free(len);
    free(alpha);
}

/*
 * x = A^T y as an explicit scatter x[j] += l_ij y[i].  nthreads <= 1: one
 * sequential pass over the rays in order.  nthreads > 1: the rays are cut
 * into nthreads contiguous chunks, each scattered into its own zeroed volume,
 * and the volumes are added in chunk order (the same sum, regrouped).
 */
void oracle_backproject(const og_geom *g, const double *y, double *x, int nthreads)
{
    int64_t nvox = (int64_t)g->nx * g->ny * g->nz;
    int64_t nr = oracle_num_rays(g);
    memset(x, 0, sizeof(double) * nvox);
    if (nthreads <= 1) {
        scatter_rays(g, y, 0, nr, x);
        return;
    }
    double *part = (double *)calloc((size_t)nthreads * nvox, sizeof(double));
#ifdef _OPENMP
    omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(static, 1)
    for (int t = 0; t < nthreads; ++t) {
        int64_t r0 = nr * t / nthreads, r1 = nr * (t + 1) / nthreads;
        scatter_rays(g, y, r0, r1, part + (size_t)t * nvox);
    }
    for (int t = 0; t < nthreads; ++t) {
        const double *pt = part + (size_t)t * nvox;
        for (int64_t j = 0; j < nvox; ++j) x[j] += pt[j];
    }
    free(part);
}

/* Number of nonzero entries of A (positive-length ray/voxel pairs). */
int64_t oracle_nnz(const og_geom *g, int nthreads)
{
    int64_t cap = alpha_capacity(g);
    int64_t nr = oracle_num_rays(g);
    int64_t total = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : total)
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *alpha = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 256)
        for (int64_t r = 0; r < nr; ++r) total += ray_segments(g, r, idx, len, alpha);
        free(idx);
        free(len);
        free(alpha);
    }
    return total;
}

/*
 * Length of ray r inside voxel (i, j, k), straight from the definition: clip the
 * segment source -> pixel against the voxel's half-open box by the slab method.
 */
static double ray_voxel_length(const og_geom *g, int64_t r, int i, int j, int k)
{
    double s[3], p[3], d[3];
    ray_endpoints(g, r, s, p);
    const double del[3] = {g->dx, g->dy, g->dz};
    const int n[3] = {g->nx, g->ny, g->nz};
    const int ijk[3] = {i, j, k};
    double lo = 0.0, hi = 1.0;
    for (int c = 0; c < 3; ++c) {
        d[c] = p[c] - s[c];
        double b0 = -0.5 * n[c] * del[c];
        /* the voxel's two planes, written exactly as the ray-driven route writes them */
        double v0 = b0 + ijk[c] * del[c];
        double v1 = b0 + (ijk[c] + 1) * del[c];
        if (d[c] != 0.0) {
            double a0 = (v0 - s[c]) / d[c], a1 = (v1 - s[c]) / d[c];
            if (a0 > a1) { double tmp = a0; a0 = a1; a1 = tmp; }
            if (a0 > lo) lo = a0;
            if (a1 < hi) hi = a1;
        } else if ((int64_t)floor((s[c] - b0) / del[c]) != ijk[c]) {
            return 0.0;             /* in-plane ray: half-open rule by the same index map */
        }
    }
    if (!(lo < hi)) return 0.0;
    return (hi - lo) * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/*
 * (A^T y)_j for the listed voxels, one by one: for every angle, every pixel
 * whose ray can meet voxel j (a window found by projecting the voxel's eight
 * corners onto the detector, widened by two pixels) contributes l_ij y_i.
 */
void oracle_backproject_voxels(const og_geom *g, const double *y, const int64_t *voxels,
                               int64_t count, double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < count; ++q) {
        int64_t vj = voxels[q];
        int i = (int)(vj % g->nx);
        int j = (int)((vj / g->nx) % g->ny);
        int k = (int)(vj / ((int64_t)g->nx * g->ny));
        double acc = 0.0;
        for (int a = 0; a < g->nangles; ++a) {
            double t = g->angles[a], ct = cos(t), st = sin(t);
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            for (int corner = 0; corner < 8; ++corner) {
                double px = -0.5 * g->nx * g->dx + (i + (corner & 1)) * g->dx;
                double py = -0.5 * g->ny * g->dy + (j + ((corner >> 1) & 1)) * g->dy;
                double pz = -0.5 * g->nz * g->dz + (k + ((corner >> 2) & 1)) * g->dz;
                /* distance from the source along the central ray, and transverse offsets */
                double along = g->dso - (px * ct + py * st);
                double across = -px * st + py * ct;
                double mag = g->dsd / along;
                double u = across * mag, v = pz * mag;
                if (u < umin) umin = u;
                if (u > umax) umax = u;
                if (v < vmin) vmin = v;
                if (v > vmax) vmax = v;
            }
            int iu0 = (int)floor(umin / g->du + 0.5 * (g->nu - 1)) - 2;
            int iu1 = (int)ceil(umax / g->du + 0.5 * (g->nu - 1)) + 2;
            int iv0 = (int)floor(vmin / g->dv + 0.5 * (g->nv - 1)) - 2;
            int iv1 = (int)ceil(vmax / g->dv + 0.5 * (g->nv - 1)) + 2;
            if (iu0 < 0) iu0 = 0;
            if (iv0 < 0) iv0 = 0;
            if (iu1 > g->nu - 1) iu1 = g->nu - 1;
            if (iv1 > g->nv - 1) iv1 = g->nv - 1;
            for (int iv = iv0; iv <= iv1; ++iv)
                for (int iu = iu0; iu <= iu1; ++iu) {
                    int64_t r = ((int64_t)a * g->nv + iv) * g->nu + iu;
                    double l = ray_voxel_length(g, r, i, j, k);
                    if (l > 0.0) acc += l * y[r];
                }
        }
        out[q] = acc;
    }
}
