/*
 * Seeded synthetic scenes for the RBSM path: shadow maps rasterised from
 * analytic occluders and light-space fragment coordinates from a camera
 * homography.  This is input generation only: it performs no shadow test and
 * no step of the revectorisation method, and both the CUDA path and the CPU
 * oracle consume its output.
 *
 * Depth convention: an orthographic light looks down the depth axis; the
 * ground plane sits at depth 1; an occluder of height h above the ground has
 * depth 1 - h.  A texel stores the smallest depth of any surface covering its
 * centre (the light pass of shadow mapping, point-sampled).
 *
 * The loops use IEEE double arithmetic with contraction off and no libm
 * call but sqrt, so given the same parameters every host writes the same
 * bytes; the parameters themselves are drawn by the Python front end.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define BAND 32

/* Fill a map with the ground depth. */
void sg_fill(float *depth, int32_t width, int32_t height, int64_t pitch, float value)
{
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < height; ++j) {
        float *row = depth + j * pitch;
        for (int64_t i = 0; i < width; ++i)
            row[i] = value;
    }
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* Oriented rectangles.  rect[k] = (cx, cy, ux, uy, ha, hb) in texel units:
 * centre, unit axis, half length along the axis and half width across it.
 * A texel centre (i + 0.5, j + 0.5) is covered when both projections lie
 * within the half extents.  dep[k] is the occluder's depth. */
void sg_raster_rects(float *depth, int32_t width, int32_t height, int64_t pitch,
                     int32_t n, const double *rect, const float *dep)
{
    int32_t nband = (height + BAND - 1) / BAND;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t band = 0; band < nband; ++band) {
        int64_t j_lo = (int64_t)band * BAND;
        int64_t j_hi = j_lo + BAND < height ? j_lo + BAND : height;
        for (int32_t k = 0; k < n; ++k) {
            const double *r = rect + 6 * k;
            double cx = r[0], cy = r[1], ux = r[2], uy = r[3], ha = r[4], hb = r[5];
            double ey = fabs(uy) * ha + fabs(ux) * hb;   /* half height of the bounding box */
            int64_t jb0 = (int64_t)floor(cy - ey - 1.0), jb1 = (int64_t)ceil(cy + ey + 1.0);
            if (jb0 < j_lo) jb0 = j_lo;
            if (jb1 > j_hi) jb1 = j_hi;
            for (int64_t j = jb0; j < jb1; ++j) {
                double py = (double)j + 0.5 - cy;
                /* span of x where |a*px + b*py| <= h for both axes */
                double lo = -1e300, hi = 1e300;
                double ax[2] = {ux, -uy}, bx[2] = {uy, ux}, hx[2] = {ha, hb};
                int empty = 0;
                for (int q = 0; q < 2; ++q) {
                    double a = ax[q], b = bx[q], h = hx[q];
                    if (fabs(a) < 1e-12) {
                        if (fabs(b * py) > h) empty = 1;
                        continue;
                    }
                    double t0 = (-h - b * py) / a, t1 = (h - b * py) / a;
                    lo = dmax(lo, dmin(t0, t1));
                    hi = dmin(hi, dmax(t0, t1));
                }
                if (empty || lo > hi)
                    continue;
                int64_t i0 = (int64_t)floor(cx + lo - 1.5), i1 = (int64_t)ceil(cx + hi + 0.5);
                if (i0 < 0) i0 = 0;
                if (i1 > width) i1 = width;
                float *row = depth + j * pitch;
                for (int64_t i = i0; i < i1; ++i) {
                    double px = (double)i + 0.5 - cx;
                    double s = px * ux + py * uy, t = -px * uy + py * ux;
                    if (fabs(s) <= ha && fabs(t) <= hb && dep[k] < row[i])
                        row[i] = dep[k];
                }
            }
        }
    }
}

/* Spheres.  sph[k] = (cx, cy, R, centre depth) in texel units; the surface
 * facing the light has depth  centre - sqrt(R^2 - rho^2) / zscale. */
static double sphere_depth(const double *s, double px, double py, double zscale, int *inside)
{
    double dx = px - s[0], dy = py - s[1];
    double rho2 = dx * dx + dy * dy, r2 = s[2] * s[2];
    if (rho2 > r2) {
        *inside = 0;
        return 0.0;
    }
    *inside = 1;
    return s[3] - sqrt(r2 - rho2) / zscale;
}

void sg_raster_spheres(float *depth, int32_t width, int32_t height, int64_t pitch,
                       int32_t n, const double *sph, double zscale)
{
    int32_t nband = (height + BAND - 1) / BAND;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t band = 0; band < nband; ++band) {
        int64_t j_lo = (int64_t)band * BAND;
        int64_t j_hi = j_lo + BAND < height ? j_lo + BAND : height;
        for (int32_t k = 0; k < n; ++k) {
            const double *s = sph + 4 * k;
            int64_t jb0 = (int64_t)floor(s[1] - s[2] - 1.0), jb1 = (int64_t)ceil(s[1] + s[2] + 1.0);
            if (jb0 < j_lo) jb0 = j_lo;
            if (jb1 > j_hi) jb1 = j_hi;
            int64_t i0 = (int64_t)floor(s[0] - s[2] - 1.0), i1 = (int64_t)ceil(s[0] + s[2] + 1.0);
            if (i0 < 0) i0 = 0;
            if (i1 > width) i1 = width;
            for (int64_t j = jb0; j < jb1; ++j) {
                float *row = depth + j * pitch;
                for (int64_t i = i0; i < i1; ++i) {
                    int in;
                    double d = sphere_depth(s, (double)i + 0.5, (double)j + 0.5, zscale, &in);
                    float df = (float)d;
                    if (in && df < row[i])
                        row[i] = df;
                }
            }
        }
    }
}

/* Cell range of sphere k in a uniform grid of `cell`-texel cells. */
static void sphere_cells(const double *s, int32_t cell, int32_t gw, int32_t gh,
                         int64_t *c0, int64_t *c1, int64_t *r0, int64_t *r1)
{
    *c0 = (int64_t)floor((s[0] - s[2]) / cell);
    *c1 = (int64_t)floor((s[0] + s[2]) / cell);
    *r0 = (int64_t)floor((s[1] - s[2]) / cell);
    *r1 = (int64_t)floor((s[1] + s[2]) / cell);
    if (*c0 < 0) *c0 = 0;
    if (*r0 < 0) *r0 = 0;
    if (*c1 > gw - 1) *c1 = gw - 1;
    if (*r1 > gh - 1) *r1 = gh - 1;
}

/* Fragments of one view.  Pixel (px, py) of a sw x sh screen maps through the
 * homography hom (row-major 3x3, screen pixel centre -> texel-space point) to
 * light texel coordinates (X, Y); x = X / width, y = Y / height.  The
 * receiver is the nearest-to-the-light of the receiver spheres covering
 * (X, Y), raised by `offset` towards the light, else the ground plane at
 * plane_z.  Spheres are looked up through a uniform grid of 64-texel cells.
 * out_kind (nullable) receives 0 for plane, 1 + sphere index otherwise.
 * Returns 0, or -1 when memory for the lookup grid is not available. */
int32_t sg_fragments(int32_t sw, int32_t sh, const double *hom,
                     int32_t width, int32_t height,
                     int32_t n_sph, const double *sph, double zscale, double offset, float plane_z,
                     float *x, float *y, float *z, int32_t *out_kind)
{
    const int32_t cell = 64;
    int32_t gw = (width + cell - 1) / cell, gh = (height + cell - 1) / cell;
    int64_t ng = (int64_t)gw * gh;
    int32_t *count = (int32_t *)calloc((size_t)ng, sizeof(int32_t));
    int32_t *start = (int32_t *)calloc((size_t)ng + 1, sizeof(int32_t));
    int32_t *fill = (int32_t *)calloc((size_t)ng, sizeof(int32_t));
    if (!count || !start || !fill) {
        free(count); free(start); free(fill);
        return -1;
    }
    int64_t c0, c1, r0, r1;
    for (int32_t k = 0; k < n_sph; ++k) {
        sphere_cells(sph + 4 * k, cell, gw, gh, &c0, &c1, &r0, &r1);
        for (int64_t r = r0; r <= r1; ++r)
            for (int64_t c = c0; c <= c1; ++c)
                count[r * gw + c] += 1;
    }
    for (int64_t g = 0; g < ng; ++g)
        start[g + 1] = start[g] + count[g];
    int32_t *list = (int32_t *)malloc((size_t)(start[ng] > 0 ? start[ng] : 1) * sizeof(int32_t));
    if (!list) {
        free(count); free(start); free(fill);
        return -1;
    }
    for (int32_t k = 0; k < n_sph; ++k) {
        sphere_cells(sph + 4 * k, cell, gw, gh, &c0, &c1, &r0, &r1);
        for (int64_t r = r0; r <= r1; ++r)
            for (int64_t c = c0; c <= c1; ++c) {
                int64_t g = r * gw + c;
                list[start[g] + fill[g]] = k;
                fill[g] += 1;
            }
    }

    #pragma omp parallel for schedule(static)
    for (int64_t py = 0; py < sh; ++py) {
        for (int64_t px = 0; px < sw; ++px) {
            double u = (double)px + 0.5, v = (double)py + 0.5;
            double w = hom[6] * u + hom[7] * v + hom[8];
            double X = (hom[0] * u + hom[1] * v + hom[2]) / w;
            double Y = (hom[3] * u + hom[4] * v + hom[5]) / w;
            double best = 1e300;
            int32_t kind = 0;
            int64_t c = (int64_t)floor(X / cell), r = (int64_t)floor(Y / cell);
            if (c >= 0 && r >= 0 && c < gw && r < gh) {
                int64_t g = r * gw + c;
                for (int32_t q = start[g]; q < start[g + 1]; ++q) {
                    int32_t k = list[q];
                    int in;
                    double d = sphere_depth(sph + 4 * k, X, Y, zscale, &in);
                    if (in && d < best) {
                        best = d;
                        kind = 1 + k;
                    }
                }
            }
            int64_t t = py * sw + px;
            x[t] = (float)(X / (double)width);
            y[t] = (float)(Y / (double)height);
            z[t] = kind ? (float)(best - offset) : plane_z;
            if (out_kind)
                out_kind[t] = kind;
        }
    }
    free(count);
    free(start);
    free(list);
    free(fill);
    return 0;
}

/* Number of threads the OpenMP runtime would use (1 without OpenMP). */
int32_t sg_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
