/*
 * Plain CPU oracle of the per-fragment revectorization-based shadow mapping
 * (RBSM) path with the optimized visibility functions of Macedo, Apolinario
 * and Aguero, "Optimized Visibility Functions for Revectorization-Based
 * Shadow Mapping" (TR-PGCOMP-007/2017).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or helper with the
 * CUDA library, and it never reads a value the CUDA library produced.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no fast-math).  Contraction
 * must stay off so that the single-precision silhouette decision below is the
 * plain IEEE sequence of operations on every host (aarch64 GCC contracts
 * a*b+c into FMA by default).
 *
 * Conventions (the paper's statement of the problem, Listing 1 / §3):
 *   - the shadow map SM is a width x height array of depths, row-major, row j
 *     at texture coordinate y in [j/height, (j+1)/height);
 *   - a fragment p = (x, y, z): x, y texture coordinates in [0,1), z its depth
 *     as seen from the light;
 *   - visibility 1 = lit, 0 = shadow (Eq. 1).
 *
 * Readings of points the paper leaves open (each is repeated where it acts):
 *   R1  nearest-texel addressing: i = floor(x*W) with x*W formed in single
 *       precision (the paper's GLSL float); neighbours are integer i+-1, j+-1.
 *   R2  texels outside the map are clamped to the edge.
 *   R3  no depth bias: Eq. 1 exactly (strict '>').
 *   R4  neighbour order (left, right, +y, -y) as in Listing 2; +y is the
 *       neighbour at the next row index.
 *   R5  checkDiscontinuity (used in Listing 3, never printed): the neighbour's
 *       own four-neighbourhood discontinuity, evaluated with the fragment's
 *       depth, shares at least one direction with the fragment's (§3.1.3).
 *   R6  computeFragmentDistanceToSE (Listing 1, never printed): one traversal
 *       per direction, in the order -x, +x, -y, +y (§3.1.3).
 *   R7  normalizeFragmentDistanceToSE (Listing 1, never printed): per axis the
 *       fragment's distance to the end that was found, over the length of the
 *       aliased edge along that axis (§3.1.4, Fig. 3(c), Eq. 5).
 *   R8  the end counts of Eq. 5 are raw on both sides of the edge.
 *   R9  the traversal visits k = 1..MAXDIST texels (Listing 3 loop bound).
 *   R11 the I-shape test of Listing 5 reads "nrd.w == -1" on its second term
 *       (the printed "nrd.w == 1" cannot be reached after the U-shape tests).
 *   R13 a traversal that runs out of steps found no end; its distance is
 *       -(MAXDIST + 1).
 *   R15 the equality tests on d and nrd compare exact codes.
 *   R17 a fragment outside [0,1) is clamped to the edge texel; its in-texel
 *       offset is still frac(x*W).  The clamp is taken on the float texel
 *       coordinate, so a NaN coordinate maps to texel 0.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

#define ORACLE_MODE_SILHOUETTE 1
#define ORACLE_MODE_FILTER     2

typedef struct {
    const float *depth;
    int32_t width, height;
    int64_t pitch;
} sm_t;

/* R2: clamp-to-edge fetch of the depth stored in texel (i, j). */
static float sm_depth(const sm_t *sm, int64_t i, int64_t j)
{
    if (i < 0) i = 0;
    if (i > sm->width - 1) i = sm->width - 1;
    if (j < 0) j = 0;
    if (j > sm->height - 1) j = sm->height - 1;
    return sm->depth[j * sm->pitch + i];
}

/* Eq. 1 (§3.1.2): s = 0 when the stored blocker is closer to the light than
 * the fragment (p_z > z(t)), 1 otherwise.  R3: no bias. */
static int shadow_test(float pz, float zt)
{
    if (pz > zt)
        return 0;
    return 1;
}

static int shadow_test_at(const sm_t *sm, int64_t i, int64_t j, float pz)
{
    return shadow_test(pz, sm_depth(sm, i, j));
}

/* Eqs. 2-3 and Listing 2: shadow tests of the four neighbours with the
 * fragment's depth (R4 order: left, right, +y, -y) and the discontinuity
 * d_k = |N_k - s|.  Returns s at (i, j); dirs[k] receives d_k. */
static int discontinuity4(const sm_t *sm, int64_t i, int64_t j, float pz, int dirs[4])
{
    int s = shadow_test_at(sm, i, j, pz);
    int nb[4];
    nb[0] = shadow_test_at(sm, i - 1, j, pz);
    nb[1] = shadow_test_at(sm, i + 1, j, pz);
    nb[2] = shadow_test_at(sm, i, j + 1, pz);
    nb[3] = shadow_test_at(sm, i, j - 1, pz);
    for (int k = 0; k < 4; ++k)
        dirs[k] = nb[k] > s ? nb[k] - s : s - nb[k];
    return s;
}

/* Listing 3, §3.1.3 and §3.2.3: walk from texel (i, j) one texel at a time in
 * direction (di, dj).  The walk ends with +k when the k-th texel has the other
 * shadow-test result (an end of the shadow edge), with -k when the k-th texel
 * has the same result but shares no discontinuity direction with the fragment
 * (R5: it is not part of the same edge), and with -(max_dist + 1) when all
 * max_dist texels continued (R9, R13). */
static int traverse_edge(const sm_t *sm, int64_t i, int64_t j, float pz, int s0,
                         const int dirs0[4], int di, int dj, int max_dist)
{
    int64_t ni = i, nj = j;
    int dist = 1;
    int found_end = 0;
    for (int step = 0; step < max_dist; ++step) {
        ni += di;
        nj += dj;
        if (shadow_test_at(sm, ni, nj, pz) != s0) {
            found_end = 1;
            break;
        }
        int dirs_n[4];
        (void)discontinuity4(sm, ni, nj, pz, dirs_n);
        int shared = 0;
        for (int k = 0; k < 4; ++k)
            if (dirs_n[k] && dirs0[k])
                shared = 1;
        if (!shared)
            break;
        dist += 1;
    }
    return found_end ? dist : -dist;
}

/* R7 and Eq. 5: normalisation along one axis.  r_neg / r_pos are the walks
 * towards decreasing / increasing index, f the in-texel offset of the fragment
 * along the axis.  The aliased edge along the axis covers |r_neg| + |r_pos| - 1
 * texels (the fragment's texel plus those each walk passed).  The position is
 * measured from the side where an end was found, which puts the origin in the
 * corner of the aliasing (§3.1.4).  code follows Eq. 5: +1 both ends found,
 * 0 one end, -1 none.  Double-precision variant. */
static double axis_position_f64(int r_neg, int r_pos, double f, int *code)
{
    int len = abs(r_neg) + abs(r_pos) - 1;
    int ends = (r_neg > 0) + (r_pos > 0);
    *code = ends == 2 ? 1 : (ends == 1 ? 0 : -1);
    if (ends == 0)
        return 1.0;
    double from_neg = ((double)(r_neg - 1) + f) / (double)len;
    double from_pos = ((double)(r_pos - 1) + (1.0 - f)) / (double)len;
    if (ends == 2)
        return from_neg < from_pos ? from_neg : from_pos;
    return r_neg > 0 ? from_neg : from_pos;
}

/* Same normalisation in single precision.  The silhouette visibility turns
 * this float into a 0/1 decision, so it is taken in the paper's precision
 * (GLSL float); the operations are one add and one correctly rounded divide. */
static float axis_position_f32(int r_neg, int r_pos, float f)
{
    int len = abs(r_neg) + abs(r_pos) - 1;
    int ends = (r_neg > 0) + (r_pos > 0);
    if (ends == 0)
        return 1.0f;
    float from_neg = ((float)(r_neg - 1) + f) / (float)len;
    float from_pos = ((float)(r_pos - 1) + (1.0f - f)) / (float)len;
    if (ends == 2)
        return from_neg < from_pos ? from_neg : from_pos;
    return r_neg > 0 ? from_neg : from_pos;
}

/* The four shadow-edge shapes of Fig. 2 (§3.1.4, §3.2.4, §4), told apart
 * from what the fragment's neighbourhood and traversal found: per axis,
 * whether the fragment has discontinuity directions on both sides
 * (opposite[a]: d.x or d.y of Eq. 4 is 0.75) and how many of the two walks
 * along it found an end (ends[a] = 0, 1, 2; Eq. 5 codes them 1, 0, -1 for
 * 2, 1, 0). */
enum { SHAPE_I, SHAPE_L, SHAPE_U, SHAPE_O };

/* §4.1, silhouette recovery: U- and O-shaped edges are those with
 * discontinuity directions on both sides of an axis or an end found on both
 * sides of an axis (the fragment sits between two shadowed neighbours); an
 * I-shaped edge is one where no end was found along an axis; every other
 * edge is L-shaped.  (U and O get the same answer.) */
static int silhouette_shape(const int opposite[2], const int ends[2])
{
    for (int a = 0; a < 2; ++a)
        if (opposite[a] || ends[a] == 2)
            return SHAPE_U;
    for (int a = 0; a < 2; ++a)
        if (ends[a] == 0)
            return SHAPE_I;
    return SHAPE_L;
}

/* §4.1: U and O edges are closed (shadow), I edges stay as the shadow test
 * found them (lit: only lit fragments get here), and an L edge is cut by
 * the revectorisation line through the corner of the aliasing: a fragment
 * is shadowed when its vertical distance ny is below 1 - its horizontal
 * distance nx (float32, as the shader computes it; a point on the line
 * stays lit). */
static double silhouette_visibility(const int opposite[2], const int ends[2], float nx, float ny)
{
    switch (silhouette_shape(opposite, ends)) {
    case SHAPE_U: return 0.0;
    case SHAPE_I: return 1.0;
    default: {
        float line = 1.0f - nx;
        return ny < line ? 0.0 : 1.0;
    }
    }
}

/* §4.2, filtering: an O-shaped edge is closed on both axes (discontinuity
 * directions on both sides of both axes, or ends on both sides of both);
 * a U-shaped edge has ends on both sides of one axis; an I-shaped edge has
 * no end along an axis; every other edge is L-shaped. */
static int filter_shape(const int opposite[2], const int ends[2])
{
    if ((opposite[0] && opposite[1]) || (ends[0] == 2 && ends[1] == 2))
        return SHAPE_O;
    if (ends[0] == 2 || ends[1] == 2)
        return SHAPE_U;
    if (ends[0] == 0 || ends[1] == 0)      /* R11 */
        return SHAPE_I;
    return SHAPE_L;
}

/* §4.2, on either side of the edge (dz = 1 - s, sign = 1 - 2 dz):
 *   O: the opposite of the shadow test (the edge is closed);
 *   U: the normalised distance across the open axis, measured from the
 *      fragment's side (ends along x: ny; ends along y: nx);
 *   I: the shadow test;
 *   L: the sum of both normalised distances from the fragment's side,
 *      clamped to [0, 1]. */
static double filter_visibility(const int opposite[2], const int ends[2], int dz, double nx, double ny)
{
    const double sgn = 1.0 - 2.0 * (double)dz;
    switch (filter_shape(opposite, ends)) {
    case SHAPE_O: return (double)dz;
    case SHAPE_U: return ends[0] == 2 ? (double)dz + sgn * ny : (double)dz + sgn * nx;
    case SHAPE_I: return 1.0 - (double)dz;
    default: {
        double v = (double)dz + sgn * ny + sgn * nx;
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        return v;
    }
    }
}

/* Listing 1 with Listings 2-5: visibility of one fragment.
 * Writes the visibility, the uint16 code, and optionally the four walks and
 * the normalised vector (nx, ny, cx, cy).
 * Code bits: 0-3 discontinuity directions (left, right, +y, -y), 4 = d.z
 * (shadow-test failed), 5-6 ends found along x (0..2), 7-8 ends found along
 * y, 9 = the fragment went through the edge traversal. */
static void rbsm_fragment_uv(const sm_t *sm, float u, float v, float pz, int mode, int max_dist,
                             double *vis_out, uint16_t *code_out, int32_t rd_out[4], double nrd_out[4])
{
    /* R1, R17: texel and in-texel offset of the texel-space position (u, v) */
    float fu = floorf(u), fv = floorf(v);
    float fx = u - fu, fy = v - fv;
    /* clamp while still a float (fmaxf/fminf pick the non-NaN operand, so a
     * NaN coordinate lands on the first texel) */
    int64_t i = (int64_t)fminf(fmaxf(fu, 0.0f), (float)(sm->width - 1));
    int64_t j = (int64_t)fminf(fmaxf(fv, 0.0f), (float)(sm->height - 1));

    int dirs[4];
    int s0 = discontinuity4(sm, i, j, pz, dirs);
    int dz = 1 - s0;
    /* Eq. 4 in quarters: d.x = (2 d_left + d_right)/4, d.y = (2 d_+y + d_-y)/4 */
    int dxq = 2 * dirs[0] + dirs[1];
    int dyq = 2 * dirs[2] + dirs[3];

    uint16_t code = (uint16_t)(dirs[0] | (dirs[1] << 1) | (dirs[2] << 2) | (dirs[3] << 3) | (dz << 4));
    int32_t rd[4] = {0, 0, 0, 0};
    double nrd[4] = {0.0, 0.0, 0.0, 0.0};
    double vis;

    if (mode == ORACLE_MODE_SILHOUETTE && s0 == 0) {
        /* Listing 1: shadowed fragments stay shadowed in silhouette recovery */
        vis = 0.0;
    } else if (dxq == 0 && dyq == 0) {
        /* Listing 1: outside a shadow edge the shadow test is the answer */
        vis = (double)s0;
    } else {
        /* R6: the four walks */
        rd[0] = traverse_edge(sm, i, j, pz, s0, dirs, -1, 0, max_dist);
        rd[1] = traverse_edge(sm, i, j, pz, s0, dirs, +1, 0, max_dist);
        rd[2] = traverse_edge(sm, i, j, pz, s0, dirs, 0, -1, max_dist);
        rd[3] = traverse_edge(sm, i, j, pz, s0, dirs, 0, +1, max_dist);
        int cx, cy;
        double nx = axis_position_f64(rd[0], rd[1], (double)fx, &cx);
        double ny = axis_position_f64(rd[2], rd[3], (double)fy, &cy);
        nrd[0] = nx;
        nrd[1] = ny;
        nrd[2] = (double)cx;
        nrd[3] = (double)cy;
        int ex = (rd[0] > 0) + (rd[1] > 0);
        int ey = (rd[2] > 0) + (rd[3] > 0);
        code = (uint16_t)(code | (ex << 5) | (ey << 7) | (1 << 9));
        const int opposite[2] = {dxq == 3, dyq == 3};
        const int ends[2] = {ex, ey};
        if (mode == ORACLE_MODE_SILHOUETTE) {
            float nx32 = axis_position_f32(rd[0], rd[1], fx);
            float ny32 = axis_position_f32(rd[2], rd[3], fy);
            vis = silhouette_visibility(opposite, ends, nx32, ny32);
        } else {
            vis = filter_visibility(opposite, ends, dz, nx, ny);
        }
    }
    *vis_out = vis;
    if (code_out)
        *code_out = code;
    if (rd_out)
        for (int k = 0; k < 4; ++k) rd_out[k] = rd[k];
    if (nrd_out)
        for (int k = 0; k < 4; ++k) nrd_out[k] = nrd[k];
}

/* R1: the texel-space position is the single-precision product x * W. */
static void rbsm_fragment(const sm_t *sm, float x, float y, float pz, int mode, int max_dist,
                          double *vis_out, uint16_t *code_out, int32_t rd_out[4], double nrd_out[4])
{
    float u = x * (float)sm->width;
    float v = y * (float)sm->height;
    rbsm_fragment_uv(sm, u, v, pz, mode, max_dist, vis_out, code_out, rd_out, nrd_out);
}

/* The visibility of an edge fragment from its shape inputs alone (per axis:
 * discontinuity directions on both sides, ends found; dz; the normalised
 * distances), for the tests that set it against the listings' branches.
 * Silhouette mode takes nx, ny as float32, as the fragment path does. */
double oracle_edge_visibility(int32_t mode, int32_t opposite_x, int32_t opposite_y, int32_t ends_x,
                              int32_t ends_y, int32_t dz, double nx, double ny)
{
    const int opposite[2] = {opposite_x != 0, opposite_y != 0};
    const int ends[2] = {ends_x, ends_y};
    if (mode == ORACLE_MODE_SILHOUETTE)
        return silhouette_visibility(opposite, ends, (float)nx, (float)ny);
    return filter_visibility(opposite, ends, dz, nx, ny);
}

/* Evaluate n fragments.  Returns 0, or -1 on invalid arguments.
 * rd (n*4 int32), nrd (n*4 double) and codes may be NULL. */
int oracle_rbsm_eval(const float *depth, int32_t width, int32_t height, int64_t pitch,
                     const float *px, const float *py, const float *pz, int64_t n,
                     int32_t mode, int32_t max_dist,
                     double *vis, uint16_t *codes, int32_t *rd, double *nrd)
{
    if (!depth || width < 1 || height < 1 || pitch < width || n < 0 || max_dist < 1)
        return -1;
    if (n > 0 && (!px || !py || !pz || !vis))
        return -1;
    if (mode != ORACLE_MODE_SILHOUETTE && mode != ORACLE_MODE_FILTER)
        return -1;
    sm_t sm = {depth, width, height, pitch};
    for (int64_t t = 0; t < n; ++t) {
        rbsm_fragment(&sm, px[t], py[t], pz[t], mode, max_dist, &vis[t],
                      codes ? &codes[t] : NULL,
                      rd ? &rd[4 * t] : NULL,
                      nrd ? &nrd[4 * t] : NULL);
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Fragments from a depth buffer (the varying p of Listing 1, "the fragment
 * transformed into light space", formed from a G-buffer).  Reading:
 *   R21 pixel (px, py) of a width x height buffer holds depth d; with the
 *       4 x 4 row-major float32 matrix M (screen to light clip space),
 *       (X, Y, Z, W) = M (px + 0.5, py + 0.5, d, 1), each row summed left to
 *       right, and p = (X / W, Y / W, Z / W), all single precision.
 * Fragment f = py * width + px.  Writes the light-space planes; returns 0,
 * or -1 on invalid arguments. */
int oracle_project(const float *depth, int32_t width, int32_t height, int64_t pitch, const float *m,
                   float *px_out, float *py_out, float *pz_out)
{
    if (!depth || !m || !px_out || !py_out || !pz_out || width < 1 || height < 1 || pitch < width)
        return -1;
    for (int64_t py = 0; py < height; ++py) {
        for (int64_t px = 0; px < width; ++px) {
            const float sx = (float)px + 0.5f, sy = (float)py + 0.5f, d = depth[py * pitch + px];
            float v[4];
            for (int r = 0; r < 4; ++r) {
                const float *row = m + 4 * r;
                v[r] = row[0] * sx + row[1] * sy + row[2] * d + row[3];
            }
            const int64_t f = py * width + px;
            px_out[f] = v[0] / v[3];
            py_out[f] = v[1] / v[3];
            pz_out[f] = v[2] / v[3];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * RPCF: percentage-closer filtering over the RSMSS answer (§5.3 suppresses
 * the skeleton artifacts of the filtered edges with PCF; the paper prints no
 * kernel for it).  Readings:
 *   R18 the k x k PCF samples are the fragment's texel-space position
 *       (u, v) = (x W, y H) (single precision, R1) shifted by whole texels,
 *       (u + a, v + b) for a, b = -(k-1)/2 .. (k-1)/2, each shift a
 *       single-precision add; every sample keeps the fragment's depth.
 *   R19 a sample's answer is the Listing 5 (RSMSS) visibility of that
 *       position, walks and all; the RPCF answer is their mean, summed with
 *       b outer and a inner.
 * k = 1 is RSMSS itself.  Returns 0, or -1 on invalid arguments (k must be
 * odd, 1..7). */
int oracle_rpcf(const float *depth, int32_t width, int32_t height, int64_t pitch,
                const float *px, const float *py, const float *pz, int64_t n,
                int32_t k, int32_t max_dist, double *vis)
{
    if (!depth || width < 1 || height < 1 || pitch < width || n < 0 || max_dist < 1)
        return -1;
    if (k < 1 || k > 7 || (k & 1) == 0)
        return -1;
    if (n > 0 && (!px || !py || !pz || !vis))
        return -1;
    sm_t sm = {depth, width, height, pitch};
    const int r = (k - 1) / 2;
    for (int64_t t = 0; t < n; ++t) {
        float u = px[t] * (float)width;
        float v = py[t] * (float)height;
        double sum = 0.0;
        for (int b = -r; b <= r; ++b) {
            for (int a = -r; a <= r; ++a) {
                double va;
                rbsm_fragment_uv(&sm, u + (float)a, v + (float)b, pz[t], ORACLE_MODE_FILTER, max_dist, &va,
                                 NULL, NULL, NULL);
                sum += va;
            }
        }
        vis[t] = sum / (double)(k * k);
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Features of the learned penumbra surrogate.  Not in the paper: this
 * project's surrogate of the Listing 5 (RSMSS) answer for edge fragments
 * reads, per fragment,
 *   bits: the shadow tests (Eq. 1, with the fragment's depth) of the 5x5
 *         texels around its texel (clamp to edge, R2); texel (i+dx, j+dy)
 *         sets bit (dy+2)*5 + (dx+2) when it is lit;
 *   fx, fy: the in-texel offsets of R1;
 *   gap:  the fragment's depth minus the smallest depth stored in the 5x5
 *         window (float32 subtraction), the blocker-receiver depth gap.
 * Returns 0, or -1 on invalid arguments.
 */
int oracle_features(const float *depth, int32_t width, int32_t height, int64_t pitch,
                    const float *px, const float *py, const float *pz, int64_t n,
                    uint32_t *bits, float *fx_out, float *fy_out, float *gap_out)
{
    if (!depth || width < 1 || height < 1 || pitch < width || n < 0)
        return -1;
    if (n > 0 && (!px || !py || !pz || !bits || !fx_out || !fy_out || !gap_out))
        return -1;
    sm_t sm = {depth, width, height, pitch};
    for (int64_t t = 0; t < n; ++t) {
        float u = px[t] * (float)width;
        float v = py[t] * (float)height;
        float fu = floorf(u), fv = floorf(v);
        int64_t i = (int64_t)fminf(fmaxf(fu, 0.0f), (float)(width - 1));
        int64_t j = (int64_t)fminf(fmaxf(fv, 0.0f), (float)(height - 1));
        uint32_t b = 0;
        float zmin = sm_depth(&sm, i, j);
        for (int dy = -2; dy <= 2; ++dy) {
            for (int dx = -2; dx <= 2; ++dx) {
                float zt = sm_depth(&sm, i + dx, j + dy);
                if (shadow_test(pz[t], zt))
                    b |= 1u << ((dy + 2) * 5 + (dx + 2));
                if (zt < zmin)
                    zmin = zt;
            }
        }
        bits[t] = b;
        fx_out[t] = u - fu;
        fy_out[t] = v - fv;
        gap_out[t] = pz[t] - zmin;
    }
    return 0;
}
