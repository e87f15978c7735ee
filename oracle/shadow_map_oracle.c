/*
 * Plain CPU oracle of the light pass that produces a shadow map from
 * analytic occluders (the step before the RBSM path: the paper renders its
 * shadow map with the graphics pipeline, §3 / Listing 1's input SM; here
 * the occluders are oriented rectangles and spheres seen by an
 * orthographic light looking down the depth axis).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA rasteriser is checked
 * against.  Only the
 * tests, the smoke check and the benchmark's CPU baseline may load it; it
 * shares no code with the CUDA library.
 *
 * Definition, by brute force: texel (i, j) samples the point
 * (i + 0.5, j + 0.5) of the light's image plane (point sampling at texel
 * centres).  It stores the smallest depth of every occluder that covers that
 * point, and `ground` when none does.
 *   rectangle (cx, cy, ux, uy, ha, hb, depth): with p = point - c, covered
 *     when |p . (ux, uy)| <= ha and |p . (-uy, ux)| <= hb;
 *   sphere (cx, cy, R, centre): with rho^2 = |point - c|^2, covered when
 *     rho^2 <= R^2; its depth there is centre - sqrt(R^2 - rho^2) / zscale
 *     (the hemisphere facing the light), rounded to float32.
 * Every product and sum is a separate IEEE double operation (the build
 * turns contraction off), in the order written.
 *
 * Build: gcc -O2 -ffp-contract=off (no fast-math).
 */
#include <math.h>
#include <stdint.h>

/* rect: n_rects x 6 doubles (cx, cy, ux, uy, ha, hb) and n_rects float
 * depths; sph: n_spheres x 4 doubles (cx, cy, R, centre depth).
 * Returns 0, or -1 on invalid arguments. */
int oracle_shadow_map(float *depth, int32_t width, int32_t height, int64_t pitch,
                      const double *rect, const float *rect_depth, int32_t n_rects,
                      const double *sph, int32_t n_spheres, double zscale, float ground)
{
    if (!depth || width < 1 || height < 1 || pitch < width || n_rects < 0 || n_spheres < 0)
        return -1;
    if ((n_rects > 0 && (!rect || !rect_depth)) || (n_spheres > 0 && !sph) || !(zscale > 0.0))
        return -1;
    for (int64_t j = 0; j < height; ++j) {
        for (int64_t i = 0; i < width; ++i) {
            const double qx = (double)i + 0.5, qy = (double)j + 0.5;
            float best = ground;
            for (int32_t k = 0; k < n_rects; ++k) {
                const double *r = rect + 6 * k;
                const double px = qx - r[0], py = qy - r[1];
                const double s = px * r[2] + py * r[3];
                const double t = -px * r[3] + py * r[2];
                if (fabs(s) <= r[4] && fabs(t) <= r[5] && rect_depth[k] < best)
                    best = rect_depth[k];
            }
            for (int32_t k = 0; k < n_spheres; ++k) {
                const double *c = sph + 4 * k;
                const double dx = qx - c[0], dy = qy - c[1];
                const double rho2 = dx * dx + dy * dy, r2 = c[2] * c[2];
                if (rho2 > r2)
                    continue;
                const float d = (float)(c[3] - sqrt(r2 - rho2) / zscale);
                if (d < best)
                    best = d;
            }
            depth[j * pitch + i] = best;
        }
    }
    return 0;
}
