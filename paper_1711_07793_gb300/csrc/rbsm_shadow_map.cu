// Shadow maps of analytic occluders (rbsm_shadow_map): the light pass whose
// output, SM, is the input of Listing 1.  Texel (i, j) point-samples
// (i + 0.5, j + 0.5) and keeps the smallest depth of the oriented
// rectangles and sphere caps covering it.
//
// A CTA owns 32 x 32 texel tiles (persistent, grid-stride over tiles).  Per
// tile it first culls the occluders, 256 at a time, with float tests that
// can only keep too many (the tile's texel centres projected on the
// rectangle's own two axes, the disc against the box of texel centres, both
// widened by half a texel), gathers the survivors in shared memory, and then
// every thread tests its 4 texels against them.  Double precision is slow on
// this GPU, so each test runs first in float, relative to the tile centre,
// with an error bound: a float decision further than the bound from its
// threshold is the exact one, and only texels within the bound of an edge
// (and the cap depths of covered sphere texels) take the exact double
// operations, in the defined order without contraction, so the map is
// bit-exact.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rbsm.h"
#include "rbsm_host.h"

namespace rbsm {
namespace {

constexpr int kTile = 32;                 // texels per tile side
constexpr int kSmThreads = 256;           // 8 rows of 32 per pass, 4 passes
constexpr int kChunk = kSmThreads;        // occluders culled per round
constexpr float kCullSlack = 0.5f;        // texels added to every (float) culling bound

// A surviving occluder of the current tile.  Besides the exact parameters
// (for the double-precision test) it carries its position relative to the
// tile centre in float and an error bound E for the float pre-test: every
// float decision further than E from its threshold is the exact one.
struct RectCand {
    double cx, cy, ux, uy, ha, hb;
    float s0, t0, uxf, uyf, haf, hbf, es, et;   // s, t at the tile centre; bounds of the float s, t
    float depth;
};

struct SphereCand {
    double cx, cy, r, c;
    float dx0, dy0, r2f, e;                       // centre offset from the tile centre; rho^2 bound
    float dmin;                                   // no texel of the cap is nearer the light than this
};

struct TileSmem {
    union {
        RectCand r[kChunk];
        SphereCand s[kChunk];
    };
    int n;
};

// Float copies of up to kFloatCopies occluders of each kind, made once per
// CTA, for the culling and the float pre-tests; `ea` bounds what the
// rounding of the centre to float moves any projection (|c - c_f| (|ux| +
// |uy|) <= (|cx| + |cy|) 2^-24 * sqrt 2, taken as 2^-22).
constexpr int kFloatCopies = 512;
struct FloatOcc {
    float cx, cy, ux, uy, ha, hb, ea;
};
struct FloatSph {
    float cx, cy, r, ea;
};

// Float error bound of a quantity whose operands are at most `mag` in
// magnitude after a handful of float roundings (2^-20 of it: 16 ulps) plus
// a fixed floor for the tile offsets (|offset| <= 31, rounding ~ 31 * 2^-24).
__device__ __forceinline__ float err_bound(float mag)
{
    return mag * 9.5367431640625e-07f + 1e-5f;    // 2^-20
}

__device__ __forceinline__ FloatOcc float_rect(const rbsm_rect &r)
{
    return FloatOcc{(float)r.cx, (float)r.cy, (float)r.ux, (float)r.uy, (float)r.ha, (float)r.hb,
                    (float)(fabs(r.cx) + fabs(r.cy)) * 2.384185791015625e-07f};    // 2^-22
}

__device__ __forceinline__ FloatSph float_sphere(const rbsm_sphere &c)
{
    return FloatSph{(float)c.cx, (float)c.cy, (float)c.radius,
                    (float)(fabs(c.cx) + fabs(c.cy) + c.radius) * 2.384185791015625e-07f};
}

// Cull occluders base + threadIdx.x against the tile centred at (tcx, tcy)
// (float copies when the CTA holds them, else the double parameters) and
// gather the survivors with their float pre-test data.
template <bool RECT>
__device__ __forceinline__ void cull_chunk(const rbsm_occluders &occ, const FloatOcc *fo, const FloatSph *fs,
                                           int base, float tcx, float tcy, TileSmem &sm)
{
    constexpr float h = 0.5f * (kTile - 1);        // half size of the box of texel centres
    const int k = base + (int)threadIdx.x;
    const int n = RECT ? occ.n_rects : occ.n_spheres;
    bool keep = false;
    RectCand rc;
    SphereCand sc;
    if (k < n) {
        if (RECT) {
            const FloatOcc f = fo ? fo[k] : float_rect(occ.rects[k]);
            // tcx - cx and the projections in float: the error is at most
            // f.ea (centre rounding) + 2^-22 (|s0| + |t0|-size terms)
            const float dx = tcx - f.cx, dy = tcy - f.cy;
            rc.s0 = dx * f.ux + dy * f.uy;
            rc.t0 = -dx * f.uy + dy * f.ux;
            // |(q - tc) . u| over the tile's centres is at most h (|ux| + |uy|)
            const float spread = h * (fabsf(f.ux) + fabsf(f.uy));
            keep = fabsf(rc.s0) <= f.ha + spread + kCullSlack && fabsf(rc.t0) <= f.hb + spread + kCullSlack;
            if (keep) {
                const rbsm_rect r = occ.rects[k];
                rc.uxf = f.ux;
                rc.uyf = f.uy;
                rc.haf = f.ha;
                rc.hbf = f.hb;
                const float mag = fabsf(dx) + fabsf(dy);
                rc.es = err_bound(fabsf(rc.s0) + f.ha + spread + mag) + f.ea;
                rc.et = err_bound(fabsf(rc.t0) + f.hb + spread + mag) + f.ea;
                rc.cx = r.cx; rc.cy = r.cy; rc.ux = r.ux; rc.uy = r.uy; rc.ha = r.ha; rc.hb = r.hb;
                rc.depth = r.depth;
            }
        } else {
            const FloatSph f = fs ? fs[k] : float_sphere(occ.spheres[k]);
            sc.dx0 = tcx - f.cx;
            sc.dy0 = tcy - f.cy;
            const float gx = fmaxf(fabsf(sc.dx0) - h, 0.0f), gy = fmaxf(fabsf(sc.dy0) - h, 0.0f);
            const float rr = f.r + kCullSlack;
            keep = gx * gx + gy * gy <= rr * rr;
            if (keep) {
                const rbsm_sphere c = occ.spheres[k];
                sc.r2f = f.r * f.r;
                const float far = fabsf(sc.dx0) + fabsf(sc.dy0) + 2.0f * h + f.r + f.ea;
                sc.e = err_bound(far * far) + 2.0f * far * f.ea;
                // the cap's depth is at least c - R / zscale (R widened by
                // 1e-6 for the rounding of R^2 and the square root), one float below
                sc.dmin = nextafterf((float)(c.centre_depth - c.radius * 1.000001 / occ.zscale), -INFINITY);
                sc.cx = c.cx; sc.cy = c.cy; sc.r = c.radius; sc.c = c.centre_depth;
            }
        }
    }
    if (threadIdx.x == 0)
        sm.n = 0;
    __syncthreads();
    if (keep) {
        const int slot = atomicAdd(&sm.n, 1);
        if (RECT)
            sm.r[slot] = rc;
        else
            sm.s[slot] = sc;
    }
    __syncthreads();
}

// inv_zscale: 1 / zscale when zscale is a power of two (dividing by it is
// then the exact multiplication by its reciprocal), else 0.
__global__ void __launch_bounds__(kSmThreads) shadow_map_kernel(const rbsm_occluders occ, float *__restrict__ depth,
                                                                int width, int height, long long pitch,
                                                                double inv_zscale)
{
    __shared__ TileSmem sm;
    __shared__ FloatOcc fo[kFloatCopies];
    __shared__ FloatSph fs[kFloatCopies];
    const bool copies = occ.n_rects <= kFloatCopies && occ.n_spheres <= kFloatCopies;
    if (copies) {
        for (int k = threadIdx.x; k < occ.n_rects; k += blockDim.x)
            fo[k] = float_rect(occ.rects[k]);
        for (int k = threadIdx.x; k < occ.n_spheres; k += blockDim.x)
            fs[k] = float_sphere(occ.spheres[k]);
        __syncthreads();
    }
    const FloatOcc *fop = copies ? fo : nullptr;
    const FloatSph *fsp = copies ? fs : nullptr;
    const int tiles_x = (width + kTile - 1) / kTile;
    const long long tiles = (long long)tiles_x * ((height + kTile - 1) / kTile);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    constexpr float h = 0.5f * (kTile - 1);
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int i0 = (int)(tile % tiles_x) * kTile, j0 = (int)(tile / tiles_x) * kTile;
        const float tcx = (float)i0 + 0.5f + h, tcy = (float)j0 + 0.5f + h;    // exact (< 2^23)
        const int i = i0 + tx;
        const double qx = __dadd_rn((double)i, 0.5);
        const float ox = (float)tx - h;                // texel centre - tile centre (exact)
        float best[4];
        double qy[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            best[p] = occ.ground;
            qy[p] = (double)(j0 + ty + 8 * p) + 0.5;   // exact
        }
        for (int base = 0; base < occ.n_rects; base += kChunk) {
            cull_chunk<true>(occ, fop, fsp, base, tcx, tcy, sm);
            for (int q = 0; q < sm.n; ++q) {
                const RectCand &r = sm.r[q];
                const float sx = ox * r.uxf, tx_ = -ox * r.uyf;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float oy = (float)(ty + 8 * p) - h;
                    const float sf = fabsf(r.s0 + (sx + oy * r.uyf));
                    const float tf = fabsf(r.t0 + (tx_ + oy * r.uxf));
                    if (sf > r.haf + r.es || tf > r.hbf + r.et || !(r.depth < best[p]))
                        continue;                      // surely outside, or it cannot lower the depth
                    bool in = sf < r.haf - r.es && tf < r.hbf - r.et;
                    if (!in) {
                        // near an edge: the exact test, double operations in the defined order
                        const double px = __dsub_rn(qx, r.cx), py = __dsub_rn(qy[p], r.cy);
                        const double s = __dadd_rn(__dmul_rn(px, r.ux), __dmul_rn(py, r.uy));
                        const double t = __dadd_rn(__dmul_rn(-px, r.uy), __dmul_rn(py, r.ux));
                        in = fabs(s) <= r.ha && fabs(t) <= r.hb;
                    }
                    if (in)
                        best[p] = r.depth;
                }
            }
            __syncthreads();                       // survivors read before the next chunk
        }
        for (int base = 0; base < occ.n_spheres; base += kChunk) {
            cull_chunk<false>(occ, fop, fsp, base, tcx, tcy, sm);
            for (int q = 0; q < sm.n; ++q) {
                const SphereCand &c = sm.s[q];
                const float dxf = c.dx0 + ox;
                const double dx = __dsub_rn(qx, c.cx);
                const double r2 = __dmul_rn(c.r, c.r);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float dyf = c.dy0 + ((float)(ty + 8 * p) - h);
                    if (!(c.dmin < best[p]) || dxf * dxf + dyf * dyf > c.r2f + c.e)
                        continue;                      // cannot lower the depth, or surely outside the disc
                    const double dy = __dsub_rn(qy[p], c.cy);
                    const double rho2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                    if (rho2 > r2)
                        continue;
                    const double root = __dsqrt_rn(__dsub_rn(r2, rho2));
                    const double drop = inv_zscale != 0.0 ? __dmul_rn(root, inv_zscale) : __ddiv_rn(root, occ.zscale);
                    const float d = __double2float_rn(__dsub_rn(c.c, drop));
                    if (d < best[p])
                        best[p] = d;
                }
            }
            __syncthreads();
        }
        if (i < width) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int j = j0 + ty + 8 * p;
                if (j < height)
                    depth[(long long)j * pitch + i] = best[p];
            }
        }
    }
}

}  // namespace
}  // namespace rbsm

extern "C" int rbsm_shadow_map(const rbsm_occluders *occ, float *depth, int32_t width, int32_t height,
                               int64_t pitch, void *stream)
{
    using namespace rbsm;
    if (!occ || !depth || width < 1 || width > RBSM_MAX_EXTENT || height < 1 || height > RBSM_MAX_EXTENT ||
        pitch < width || occ->n_rects < 0 || occ->n_spheres < 0 || (occ->n_rects > 0 && !occ->rects) ||
        (occ->n_spheres > 0 && !occ->spheres) || !(occ->zscale > 0.0) || occ->flags != 0)
        return RBSM_ERR_ARG;
    static KernelSetup setup;
    int occupancy = 0;
    int rc = setup.get(shadow_map_kernel, kSmThreads, 0, &occupancy);
    if (rc != RBSM_OK)
        return rc;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    const long long tiles = (long long)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
    long long grid = (long long)sms * occupancy;
    if (grid > tiles)
        grid = tiles;
    int e2 = 0;
    const double inv = std::frexp(occ->zscale, &e2) == 0.5 ? std::ldexp(1.0, 1 - e2) : 0.0;
    shadow_map_kernel<<<(unsigned)grid, kSmThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        *occ, depth, width, height, pitch, inv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}
