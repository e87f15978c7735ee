// Shadow maps of analytic occluders (rbsm_shadow_map): the light pass whose
// output, SM, is the input of Listing 1.  Texel (i, j) point-samples
// (i + 0.5, j + 0.5) and keeps the smallest depth of the oriented
// rectangles and sphere caps covering it.
//
// A CTA owns 32 x 32 texel tiles (persistent, grid-stride over tiles).  Per
// tile it culls the occluders of both kinds, 256 at a time, with float tests
// that can only keep too many (the tile's texel centres projected on the
// rectangle's own two axes, the disc against the box of texel centres, both
// widened by half a texel), gathers the survivors in shared memory in index
// order, and every thread tests its 4 texels against them.  Double precision is slow on
// this GPU, so the map's double-precision definition is reached mostly in
// float:
//   * the coverage tests run first in float, relative to the tile centre,
//     with an error bound: a decision further than the bound from its
//     threshold is the exact one;
//   * a covered sphere texel's cap depth, RN32(c - sqrt(R^2 - rho^2) / z)
//     of the double operations, is evaluated in float-float arithmetic
//     (Knuth's TwoSum, the FMA product error, one Newton step for the
//     square root) with a rigorous bound B on its distance from the double
//     result; when the float-float value is further than B from every float
//     rounding boundary, its rounding is the double result's;
//   * everything else (texels within the bound of an edge, the few cap
//     depths near a rounding boundary, scales z that are not powers of two)
//     takes the exact double operations in the defined order without
//     contraction,
// so the map is bit-exact.
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
    float s0, t0, uxf, uyf, haf, hbf, es, et;   // s, t at the tile centre; bounds of the float s, t
    float depth;
    int k;                                        // the rectangle (its double parameters for the exact test)
};

struct SphereCand {
    float dx0, dy0, r2f, e;                       // centre offset from the tile centre; rho^2 bound
    float dmin;                                   // no texel of the cap is nearer the light than this
    // float-float data of the cap depth: tile centre - disc centre
    // (dx0h + dx0l, dy0h + dy0l; within 2^-47 (|offset| + |centre|)),
    // R^2 = r2h + r2l and c = ch + cl (within 2^-47 of the doubles), the
    // centre's magnitude (cxa, cya); fast = 0 keeps every texel on the
    // double operations
    float dx0h, dx0l, dy0h, dy0l, r2h, r2l, ch, cl, cxa, cya;
    int fast;
    int k;                                        // the sphere (its double parameters for the exact depth)
};

// The survivors of one culling round (at most kChunk of both kinds): the
// rectangles in index order from slot 0, then the spheres in index order.
union Cand {
    RectCand r;
    SphereCand s;
};

constexpr int kSmWarps = kSmThreads / 32;

// Each thread writes its survivor to its own slot of the round's buffer
// (two buffers, alternating by round, so that a warp starting the next
// round never overwrites candidates another warp still reads); the
// order-keeping compaction moves only indices.
struct TileSmem {
    Cand c[2][kChunk];
    int idx[kChunk];                          // survivors' slots: rectangles, then spheres, in index order
    int cnt_r[kSmWarps], cnt_s[kSmWarps];     // survivors per warp, for the order-keeping offsets
};

// Float copies of up to kFloatCopies occluders of each kind, made once per
// CTA, for the culling and the float pre-tests; `ea` bounds what the
// rounding of the centre to float moves any projection (|c - c_f| (|ux| +
// |uy|) <= (|cx| + |cy|) 2^-24 * sqrt 2, taken as 2^-22).
constexpr int kFloatCopies = 256;
struct FloatOcc {
    float cx, cy, ux, uy, ha, hb, ea, depth;
};
struct FloatSph {
    float cx, cy, r, ea;         // cx, cy: the centre rounded to float
    float cxl, cyl;              // what that rounding dropped, rounded (cx + cxl within 2^-48 |cx|)
    float dmin;                  // no texel of the cap is nearer the light than this
    float r2h, r2l, ch, cl;      // R^2 and c as float pairs (within 2^-47 of the doubles)
    int fast;                    // R^2 and c in range for the float-float cap depth
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
                    (float)(fabs(r.cx) + fabs(r.cy)) * 2.384185791015625e-07f,    // 2^-22
                    r.depth};
}

__device__ __forceinline__ FloatSph float_sphere(const rbsm_sphere &c, double zscale)
{
    FloatSph f;
    f.cx = (float)c.cx;
    f.cy = (float)c.cy;
    f.cxl = (float)(c.cx - (double)f.cx);
    f.cyl = (float)(c.cy - (double)f.cy);
    f.r = (float)c.radius;
    f.ea = (float)(fabs(c.cx) + fabs(c.cy) + c.radius) * 2.384185791015625e-07f;
    // the cap's depth is at least c - R / zscale (R widened by 1e-6 for the
    // rounding of R^2 and the square root), one float below
    f.dmin = nextafterf((float)(c.centre_depth - c.radius * 1.000001 / zscale), -INFINITY);
    f.r2h = (float)(c.radius * c.radius);
    f.r2l = (float)fma(c.radius, c.radius, -(double)f.r2h);
    f.ch = (float)c.centre_depth;
    f.cl = (float)(c.centre_depth - (double)f.ch);
    f.fast = f.r2h >= 1e-30f && f.r2h <= 1e30f && fabsf(f.ch) <= 1e30f;
    return f;
}

// n as a float for 0 <= n < 2^23, from the bit pattern of 2^23 + n (an
// exact conversion in two integer/float operations).
__device__ __forceinline__ float small_int_float(int n)
{
    return __fsub_rn(__int_as_float(0x4B000000 | n), 8388608.0f);
}

// Knuth's TwoSum: s + e == a + b exactly (round to nearest; the _rn
// intrinsics are never contracted).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The terms of R^2 - dx^2 that depend on the texel column only.
struct CapColumn {
    float s1;      // r2h - px, high part (TwoSum)
    float low;     // its error + r2l - (dx^2 - px), rounded
    float ex;      // r2h + dx^2 + mx^2, the column's share of the bound on A
};

__device__ __forceinline__ CapColumn cap_column(const SphereCand &c, float ox)
{
    // dx = ox + (dx0h + dx0l) as dxh + dxl (ox is exact, within 15.5)
    float sh, sl, dxh, dxl;
    two_sum(ox, c.dx0h, sh, sl);
    two_sum(sh, __fadd_rn(sl, c.dx0l), dxh, dxl);
    const float px = __fmul_rn(dxh, dxh);
    const float pxe = __fmaf_rn(dxh, dxh, -px);                   // dxh^2 - px, exact
    const float cxt = __fmul_rn(__fmul_rn(2.0f, dxh), dxl);       // 2 dxh dxl
    CapColumn k;
    float e1;
    two_sum(c.r2h, -px, k.s1, e1);
    k.low = __fsub_rn(__fsub_rn(__fadd_rn(e1, c.r2l), pxe), cxt);
    const float mx = fabsf(ox) + fabsf(c.dx0h);
    k.ex = c.r2h + px + mx * (mx + c.cxa);
    return k;
}

// The cap depth of a texel by float-float arithmetic.  Returns 1 with *d =
// RN32 of the double operations' depth (the texel is covered), 0 when the
// double operations surely find the texel outside the disc, and -1 when
// this cannot decide (the caller takes the double operations).
//
// Error analysis (u = 2^-24 float, 2^-53 double unit roundoff):
//   A = R^2 - rho^2 (real) is held as ah + al with |ah + al - A| <= E_A =
//   2^-41 (R^2 + dx^2 + dy^2 + mx (mx + |cx|) + my (my + |cy|)), mx =
//   |ox| + |dx0h|: the split of R^2 loses 2^-47 R^2, the offset dx within
//   2^-45 (mx + |cx|) (so dx^2 within 2^-44 mx (mx + |cx|)), the squares are
//   exact (FMA) up to the 2 dxh dxl term (2^-47 dx^2) and the dropped dxl^2
//   (2^-48 dx^2), and the seven low terms are summed with error at most 6u
//   times their magnitudes (2^-43.1 of the squares).  When ah > 4 E_A and ah > 2^-40
//   R^2, A > 2^-41 R^2, far above the 5 * 2^-53 R^2 that the double
//   operations can move rho^2 <= R^2, so they find the texel covered.
//   sqrt(ah + al) ~ r0 + corr with r0 = sqrt(ah) (correctly rounded) and
//   one Newton step, corr = (ah - r0^2 + al) / (2 r0): error at most
//   2^-42 r0 with a reciprocal good to 2^-21, plus E_A / r0 from A.  The
//   scale 1/z is a power of two (exact in float), so the drop is
//   (r0 + corr)/z exactly.  v = (ch - dh) + ((vl + cl) - dl) then carries
//   2^-48 |c| from the split of c and 2^-22 (|vl| + |cl| + |dl|) from the
//   two roundings.  The double operations themselves are within 2^-53 (|c|
//   + 4 D + 8.2 R^2 / (r0 z)) of the real depth (D = the drop; rho^2 within
//   4 roundings, A within 6u_d R^2, then the square root, the scale and the
//   subtraction).  B below adds all of these with a factor 2 to spare, and
//   the test asks for 2 B of room, so the decision holds under the rounding
//   of B's own evaluation.
__device__ __forceinline__ int cap_fast(const SphereCand &c, const CapColumn &k, float oy, float invf, float &d)
{
    float sh, sl, dyh, dyl;
    two_sum(oy, c.dy0h, sh, sl);
    two_sum(sh, __fadd_rn(sl, c.dy0l), dyh, dyl);
    const float py = __fmul_rn(dyh, dyh);
    const float pye = __fmaf_rn(dyh, dyh, -py);
    const float cyt = __fmul_rn(__fmul_rn(2.0f, dyh), dyl);
    float s2, e2, ah, al;
    two_sum(k.s1, -py, s2, e2);
    two_sum(s2, __fsub_rn(__fsub_rn(__fadd_rn(k.low, e2), pye), cyt), ah, al);
    const float my = fabsf(oy) + fabsf(c.dy0h);
    const float ea = 4.547473508864641e-13f * (k.ex + py + my * (my + c.cya));   // 2^-41
    const float lim = 9.094947017729282e-13f * c.r2h;                     // 2^-40 R^2
    if (!(ah > 4.0f * ea && ah > lim))
        return ah < -(4.0f * ea + lim) ? 0 : -1;
    const float r0 = __fsqrt_rn(ah);
    const float rr = __fdividef(1.0f, r0);                                 // 1 / r0 within 2 ulp
    const float corr = __fmul_rn(__fadd_rn(__fmaf_rn(-r0, r0, ah), al), __fmul_rn(0.5f, rr));
    const float dh = __fmul_rn(r0, invf), dl = __fmul_rn(corr, invf);    // exact (power of two)
    float vh, vl, f, r;
    two_sum(c.ch, -dh, vh, vl);
    two_sum(vh, __fsub_rn(__fadd_rn(vl, c.cl), dl), f, r);               // f + r = the float-float depth
    const float B = 7.105427357601002e-15f * fabsf(c.ch)                                  // 2^-47
                    + invf * (4.547473508864641e-13f * r0                                  // 2^-41
                              + (1.01f * ea + 8.881784197001252e-16f * c.r2h) * rr)       // 2^-50
                    + 2.384185791015625e-07f * (fabsf(vl) + fabsf(c.cl) + fabsf(dl))       // 2^-22
                    + 7.52316384526264e-37f;                                               // 2^-120
    // half the gap from f to the float on r's side: 2^(e-24) for f in
    // [2^e, 2^(e+1)), 2^(e-25) below a power of two; positive normal f only
    const unsigned bits = __float_as_uint(f), ef = bits >> 23;
    if (ef < 26u || ef > 254u)
        return -1;
    const unsigned eh = ((bits & 0x7fffffu) == 0u && r < 0.0f) ? ef - 25u : ef - 24u;
    if (!(__fsub_rn(__uint_as_float(eh << 23), fabsf(r)) > 2.0f * B))
        return -1;
    d = f;
    return 1;
}

// The exact tests, out of line: the double-precision texel centre and the
// double operations in the defined order, without contraction.  Kept out
// of the tile loop so that it holds no double values (their conversions and
// arithmetic run on the slow FP64 pipe) for the few texels that need them.
__device__ __noinline__ bool rect_covers_exact(const rbsm_rect *rp, int i, int j)
{
    const rbsm_rect r = *rp;
    const double px = __dsub_rn((double)i + 0.5, r.cx), py = __dsub_rn((double)j + 0.5, r.cy);
    const double s = __dadd_rn(__dmul_rn(px, r.ux), __dmul_rn(py, r.uy));
    const double t = __dadd_rn(__dmul_rn(-px, r.uy), __dmul_rn(py, r.ux));
    return fabs(s) <= r.ha && fabs(t) <= r.hb;
}

// The cap depth of texel (i, j), or +infinity when the disc does not cover
// it (a value that lowers no depth, as an uncovered texel).
__device__ __noinline__ float cap_depth_exact(const rbsm_sphere *cp, int i, int j, double inv_zscale, double zscale)
{
    const rbsm_sphere c = *cp;
    const double dx = __dsub_rn((double)i + 0.5, c.cx), dy = __dsub_rn((double)j + 0.5, c.cy);
    const double r2 = __dmul_rn(c.radius, c.radius);
    const double rho2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (rho2 > r2)
        return INFINITY;
    const double root = __dsqrt_rn(__dsub_rn(r2, rho2));
    const double drop = inv_zscale != 0.0 ? __dmul_rn(root, inv_zscale) : __ddiv_rn(root, zscale);
    return __double2float_rn(__dsub_rn(c.centre_depth, drop));
}

// Cull the occluders of combined index base + threadIdx.x (rectangles
// 0..n_rects-1, then spheres) against the tile centred at (tcx, tcy) (float
// copies when the CTA holds them, else the double parameters) and gather
// the survivors with their float pre-test data (and, for spheres when
// `fast`, the float-float data of the cap depth), each kind in index order
// (ballots and per-warp counts, so every texel meets its occluders in the
// definition's order).  nr, ns: the survivors of each kind.
template <bool COPIES>
__device__ __forceinline__ void cull_round(const rbsm_occluders &occ, const FloatOcc *fo, const FloatSph *fs,
                                           long long base, float tcx, float tcy, bool fast, TileSmem &sm,
                                           Cand *buf, int &nr, int &ns)
{
    constexpr float h = 0.5f * (kTile - 1);        // half size of the box of texel centres
    const long long g = base + (long long)threadIdx.x;
    const unsigned lane = threadIdx.x & 31u;
    const int warp = threadIdx.x >> 5;
    bool keep_r = false, keep_s = false;
    RectCand rc;
    SphereCand sc;
    if (g < occ.n_rects) {
        const int k = (int)g;
        const FloatOcc f = COPIES ? fo[k] : float_rect(occ.rects[k]);
        // tcx - cx and the projections in float: the error is at most
        // f.ea (centre rounding) + 2^-22 (|s0| + |t0|-size terms)
        const float dx = tcx - f.cx, dy = tcy - f.cy;
        rc.s0 = dx * f.ux + dy * f.uy;
        rc.t0 = -dx * f.uy + dy * f.ux;
        // |(q - tc) . u| over the tile's centres is at most h (|ux| + |uy|)
        const float spread = h * (fabsf(f.ux) + fabsf(f.uy));
        keep_r = fabsf(rc.s0) <= f.ha + spread + kCullSlack && fabsf(rc.t0) <= f.hb + spread + kCullSlack;
        if (keep_r) {
            rc.uxf = f.ux;
            rc.uyf = f.uy;
            rc.haf = f.ha;
            rc.hbf = f.hb;
            const float mag = fabsf(dx) + fabsf(dy);
            rc.es = err_bound(fabsf(rc.s0) + f.ha + spread + mag) + f.ea;
            rc.et = err_bound(fabsf(rc.t0) + f.hb + spread + mag) + f.ea;
            rc.depth = f.depth;
            rc.k = k;
            buf[threadIdx.x].r = rc;
        }
    } else if (g - occ.n_rects < occ.n_spheres) {
        const int k = (int)(g - occ.n_rects);
        const FloatSph f = COPIES ? fs[k] : float_sphere(occ.spheres[k], occ.zscale);
        sc.dx0 = tcx - f.cx;
        sc.dy0 = tcy - f.cy;
        const float gx = fmaxf(fabsf(sc.dx0) - h, 0.0f), gy = fmaxf(fabsf(sc.dy0) - h, 0.0f);
        const float rr = f.r + kCullSlack;
        keep_s = gx * gx + gy * gy <= rr * rr;
        if (keep_s) {
            sc.r2f = f.r * f.r;
            const float far = fabsf(sc.dx0) + fabsf(sc.dy0) + 2.0f * h + f.r + f.ea;
            sc.e = err_bound(far * far) + 2.0f * far * f.ea;
            sc.dmin = f.dmin;
            sc.k = k;
            // tile centre - disc centre in float-float: (tc - cx_f) exactly
            // (TwoSum), then the dropped part of the centre
            float a, e;
            two_sum(tcx, -f.cx, a, e);
            two_sum(a, __fsub_rn(e, f.cxl), sc.dx0h, sc.dx0l);
            two_sum(tcy, -f.cy, a, e);
            two_sum(a, __fsub_rn(e, f.cyl), sc.dy0h, sc.dy0l);
            sc.r2h = f.r2h; sc.r2l = f.r2l; sc.ch = f.ch; sc.cl = f.cl;
            sc.cxa = fabsf(f.cx);
            sc.cya = fabsf(f.cy);
            sc.fast = fast && f.fast && sc.cxa <= 1e15f && sc.cya <= 1e15f;
            buf[threadIdx.x].s = sc;
        }
    }
    const unsigned br = __ballot_sync(0xffffffffu, keep_r), bs = __ballot_sync(0xffffffffu, keep_s);
    if (lane == 0) {
        sm.cnt_r[warp] = __popc(br);
        sm.cnt_s[warp] = __popc(bs);
    }
    __syncthreads();
    int off_r = 0, off_s = 0;
    nr = 0;
    ns = 0;
#pragma unroll
    for (int w = 0; w < kSmWarps; ++w) {
        const int cr = sm.cnt_r[w], cs = sm.cnt_s[w];
        off_r += w < warp ? cr : 0;
        off_s += w < warp ? cs : 0;
        nr += cr;
        ns += cs;
    }
    const unsigned below = (1u << lane) - 1u;
    if (keep_r)
        sm.idx[off_r + __popc(br & below)] = (int)threadIdx.x;
    if (keep_s)
        sm.idx[nr + off_s + __popc(bs & below)] = (int)threadIdx.x;
    __syncthreads();
}

// inv_zscale: 1 / zscale when zscale is a power of two (dividing by it is
// then the exact multiplication by its reciprocal), else 0.  COPIES: the
// CTA holds float copies of all occluders (neither kind has more than
// kFloatCopies); a compile-time choice, so that the culling holds no
// double-to-float conversions (slow FP64 pipe) when it reads the copies.
template <bool COPIES>
__global__ void __launch_bounds__(kSmThreads, 4) shadow_map_kernel(const rbsm_occluders occ, float *__restrict__ depth,
                                                                int width, int height, long long pitch,
                                                                double inv_zscale)
{
    // the next map's kernel (a programmatic dependent when the maps share no
    // memory) may take SMs as this one's CTAs finish
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ TileSmem sm;
    __shared__ FloatOcc fo[COPIES ? kFloatCopies : 1];
    __shared__ FloatSph fs[COPIES ? kFloatCopies : 1];
    if (COPIES) {
        for (int k = threadIdx.x; k < occ.n_rects; k += blockDim.x)
            fo[k] = float_rect(occ.rects[k]);
        for (int k = threadIdx.x; k < occ.n_spheres; k += blockDim.x)
            fs[k] = float_sphere(occ.spheres[k], occ.zscale);
        __syncthreads();
    }
    const FloatOcc *fop = fo;
    const FloatSph *fsp = fs;
    // the float-float cap depth needs 1 / zscale exact in float
    const bool fast = inv_zscale >= 7.888609052210118e-31 && inv_zscale <= 1.2676506002282294e30;   // 2^-100, 2^100
    const float invf = (float)inv_zscale;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    constexpr float h = 0.5f * (kTile - 1);
    // texel centre - tile centre, exact: ox for this thread's column, oy[p]
    // for its rows ty + 8 p
    const float ox = __fsub_rn(small_int_float(tx), h);
    float oys[4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
        oys[p] = __fsub_rn(small_int_float(ty + 8 * p), h);
    const long long n_all = (long long)occ.n_rects + occ.n_spheres;
    const long long pitch8 = pitch * 8;
    unsigned round = 0;                        // culling rounds so far (selects the candidate buffer)
    // the tile's column and row, stepped by the grid stride (no division per
    // tile), and the offset of this thread's first row in the map
    const int tiles_x = (width + kTile - 1) / kTile;
    const int tiles = tiles_x * ((height + kTile - 1) / kTile);     // <= 2^22
    int tcol = (int)blockIdx.x % tiles_x, trow = (int)blockIdx.x / tiles_x;
    const int step_col = (int)gridDim.x % tiles_x, step_row = (int)gridDim.x / tiles_x;
    const long long tile_rows = (long long)kTile * pitch;
    const long long step_rows = (long long)step_row * tile_rows;
    long long row0 = (long long)trow * tile_rows + (long long)ty * pitch;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int i0 = tcol * kTile, j0 = trow * kTile;
        float *out = depth + row0 + i0 + tx;
        tcol += step_col;
        trow += step_row;
        row0 += step_rows;
        if (tcol >= tiles_x) {
            tcol -= tiles_x;
            ++trow;
            row0 += tile_rows;
        }
        // tile centre (i0 + 0.5 + 15.5, j0 + 16), exact (< 2^23)
        const float tcx = small_int_float(i0 + kTile / 2), tcy = small_int_float(j0 + kTile / 2);
        const int i = i0 + tx;
        float best[4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
            best[p] = occ.ground;
        // occluders in rounds of kChunk: rectangles, then spheres, in index
        // order
        for (long long base = 0; base < n_all; base += kChunk) {
            int nr, ns;
            Cand *buf = sm.c[round & 1];
            ++round;
            cull_round<COPIES>(occ, fop, fsp, base, tcx, tcy, fast, sm, buf, nr, ns);
            for (int q = 0; q < nr; ++q) {
                const RectCand &r = buf[sm.idx[q]].r;
                const float sx = ox * r.uxf, tx_ = -ox * r.uyf;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float oy = oys[p];
                    const float sf = fabsf(r.s0 + (sx + oy * r.uyf));
                    const float tf = fabsf(r.t0 + (tx_ + oy * r.uxf));
                    if (sf > r.haf + r.es || tf > r.hbf + r.et || !(r.depth < best[p]))
                        continue;                      // surely outside, or it cannot lower the depth
                    bool in = sf < r.haf - r.es && tf < r.hbf - r.et;
                    if (!in)
                        in = rect_covers_exact(occ.rects + r.k, i, j0 + ty + 8 * p);     // near an edge
                    if (in)
                        best[p] = r.depth;
                }
            }
            for (int q = 0; q < ns; ++q) {
                const SphereCand &c = buf[sm.idx[nr + q]].s;
                const float dxf = c.dx0 + ox;
                const CapColumn col = cap_column(c, ox);
                // one copy of the cap code for the 4 rows (fewer registers):
                // the rows' depths rotate through best[0]
                float oy = oys[0];
#pragma unroll 1
                for (int p = 0; p < 4; ++p) {
                    const float dyf = c.dy0 + oy;
                    // skip when it cannot lower the depth, or surely outside the disc
                    if (c.dmin < best[0] && !(dxf * dxf + dyf * dyf > c.r2f + c.e)) {
                        float d = 0.0f;
                        const int cap = c.fast ? cap_fast(c, col, oy, invf, d) : -1;
                        if (cap < 0)
                            d = cap_depth_exact(occ.spheres + c.k, i, j0 + ty + 8 * p, inv_zscale, occ.zscale);
                        if (cap != 0 && d < best[0])
                            best[0] = d;
                    }
                    const float b = best[0];
                    best[0] = best[1];
                    best[1] = best[2];
                    best[2] = best[3];
                    best[3] = b;
                    oy = __fadd_rn(oy, 8.0f);              // exact
                }
            }
        }
        if (i < width) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (j0 + ty + 8 * p < height)
                    *out = best[p];
                out += pitch8;
            }
        }
    }
}

bool occluders_ok(const rbsm_occluders *occ)
{
    return occ && occ->n_rects >= 0 && occ->n_spheres >= 0 && (occ->n_rects == 0 || occ->rects) &&
           (occ->n_spheres == 0 || occ->spheres) && occ->zscale > 0.0 && occ->flags == 0;
}

// One map's launch; `overlap`: a programmatic dependent of the previous
// kernel on the stream (it does not wait for it).
int launch_map(const rbsm_occluders &occ, float *depth, int width, int height, long long pitch, bool overlap,
               cudaStream_t stream)
{
    const bool copies = occ.n_rects <= kFloatCopies && occ.n_spheres <= kFloatCopies;
    static KernelSetup setup_copies, setup_plain;
    auto kern = copies ? shadow_map_kernel<true> : shadow_map_kernel<false>;
    int occupancy = 0;
    int rc = (copies ? setup_copies : setup_plain).get(kern, kSmThreads, 0, &occupancy);
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
    const double inv = std::frexp(occ.zscale, &e2) == 0.5 ? std::ldexp(1.0, 1 - e2) : 0.0;
    cudaError_t e;
    if (overlap) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(kSmThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, occ, depth, width, height, pitch, inv);
    } else {
        kern<<<(unsigned)grid, kSmThreads, 0, stream>>>(occ, depth, width, height, pitch, inv);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}

bool spans_meet(uintptr_t a_lo, uintptr_t a_hi, uintptr_t b_lo, uintptr_t b_hi)
{
    return a_lo < b_hi && b_lo < a_hi;
}

}  // namespace
}  // namespace rbsm

extern "C" int rbsm_shadow_map(const rbsm_occluders *occ, float *depth, int32_t width, int32_t height,
                               int64_t pitch, void *stream)
{
    using namespace rbsm;
    if (!occluders_ok(occ) || !depth || width < 1 || width > RBSM_MAX_EXTENT || height < 1 ||
        height > RBSM_MAX_EXTENT || pitch < width)
        return RBSM_ERR_ARG;
    return launch_map(*occ, depth, width, height, pitch, false, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int rbsm_shadow_maps(const rbsm_occluders *occ, float *const *depth, int32_t n_maps, int32_t width,
                                int32_t height, int64_t pitch, void *stream)
{
    using namespace rbsm;
    if (!occ || !depth || n_maps < 1 || n_maps > RBSM_SHADOW_MAPS_MAX || width < 1 || width > RBSM_MAX_EXTENT ||
        height < 1 || height > RBSM_MAX_EXTENT || pitch < width)
        return RBSM_ERR_ARG;
    for (int k = 0; k < n_maps; ++k)
        if (!occluders_ok(occ + k) || !depth[k])
            return RBSM_ERR_ARG;
    // the maps' kernels may overlap when no map's memory meets another map's
    // or any occluder array
    const uintptr_t map_bytes = ((uintptr_t)pitch * (uintptr_t)(height - 1) + (uintptr_t)width) * sizeof(float);
    bool independent = n_maps > 1;
    for (int a = 0; a < n_maps && independent; ++a) {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(depth[a]), hi = lo + map_bytes;
        for (int b = 0; b < n_maps && independent; ++b) {
            const uintptr_t blo = reinterpret_cast<uintptr_t>(depth[b]);
            if (b != a && spans_meet(lo, hi, blo, blo + map_bytes))
                independent = false;
            const uintptr_t r = reinterpret_cast<uintptr_t>(occ[b].rects);
            const uintptr_t sp = reinterpret_cast<uintptr_t>(occ[b].spheres);
            if (occ[b].n_rects > 0 && spans_meet(lo, hi, r, r + (uintptr_t)occ[b].n_rects * sizeof(rbsm_rect)))
                independent = false;
            if (occ[b].n_spheres > 0 &&
                spans_meet(lo, hi, sp, sp + (uintptr_t)occ[b].n_spheres * sizeof(rbsm_sphere)))
                independent = false;
        }
    }
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int k = 0; k < n_maps; ++k) {
        const int rc = launch_map(occ[k], depth[k], width, height, pitch, independent && k > 0, s);
        if (rc != RBSM_OK)
            return rc;
    }
    return RBSM_OK;
}
