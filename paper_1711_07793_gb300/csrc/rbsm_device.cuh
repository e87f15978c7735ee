// Device-side steps of the RBSM per-fragment path for sm_103a.
//
// Per fragment: texel and in-texel offsets (float32, as the paper's GLSL),
// shadow test of the texel and of its four neighbours (Eq. 1, Eq. 2),
// discontinuity directions (Eqs. 3-4).  Fragments off the shadow edge are
// finished there (the plain shadow test, Listing 1).  Edge fragments walk the
// edge (Listing 3), normalise their position (Eq. 5) and take the optimized
// visibility (Listing 4 and/or Listing 5).
//
// Work unit: a warp tile of 128 consecutive fragments (below).  Edge
// fragments of a tile are compacted so that their long, data-dependent walks
// run on adjacent lanes instead of serialising all four fragments of a lane.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rbsm {

constexpr int kPerThread = 4;

struct MapDev {
    const float *depth;
    int32_t width;
    int32_t height;
    long long pitch;
    cudaTextureObject_t tex;     // 0 = none (plain loads)
};

// Nearest texel with clamp-to-edge addressing; read through the read-only
// (L1-cached) path because neighbouring fragments reuse the same texels.
__device__ __forceinline__ float texel(const MapDev &m, int i, int j)
{
    i = min(max(i, 0), m.width - 1);
    j = min(max(j, 0), m.height - 1);
    return __ldg(m.depth + (long long)j * m.pitch + i);
}

// Eq. 1: 0 (shadowed) when the stored blocker is nearer the light than the
// fragment, 1 otherwise.  No bias.
__device__ __forceinline__ int shadow_test(float pz, float zt)
{
    return pz > zt ? 0 : 1;
}

// Texel and in-texel offset of a texel-space position u along one axis:
// t = clamp(floor(u)), f = u - floor(u) (float32, as the paper's GLSL).
__device__ __forceinline__ void texel_of(float u, int size, int &t, float &f)
{
    float fu = floorf(u);
    f = __fsub_rn(u, fu);
    float c = fminf(fmaxf(fu, 0.0f), (float)(size - 1));
    t = (int)c;
}

// The same from a texture coordinate: u = x * size.
__device__ __forceinline__ void texel_coord(float x, int size, int &t, float &f)
{
    texel_of(__fmul_rn(x, (float)size), size, t, f);
}

// Listing 3 along one axis, both directions.  A texel of the walk continues
// the edge when it keeps the fragment's shadow-test result and shares a
// discontinuity direction with the fragment.  Along x only the +-y
// directions can be shared: the walk's texel has the same result as the
// texel it came from (so no shared direction back along the walk), and the
// fragment has no discontinuity in the walking direction (else the first
// step ends the walk).  Both facts hold with clamp-to-edge addressing too;
// along y the same holds with the axes swapped.  A walk returns +k for an
// end found at step k, -k for a texel that left the edge, -(max_dist+1) when
// all steps continued: rn for the walk towards lower indices, rp for the
// walk towards higher ones.
//
// The walks read three fixed lines of the map (the row or column of the
// fragment and its two neighbours).  `line` points at the first texel of
// the fragment's own line, `stride` is the distance between consecutive
// texels of a line, `pos`/`last` the fragment's index and the last index
// along it; each direction steps a pointer along the line and holds it at
// the border (clamp to edge).  The side lines that share a direction
// (use_a/use_b) lie da and db elements from the line; with kAdjacent (the
// walks along y) they are the columns i-1 and i+1, read at the immediate
// offsets -1 and +1.  A side is only read when the fragment has a
// discontinuity towards it, and at the map border the clamped neighbour is
// the texel itself and shows none, so a side that is read exists and the
// offsets never leave the map.  The two directions advance together and
// every load of a step (of both walks; a finished walk issues none) is in
// flight before the first test, so a step costs one memory latency.  Loads
// of later steps are not issued ahead: the extra, mostly wasted, requests
// cost more than the latency they hide.
template <bool kAdjacent>
__device__ __forceinline__ void walk_pair(const float *line, long long da, long long db, long long stride,
                                          int pos, int last, bool use_a, bool use_b, float pz, int s0,
                                          int max_dist, int &rn, int &rp)
{
    rn = 0;
    rp = 0;
    const float *pn = line + (long long)pos * stride;
    const float *pp = pn;
    const int room_n = pos, room_p = last - pos;
    const long long oa = kAdjacent ? -1 : da, ob = kAdjacent ? 1 : db;
    for (int k = 1; k <= max_dist; ++k) {
        const bool an = rn == 0, ap = rp == 0;
        if (k <= room_n)
            pn -= stride;
        if (k <= room_p)
            pp += stride;
        const float zcn = an ? __ldg(pn) : 0.0f;
        const float zan = an && use_a ? __ldg(pn + oa) : 0.0f;
        const float zbn = an && use_b ? __ldg(pn + ob) : 0.0f;
        const float zcp = ap ? __ldg(pp) : 0.0f;
        const float zap = ap && use_a ? __ldg(pp + oa) : 0.0f;
        const float zbp = ap && use_b ? __ldg(pp + ob) : 0.0f;
        if (an) {
            if (shadow_test(pz, zcn) != s0)
                rn = k;
            else if (!((use_a && shadow_test(pz, zan) != s0) || (use_b && shadow_test(pz, zbn) != s0)))
                rn = -k;
        }
        if (ap) {
            if (shadow_test(pz, zcp) != s0)
                rp = k;
            else if (!((use_a && shadow_test(pz, zap) != s0) || (use_b && shadow_test(pz, zbp) != s0)))
                rp = -k;
        }
        if (rn != 0 && rp != 0)
            return;
    }
    if (rn == 0)
        rn = -(max_dist + 1);
    if (rp == 0)
        rp = -(max_dist + 1);
}

// The walks along x from texel (i, j): rows j, j+1 (shared +y) and j-1
// (shared -y).
__device__ __forceinline__ void walks_x(const MapDev &m, int i, int j, float pz, int s0,
                                        bool up, bool down, int max_dist, int &rn, int &rp)
{
    const float *row = m.depth + (long long)j * m.pitch;
    const long long du = j < m.height - 1 ? m.pitch : 0, dd = j > 0 ? -m.pitch : 0;
    walk_pair<false>(row, du, dd, 1, i, m.width - 1, up, down, pz, s0, max_dist, rn, rp);
}

// The walks along y from texel (i, j): columns i, i-1 (shared left) and i+1
// (shared right).
__device__ __forceinline__ void walks_y(const MapDev &m, int i, int j, float pz, int s0,
                                        bool left, bool right, int max_dist, int &rn, int &rp)
{
    walk_pair<true>(m.depth + i, 0, 0, m.pitch, j, m.height - 1, left, right, pz, s0, max_dist, rn, rp);
}

// Walks through the map's texture view, S steps per iteration (S even).
// A 2x2 gather returns two consecutive texels of the walk's line and of one
// neighbouring line, so an iteration takes S steps of a direction with S/2
// gathers per side line in use (one side: S/2, both: S).  The texture
// clamps to the edge as the scalar walk clamps its indices, so every step
// reads the texels walk_pair reads; steps past an end or past max_dist are
// fetched but not tested.  Gather order: x = (lo col, hi row), y = (hi, hi),
// z = (hi, lo), w = (lo, lo); a gather at (X, Y) covers columns X-1, X and
// rows Y-1, Y.  Used by RPCF for k != 3, whose drains it speeds up (against
// the scalar walk stepping one pointer per direction: k = 1 / 7 at 128.4 /
// 11.1 against 124.1 / 10.9 Gfrag/s, k = 3 at 40.25 against 40.6); the
// batched kernel keeps the scalar walk (C5 0.351 vs 0.385 ms on 8 frames,
// C4 94 vs 107 us per frame, measured against the earlier scalar walk).

template <int S>
__device__ __forceinline__ void walk_steps(const float (&zl)[S], const float (&za)[S], const float (&zb)[S],
                                           bool use_a, bool use_b, float pz, int s0, int k, int max_dist, int &r)
{
#pragma unroll
    for (int t = 0; t < S; ++t) {
        if (r == 0 && k + t <= max_dist) {
            if (shadow_test(pz, zl[t]) != s0)
                r = k + t;
            else if (!((use_a && shadow_test(pz, za[t]) != s0) || (use_b && shadow_test(pz, zb[t]) != s0)))
                r = -(k + t);
        }
    }
}

// Along x from texel (i, j): line row j, sides rows j+1 (up) and j-1 (down).
template <int S>
__device__ __forceinline__ void walks_x_tex(const MapDev &m, int i, int j, float pz, int s0, bool up, bool down,
                                            int max_dist, int &rn, int &rp)
{
    rn = 0;
    rp = 0;
    const float fj = (float)j;
    const bool hi_pair = up || !down;      // the line from the rows j, j+1 gather unless only j-1 is in use
    for (int k = 1; k <= max_dist; k += S) {
        const bool on = rn == 0, op = rp == 0;
        float ln[S], la[S], lb[S], lp[S], pa[S], pb[S];
#pragma unroll
        for (int g = 0; g < S / 2; ++g) {
            // +x: columns i+k+2g (lo, step k+2g) and i+k+2g+1 (hi)
            const float xp = (float)(i + k + 2 * g + 1);
            float4 pu = make_float4(0.0f, 0.0f, 0.0f, 0.0f), pd = pu;
            if (op && hi_pair)
                pu = tex2Dgather<float4>(m.tex, xp, fj + 1.0f, 0);
            if (op && down)
                pd = tex2Dgather<float4>(m.tex, xp, fj, 0);
            lp[2 * g] = hi_pair ? pu.w : pd.x;
            lp[2 * g + 1] = hi_pair ? pu.z : pd.y;
            pa[2 * g] = pu.x;
            pa[2 * g + 1] = pu.y;
            pb[2 * g] = pd.w;
            pb[2 * g + 1] = pd.z;
            // -x: columns i-k-2g (hi, step k+2g) and i-k-2g-1 (lo)
            const float xn = (float)(i - k - 2 * g);
            float4 nu = make_float4(0.0f, 0.0f, 0.0f, 0.0f), nd = nu;
            if (on && hi_pair)
                nu = tex2Dgather<float4>(m.tex, xn, fj + 1.0f, 0);
            if (on && down)
                nd = tex2Dgather<float4>(m.tex, xn, fj, 0);
            ln[2 * g] = hi_pair ? nu.z : nd.y;
            ln[2 * g + 1] = hi_pair ? nu.w : nd.x;
            la[2 * g] = nu.y;
            la[2 * g + 1] = nu.x;
            lb[2 * g] = nd.z;
            lb[2 * g + 1] = nd.w;
        }
        walk_steps<S>(ln, la, lb, up, down, pz, s0, k, max_dist, rn);
        walk_steps<S>(lp, pa, pb, up, down, pz, s0, k, max_dist, rp);
        if (rn != 0 && rp != 0)
            break;
    }
    rn = rn == 0 ? -(max_dist + 1) : rn;
    rp = rp == 0 ? -(max_dist + 1) : rp;
}

// Along y from texel (i, j): line column i, sides columns i-1 (left) and
// i+1 (right).
template <int S>
__device__ __forceinline__ void walks_y_tex(const MapDev &m, int i, int j, float pz, int s0, bool left, bool right,
                                            int max_dist, int &rn, int &rp)
{
    rn = 0;
    rp = 0;
    const float fi = (float)i;
    const bool lo_pair = left || !right;   // the line from the columns i-1, i gather unless only i+1 is in use
    for (int k = 1; k <= max_dist; k += S) {
        const bool on = rn == 0, op = rp == 0;
        float ln[S], la[S], lb[S], lp[S], pa[S], pb[S];
#pragma unroll
        for (int g = 0; g < S / 2; ++g) {
            // +y: rows j+k+2g (lo, step k+2g) and j+k+2g+1 (hi)
            const float yp = (float)(j + k + 2 * g + 1);
            float4 pl = make_float4(0.0f, 0.0f, 0.0f, 0.0f), pr = pl;
            if (op && lo_pair)
                pl = tex2Dgather<float4>(m.tex, fi, yp, 0);
            if (op && right)
                pr = tex2Dgather<float4>(m.tex, fi + 1.0f, yp, 0);
            lp[2 * g] = lo_pair ? pl.z : pr.w;
            lp[2 * g + 1] = lo_pair ? pl.y : pr.x;
            pa[2 * g] = pl.w;
            pa[2 * g + 1] = pl.x;
            pb[2 * g] = pr.z;
            pb[2 * g + 1] = pr.y;
            // -y: rows j-k-2g (hi, step k+2g) and j-k-2g-1 (lo)
            const float yn = (float)(j - k - 2 * g);
            float4 nl = make_float4(0.0f, 0.0f, 0.0f, 0.0f), nr = nl;
            if (on && lo_pair)
                nl = tex2Dgather<float4>(m.tex, fi, yn, 0);
            if (on && right)
                nr = tex2Dgather<float4>(m.tex, fi + 1.0f, yn, 0);
            ln[2 * g] = lo_pair ? nl.y : nr.x;
            ln[2 * g + 1] = lo_pair ? nl.z : nr.w;
            la[2 * g] = nl.x;
            la[2 * g + 1] = nl.w;
            lb[2 * g] = nr.y;
            lb[2 * g + 1] = nr.z;
        }
        walk_steps<S>(ln, la, lb, left, right, pz, s0, k, max_dist, rn);
        walk_steps<S>(lp, pa, pb, left, right, pz, s0, k, max_dist, rp);
        if (rn != 0 && rp != 0)
            break;
    }
    rn = rn == 0 ? -(max_dist + 1) : rn;
    rp = rp == 0 ? -(max_dist + 1) : rp;
}

// Eq. 5 and the normalisation along one axis: the position of the fragment
// measured from the end that was found, over the length of the aliased edge
// along that axis (|r_neg| + |r_pos| - 1 texels).  With no end found the
// position is 1.  The both-ends position is never read by Listings 4 and 5.
__device__ __forceinline__ float axis_position(int r_neg, int r_pos, float f)
{
    int len = abs(r_neg) + abs(r_pos) - 1;
    if (r_neg > 0 && r_pos <= 0)
        return __fdiv_rn(__fadd_rn((float)(r_neg - 1), f), (float)len);
    if (r_pos > 0 && r_neg <= 0)
        return __fdiv_rn(__fadd_rn((float)(r_pos - 1), __fsub_rn(1.0f, f)), (float)len);
    return 1.0f;
}

// Listing 4 (§4.1).  dx3/dy3: edges on both sides of the axis (d == 0.75);
// ex/ey: ends found along each axis (Eq. 5 code + 1).
__device__ __forceinline__ float silhouette(bool dx3, bool dy3, int ex, int ey, float nx, float ny)
{
    if (dx3 || dy3)
        return 0.0f;                        // short U / O
    if (ex == 2 || ey == 2)
        return 0.0f;                        // long U / O
    if (ex == 0 || ey == 0)
        return 1.0f;                        // I
    return ny < __fsub_rn(1.0f, nx) ? 0.0f : 1.0f;   // L: step(1 - nx, ny)
}

// Listing 5 (§4.2); dz = 1 - s.  The sign factor is +-1, applied as an
// exact negation.
__device__ __forceinline__ float filter(bool dx3, bool dy3, int dz, int ex, int ey, float nx, float ny)
{
    float z = (float)dz;
    float sx = dz ? -nx : nx;
    float sy = dz ? -ny : ny;
    if (dx3 && dy3)
        return z;                           // short O
    if (ex == 2 && ey == 2)
        return z;                           // long O
    if (ex == 2)
        return __fadd_rn(z, sy);            // U open along y
    if (ey == 2)
        return __fadd_rn(z, sx);            // U open along x
    if (ex == 0 || ey == 0)
        return 1.0f - z;                    // I
    float v = __fadd_rn(__fadd_rn(z, sy), sx);   // L: clamp(v, 0, 1)
    v = v < 0.0f ? 0.0f : v;                      // comparisons keep a NaN a NaN
    return v > 1.0f ? 1.0f : v;
}

// Features of the learned surrogate (this project's addition; not in the paper).
// 5x5 shadow-test pattern and nearest blocker depth around texel (i, j)
// (clamp to edge): bit (dy+2)*5 + (dx+2) is set when texel (i+dx, j+dy) is
// lit for depth pz.
__device__ __forceinline__ void window5(const MapDev &m, int i, int j, float pz, uint32_t &bits, float &zmin)
{
    bits = 0;
    zmin = texel(m, i, j);
    int cols[5];
#pragma unroll
    for (int d = 0; d < 5; ++d)
        cols[d] = min(max(i + d - 2, 0), m.width - 1);
#pragma unroll
    for (int dy = 0; dy < 5; ++dy) {
        const float *row = m.depth + (long long)min(max(j + dy - 2, 0), m.height - 1) * m.pitch;
#pragma unroll
        for (int dx = 0; dx < 5; ++dx) {
            const float zt = __ldg(row + cols[dx]);
            bits |= (uint32_t)shadow_test(pz, zt) << (dy * 5 + dx);
            zmin = fminf(zmin, zt);
        }
    }
}

__device__ __forceinline__ void fragment_features(const MapDev &m, float x, float y, float pz, uint32_t &bits,
                                                  float &fx, float &fy, float &gap)
{
    int i, j;
    texel_coord(x, m.width, i, fx);
    texel_coord(y, m.height, j, fy);
    float zmin;
    window5(m, i, j, pz, bits, zmin);
    gap = __fsub_rn(pz, zmin);
}

// Whether the four Listing 3 walks from the fragment's texel stop inside its
// 5x5 window, read from the window's shadow-test pattern (bit (dy+2)*5 +
// (dx+2): texel (i+dx, j+dy) lit).  A walk along x goes on past step k when
// texel (k, 0) has the fragment's test and shares a discontinuity
// direction with the fragment's texel; along a continuing walk only the
// perpendicular directions can be shared (the +-y neighbours of (k, 0)
// against those of (0, 0)).  Steps 1 and 2 read only window texels, so when
// no walk goes on past step 2 (or max_dist <= 2) the exact answer is a
// function of the pattern and the in-texel offsets alone; otherwise it
// depends on texels the window does not hold.
__device__ __forceinline__ bool walks_inside_window(uint32_t pattern, int max_dist)
{
    if (max_dist <= 2)
        return true;
    const uint32_t s0 = (pattern >> 12) & 1u;
    // d[k] = bit k of "texel differs from the fragment's test"
    const uint32_t d = pattern ^ (s0 ? 0x1FFFFFFu : 0u);
    auto diff = [&](int dx, int dy) { return (d >> ((dy + 2) * 5 + (dx + 2))) & 1u; };
    const uint32_t up0 = diff(0, 1), dn0 = diff(0, -1), lf0 = diff(-1, 0), rt0 = diff(1, 0);
    auto goes_on_x = [&](int dx) { return !diff(dx, 0) && ((up0 & diff(dx, 1)) | (dn0 & diff(dx, -1))); };
    auto goes_on_y = [&](int dy) { return !diff(0, dy) && ((lf0 & diff(-1, dy)) | (rt0 & diff(1, dy))); };
    return !(goes_on_x(1) && goes_on_x(2)) && !(goes_on_x(-1) && goes_on_x(-2)) &&
           !(goes_on_y(1) && goes_on_y(2)) && !(goes_on_y(-1) && goes_on_y(-2));
}

// Result of one fragment.
struct FragResult {
    float sil;
    float fil;
    uint16_t code;
};

// Steps 1-2 from the five depths of the texel and its neighbours.
// (The tests stay predicates: a neighbour's discontinuity is its test
// differing from the centre's, and the answer is selected, not converted.)
template <int MODE, bool CODES>
__device__ __forceinline__ bool classify_from(float pz, float zc, float zl, float zr, float zu, float zd,
                                              FragResult &r, uint32_t &bits)
{
    const bool shadowed = pz > zc;             // Eq. 1: s0 = 0
    if (MODE == 1 && !CODES && shadowed) {
        r.sil = 0.0f;
        r.code = 0;
        bits = 0;
        return false;
    }
    const uint32_t dl = (pz > zl) != shadowed;
    const uint32_t dr = (pz > zr) != shadowed;
    const uint32_t du = (pz > zu) != shadowed;
    const uint32_t dd = (pz > zd) != shadowed;
    const uint32_t d4 = dl | (dr << 1) | (du << 2) | (dd << 3);
    bits = (shadowed ? 0u : 1u) | (d4 << 1);
    r.code = (uint16_t)(d4 | (shadowed ? 16u : 0u));
    const float sv = shadowed ? 0.0f : 1.0f;
    r.sil = sv;
    r.fil = sv;
    const bool edge = d4 != 0;
    if (MODE == 1)
        return edge && !shadowed;
    return edge;
}

// Steps 1-2 for one fragment: texel, shadow test, four-neighbourhood.
// Returns true when the fragment needs the edge walk for this mode; packs
// s0 and the four directions into `bits` (bit 0 = s0, bits 1-4 = left,
// right, +y, -y).  Clamp-to-edge is applied branch-free: a neighbour
// outside the map is the centre texel itself, so the five loads of a
// fragment (and of the other fragments of the lane) can all be in flight at
// once.
template <int MODE, bool CODES>
__device__ __forceinline__ bool classify_uv(const MapDev &m, float u, float v, float pz,
                                            FragResult &r, uint32_t &bits)
{
    if (m.tex) {
        // Texel coordinates in float (clamp(floor(u)) is an integer-valued
        // float, exact below 2^24), then two 2x2 gathers (point sampling,
        // clamp to edge, unnormalised coordinates; the footprint of a gather
        // at (u, v) is columns u-1, u and rows v-1, v): at (i, j) columns
        // i-1..i, rows j-1..j; at (i+1, j+1) columns i..i+1, rows j..j+1.
        // Gather order: x = (lo col, hi row), y = (hi, hi), z = (hi, lo),
        // w = (lo, lo).
        const float ci = fminf(fmaxf(floorf(u), 0.0f), (float)(m.width - 1));
        const float cj = fminf(fmaxf(floorf(v), 0.0f), (float)(m.height - 1));
        const float4 a = tex2Dgather<float4>(m.tex, ci, cj, 0);
        const float4 b = tex2Dgather<float4>(m.tex, ci + 1.0f, cj + 1.0f, 0);
        return classify_from<MODE, CODES>(pz, a.y, a.x, b.z, b.x, a.z, r, bits);
    }
    int i, j;
    float fx, fy;
    texel_of(u, m.width, i, fx);
    texel_of(v, m.height, j, fy);
    const float *c = m.depth + (long long)j * m.pitch + i;
    const float zc = __ldg(c);
    // Listing 1: in silhouette recovery a shadowed fragment stays shadowed and
    // needs no neighbourhood (unless codes are requested).
    if (MODE == 1 && !CODES && pz > zc) {
        r.sil = 0.0f;
        r.code = 0;
        bits = 0;
        return false;
    }
    const long long up = j < m.height - 1 ? m.pitch : 0;
    const long long dn = j > 0 ? m.pitch : 0;
    const int lf = i > 0 ? 1 : 0;
    const int rt = i < m.width - 1 ? 1 : 0;
    return classify_from<MODE, CODES>(pz, zc, __ldg(c - lf), __ldg(c + rt), __ldg(c + up), __ldg(c - dn), r, bits);
}

// Steps 1-2 from a texture coordinate (u = x * W, v = y * H in float32).
template <int MODE, bool CODES>
__device__ __forceinline__ bool classify(const MapDev &m, float x, float y, float pz,
                                         FragResult &r, uint32_t &bits)
{
    return classify_uv<MODE, CODES>(m, __fmul_rn(x, (float)m.width), __fmul_rn(y, (float)m.height), pz, r, bits);
}

// Steps 3-4 for one edge fragment at texel-space position (u, v)
// (recomputes its texel).  TEX_STEPS > 0: walk through the map's texture
// view (when it has one), TEX_STEPS steps per iteration.
template <int MODE, int TEX_STEPS = 0>
__device__ __forceinline__ void resolve_edge_uv(const MapDev &m, float u, float v, float pz,
                                                uint32_t bits, int max_dist, FragResult &r)
{
    int i, j;
    float fx, fy;
    texel_of(u, m.width, i, fx);
    texel_of(v, m.height, j, fy);
    int s0 = bits & 1;
    bool dl = (bits >> 1) & 1, dr = (bits >> 2) & 1, du = (bits >> 3) & 1, dd = (bits >> 4) & 1;
    // computeFragmentDistanceToSE: the four walks -x, +x, -y, +y
    int rxn, rxp, ryn, ryp;
    bool done = false;
    if constexpr (TEX_STEPS > 0) {
        if (m.tex) {
            walks_x_tex<TEX_STEPS>(m, i, j, pz, s0, du, dd, max_dist, rxn, rxp);
            walks_y_tex<TEX_STEPS>(m, i, j, pz, s0, dl, dr, max_dist, ryn, ryp);
            done = true;
        }
    }
    if (!done) {
        walks_x(m, i, j, pz, s0, du, dd, max_dist, rxn, rxp);
        walks_y(m, i, j, pz, s0, dl, dr, max_dist, ryn, ryp);
    }
    int ex = (rxn > 0) + (rxp > 0);
    int ey = (ryn > 0) + (ryp > 0);
    float nx = axis_position(rxn, rxp, fx);
    float ny = axis_position(ryn, ryp, fy);
    bool dx3 = dl && dr, dy3 = du && dd;
    r.code = (uint16_t)(r.code | (ex << 5) | (ey << 7) | (1 << 9));
    if (MODE & 1)
        r.sil = s0 ? silhouette(dx3, dy3, ex, ey, nx, ny) : 0.0f;
    if (MODE & 2)
        r.fil = filter(dx3, dy3, 1 - s0, ex, ey, nx, ny);
}

// Steps 3-4 from a texture coordinate.
template <int MODE>
__device__ __forceinline__ void resolve_edge(const MapDev &m, float x, float y, float pz,
                                             uint32_t bits, int max_dist, FragResult &r)
{
    resolve_edge_uv<MODE>(m, __fmul_rn(x, (float)m.width), __fmul_rn(y, (float)m.height), pz, bits, max_dist, r);
}

// ------------------------------------------------------------ warp tiles --
//
// A warp owns a tile of kWarpTile = 32 lanes x 4 consecutive fragments.  Warps
// never wait for each other (no CTA barrier).  Per tile a warp classifies its
// fragments, stores every answer at once (edge fragments get a provisional
// value) and appends its edge fragments to its own shared-memory queue.  The
// queue is drained 32 entries at a time, so the walks run with all 32 lanes
// busy, and the drained answers overwrite the provisional ones (still in L2).
// While a warp works on one tile, the copies of its next tile's coordinates
// into the warp's shared-memory buffer are already in flight (cp.async;
// `stage_tile` / `fetch_tile`; the depth-buffer kernel keeps its next tile's
// depths in registers, a quarter of the bytes).

constexpr int kWarpTile = 32 * kPerThread;   // 128 fragments
constexpr int kQueueCap = kWarpTile + 32;    // < 32 left over + one tile

// One deferred edge fragment (8 bytes): which fragment, and what its
// classification found.  The drain reads the fragment's x, y, z again (edge
// fragments are a few percent of the stream, so keeping the queue small and
// the shared memory free for the L1 cache pays more).
struct EdgeEntry {
    uint32_t idx;            // fragment index within the job (fragment sets hold < 2^31)
    uint32_t bits_job;       // s0 | d4 << 1 (5 bits) | job << 8
};

struct WarpQueue {
    EdgeEntry q[kQueueCap];
};

// Coordinates of one warp tile held by a lane (4 fragments).
struct LaneCoords {
    float x[kPerThread], y[kPerThread], z[kPerThread];
};

// Where a warp tile lives: fragments [first, first + count) of a job.
struct WarpTileIO {
    const float *x, *y, *z;
    float *sil, *fil;
    uint16_t *codes;
    long long first;
    int count;               // 1..kWarpTile
    int job;
    bool vec;                // count == kWarpTile and every plane 16-byte aligned
};

// A job as the deferred answers need it: its map, its fragments, its outputs.
struct JobOut {
    MapDev map;
    const float *x, *y, *z;
    float *sil, *fil;
    uint16_t *codes;
    int mode;
};

// Issue the loads of a warp tile.  Vector path: lane l owns fragments
// 4l..4l+3 (one 16-byte load per plane).  Scalar path: lane l owns
// fragments l, l+32, l+64, l+96 (coalesced 4-byte loads).
__device__ __forceinline__ void load_tile(const WarpTileIO &t, unsigned lane, LaneCoords &c)
{
    if (t.vec) {
        const float4 vx = __ldcs(reinterpret_cast<const float4 *>(t.x + t.first) + lane);
        const float4 vy = __ldcs(reinterpret_cast<const float4 *>(t.y + t.first) + lane);
        const float4 vz = __ldcs(reinterpret_cast<const float4 *>(t.z + t.first) + lane);
        c.x[0] = vx.x; c.x[1] = vx.y; c.x[2] = vx.z; c.x[3] = vx.w;
        c.y[0] = vy.x; c.y[1] = vy.y; c.y[2] = vy.z; c.y[3] = vy.w;
        c.z[0] = vz.x; c.z[1] = vz.y; c.z[2] = vz.z; c.z[3] = vz.w;
    } else {
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            const int s = (int)lane + 32 * e;
            const bool ok = s < t.count;
            c.x[e] = ok ? __ldcs(t.x + t.first + s) : 0.0f;
            c.y[e] = ok ? __ldcs(t.y + t.first + s) : 0.0f;
            c.z[e] = ok ? __ldcs(t.z + t.first + s) : 0.0f;
        }
    }
}

// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only).
__device__ __forceinline__ void copy_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// Start the copies of a tile's coordinates into the warp's buffer (vector
// tiles; others are loaded directly when they come up).  Each lane copies
// and later reads only its own float4 of each plane.
__device__ __forceinline__ void stage_tile(const WarpTileIO &t, unsigned lane, float4 (&buf)[3][32])
{
    if (t.vec) {
        copy_async16(&buf[0][lane], reinterpret_cast<const float4 *>(t.x + t.first) + lane);
        copy_async16(&buf[1][lane], reinterpret_cast<const float4 *>(t.y + t.first) + lane);
        copy_async16(&buf[2][lane], reinterpret_cast<const float4 *>(t.z + t.first) + lane);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The staged tile's coordinates in registers (waits for the copies).
__device__ __forceinline__ void fetch_tile(const WarpTileIO &t, unsigned lane, const float4 (&buf)[3][32],
                                           LaneCoords &c)
{
    if (t.vec) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        const float4 vx = buf[0][lane], vy = buf[1][lane], vz = buf[2][lane];
        c.x[0] = vx.x; c.x[1] = vx.y; c.x[2] = vx.z; c.x[3] = vx.w;
        c.y[0] = vy.x; c.y[1] = vy.y; c.y[2] = vy.z; c.y[3] = vy.w;
        c.z[0] = vz.x; c.z[1] = vz.y; c.z[2] = vz.z; c.z[3] = vz.w;
    } else {
        load_tile(t, lane, c);
    }
}

// The same with lane l holding fragments l, l + 32, l + 64, l + 96 for
// vector tiles too (the scalar tiles' order): the staged planes are read
// back transposed, so a warp's lanes hold consecutive fragments at each
// element.  Consecutive fragments fall on the same or neighbouring texels,
// so one gather instruction of the warp touches a few cache lines instead
// of a strip four fragments apart per lane.  The buffer is read by other
// lanes than the one that copied it: a warp barrier after the wait, and
// another before the buffer is refilled.
__device__ __forceinline__ void fetch_tile_strided(const WarpTileIO &t, unsigned lane, const float4 (&buf)[3][32],
                                                   LaneCoords &c)
{
    if (t.vec) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        const float *bx = reinterpret_cast<const float *>(buf[0]);
        const float *by = reinterpret_cast<const float *>(buf[1]);
        const float *bz = reinterpret_cast<const float *>(buf[2]);
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            c.x[e] = bx[lane + 32 * e];
            c.y[e] = by[lane + 32 * e];
            c.z[e] = bz[lane + 32 * e];
        }
        __syncwarp();
    } else {
        load_tile(t, lane, c);
    }
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Walk, normalise and answer one deferred edge fragment; write its answers.
// FIXED_MODE 1..3 when every job of the launch has that mode, 0 to read it
// from the job.
template <int FIXED_MODE = 0>
__device__ __forceinline__ void resolve_entry(const JobOut &o, const EdgeEntry &q, int max_dist)
{
    const uint32_t bits = q.bits_job & 0x1fu;
    const uint32_t d4 = bits >> 1, s0 = bits & 1u;
    FragResult r{0.0f, 0.0f, (uint16_t)(d4 | ((1u - s0) << 4))};
    const float x = __ldg(o.x + q.idx), y = __ldg(o.y + q.idx), z = __ldg(o.z + q.idx);
    switch (FIXED_MODE ? FIXED_MODE : o.mode) {
    case 1: resolve_edge<1>(o.map, x, y, z, bits, max_dist, r); break;
    case 2: resolve_edge<2>(o.map, x, y, z, bits, max_dist, r); break;
    default: resolve_edge<3>(o.map, x, y, z, bits, max_dist, r); break;
    }
    if (o.mode & 1) o.sil[q.idx] = r.sil;
    if (o.mode & 2) o.fil[q.idx] = r.fil;
    if (o.codes) o.codes[q.idx] = r.code;
}

// Drain full rounds of 32 queued edge fragments (or everything when
// `all`).  `jobs(job)` returns the JobOut of a job.  The count is uniform
// across the warp.
template <typename Jobs, int FIXED_MODE = 0>
__device__ __forceinline__ void drain_queue(const Jobs &jobs, WarpQueue &wq, int &count, int max_dist, bool all)
{
    const unsigned lane = lane_id();
    while (count >= 32 || (all && count > 0)) {
        __syncwarp();                      // queue entries and provisional stores are visible
        const int base = count >= 32 ? count - 32 : 0;
        const int k = base + (int)lane;
        if (k < count) {
            const EdgeEntry q = wq.q[k];
            resolve_entry<FIXED_MODE>(jobs((int)(q.bits_job >> 8)), q, max_dist);
        }
        __syncwarp();                      // entries read before they are overwritten
        count = base;
    }
}

// Classify one warp tile whose coordinates the lane holds, store its answers
// (provisional for edge fragments) and queue its edge fragments.
template <int MODE, bool CODES>
__device__ __forceinline__ void classify_warp_tile(const MapDev &m, const WarpTileIO &t, const LaneCoords &c,
                                                   WarpQueue &wq, int &count)
{
    const unsigned lane = lane_id();
    const unsigned below = (1u << lane) - 1u;
    FragResult r[kPerThread];
    uint32_t bits[kPerThread];
    bool edge[kPerThread];
    // classify the lane's four fragments first (no warp-wide step in between,
    // so all their texel loads are issued back to back) ...
    if (t.vec) {
#pragma unroll
        for (int e = 0; e < kPerThread; ++e)
            edge[e] = classify<MODE, CODES>(m, c.x[e], c.y[e], c.z[e], r[e], bits[e]);
    } else {
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            r[e] = FragResult{0.0f, 0.0f, 0};
            bits[e] = 0;
            edge[e] = false;
            if ((int)lane + 32 * e < t.count)
                edge[e] = classify<MODE, CODES>(m, c.x[e], c.y[e], c.z[e], r[e], bits[e]);
        }
    }
    // ... then queue the edge fragments, one ballot per element
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
        const int s = t.vec ? (int)(kPerThread * lane) + e : (int)lane + 32 * e;
        const unsigned mask = __ballot_sync(0xffffffffu, edge[e]);
        if (edge[e]) {
            wq.q[count + __popc(mask & below)] =
                EdgeEntry{(uint32_t)(t.first + s), bits[e] | ((uint32_t)t.job << 8)};
        }
        count += __popc(mask);
    }
    if (t.vec) {
        if (MODE & 1)
            __stcg(reinterpret_cast<float4 *>(t.sil + t.first) + lane,
                   make_float4(r[0].sil, r[1].sil, r[2].sil, r[3].sil));
        if (MODE & 2)
            __stcg(reinterpret_cast<float4 *>(t.fil + t.first) + lane,
                   make_float4(r[0].fil, r[1].fil, r[2].fil, r[3].fil));
        if (CODES) {
            const uint2 cc = make_uint2((uint32_t)r[0].code | ((uint32_t)r[1].code << 16),
                                        (uint32_t)r[2].code | ((uint32_t)r[3].code << 16));
            __stcg(reinterpret_cast<uint2 *>(t.codes + t.first) + lane, cc);
        }
    } else {
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            const int s = (int)lane + 32 * e;
            if (s >= t.count)
                continue;
            const long long g = t.first + s;
            if (MODE & 1) t.sil[g] = r[e].sil;
            if (MODE & 2) t.fil[g] = r[e].fil;
            if (CODES) t.codes[g] = r[e].code;
        }
    }
}

// Dispatch on the runtime mode / codes pair of a job.
__device__ __forceinline__ void classify_warp_tile_rt(int mode, bool codes, const MapDev &m, const WarpTileIO &t,
                                                      const LaneCoords &c, WarpQueue &wq, int &count)
{
    switch (mode * 2 + (codes ? 1 : 0)) {
    case 2: classify_warp_tile<1, false>(m, t, c, wq, count); break;
    case 3: classify_warp_tile<1, true>(m, t, c, wq, count); break;
    case 4: classify_warp_tile<2, false>(m, t, c, wq, count); break;
    case 5: classify_warp_tile<2, true>(m, t, c, wq, count); break;
    case 6: classify_warp_tile<3, false>(m, t, c, wq, count); break;
    default: classify_warp_tile<3, true>(m, t, c, wq, count); break;
    }
}

}  // namespace rbsm
