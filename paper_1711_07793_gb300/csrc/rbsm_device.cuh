// Device-side steps of the RBSM per-fragment path for sm_103a.
//
// One CTA owns a tile of kTile consecutive fragments at a time:
//   1. load the tile's x/y/z planes with 16-byte vector loads (or coalesced
//      scalar loads for unaligned planes) into shared memory and registers;
//   2. classify every fragment: shadow test of its texel (Eq. 1) and of its
//      four neighbours, discontinuity directions (Eqs. 2-4).  Fragments off
//      the shadow edge are finished here (plain shadow test, Listing 1);
//      edge fragments are appended to a per-CTA queue with one warp-aggregated
//      atomic per warp;
//   3. the whole CTA drains the queue with converged lanes: the four edge
//      walks (Listing 3), the normalisation (Eq. 5) and the optimized
//      visibility (Listing 4 and/or Listing 5);
//   4. store the tile's answers with vector stores.
// Compacting edge fragments keeps their long, data-dependent walks from
// idling the 31 other lanes of a warp whose fragments are all off the edge.
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

// Texel coordinate and in-texel offset along one axis, float32 as the
// paper's GLSL: u = x * size, t = clamp(floor(u)), f = u - floor(u).
__device__ __forceinline__ void texel_coord(float x, int size, int &t, float &f)
{
    float u = __fmul_rn(x, (float)size);
    float fu = floorf(u);
    f = __fsub_rn(u, fu);
    float c = fminf(fmaxf(fu, 0.0f), (float)(size - 1));
    t = (int)c;
}

// Listing 3 along x.  A texel of the walk continues the edge when it keeps
// the fragment's shadow-test result and shares a discontinuity direction
// with the fragment.  Along x only the +-y directions can be shared: the
// walk's texel has the same result as the texel it came from (so no shared
// direction back along the walk), and the fragment has no discontinuity in
// the walking direction (else the first step ends the walk).  Returns +k for
// an end found at step k, -k for a texel that left the edge, -(max_dist+1)
// when all steps continued.
__device__ __forceinline__ int walk_x(const MapDev &m, int i, int j, float pz, int s0,
                                      bool up, bool down, int di, int max_dist)
{
    for (int k = 1; k <= max_dist; ++k) {
        int c = i + k * di;
        if (shadow_test(pz, texel(m, c, j)) != s0)
            return k;
        bool keep = (up && shadow_test(pz, texel(m, c, j + 1)) != s0) ||
                    (down && shadow_test(pz, texel(m, c, j - 1)) != s0);
        if (!keep)
            return -k;
    }
    return -(max_dist + 1);
}

// Listing 3 along y (only the left/right directions can be shared).
__device__ __forceinline__ int walk_y(const MapDev &m, int i, int j, float pz, int s0,
                                      bool left, bool right, int dj, int max_dist)
{
    for (int k = 1; k <= max_dist; ++k) {
        int r = j + k * dj;
        if (shadow_test(pz, texel(m, i, r)) != s0)
            return k;
        bool keep = (left && shadow_test(pz, texel(m, i - 1, r)) != s0) ||
                    (right && shadow_test(pz, texel(m, i + 1, r)) != s0);
        if (!keep)
            return -k;
    }
    return -(max_dist + 1);
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

// Result of one fragment.
struct FragResult {
    float sil;
    float fil;
    uint16_t code;
};

// Steps 1-2 for one fragment: texel, shadow test, four-neighbourhood.
// Returns true when the fragment needs the edge walk for this mode; packs
// s0 and the four directions into `bits` (bit 0 = s0, bits 1-4 = left,
// right, +y, -y).
template <int MODE, bool CODES>
__device__ __forceinline__ bool classify(const MapDev &m, float x, float y, float pz,
                                         FragResult &r, uint32_t &bits)
{
    int i, j;
    float fx, fy;
    texel_coord(x, m.width, i, fx);
    texel_coord(y, m.height, j, fy);
    int s0 = shadow_test(pz, texel(m, i, j));
    // Listing 1: in silhouette recovery a shadowed fragment stays shadowed and
    // needs no neighbourhood (unless codes are requested).
    if (MODE == 1 && !CODES && s0 == 0) {
        r.sil = 0.0f;
        r.code = 0;
        bits = 0;
        return false;
    }
    int dl = shadow_test(pz, texel(m, i - 1, j)) != s0;
    int dr = shadow_test(pz, texel(m, i + 1, j)) != s0;
    int du = shadow_test(pz, texel(m, i, j + 1)) != s0;
    int dd = shadow_test(pz, texel(m, i, j - 1)) != s0;
    uint32_t d4 = dl | (dr << 1) | (du << 2) | (dd << 3);
    bits = (uint32_t)s0 | (d4 << 1);
    r.code = (uint16_t)(d4 | ((1 - s0) << 4));
    float s = (float)s0;
    r.sil = (MODE & 1) ? ((s0 == 0) ? 0.0f : s) : 0.0f;
    r.fil = s;
    bool edge = d4 != 0;
    if (MODE == 1)
        return edge && s0 == 1;
    return edge;
}

// Steps 3-4 for one edge fragment (recomputes its texel from x, y).
template <int MODE>
__device__ __forceinline__ void resolve_edge(const MapDev &m, float x, float y, float pz,
                                             uint32_t bits, int max_dist, FragResult &r)
{
    int i, j;
    float fx, fy;
    texel_coord(x, m.width, i, fx);
    texel_coord(y, m.height, j, fy);
    int s0 = bits & 1;
    bool dl = (bits >> 1) & 1, dr = (bits >> 2) & 1, du = (bits >> 3) & 1, dd = (bits >> 4) & 1;
    // computeFragmentDistanceToSE: the four walks -x, +x, -y, +y
    int rxn = walk_x(m, i, j, pz, s0, du, dd, -1, max_dist);
    int rxp = walk_x(m, i, j, pz, s0, du, dd, +1, max_dist);
    int ryn = walk_y(m, i, j, pz, s0, dl, dr, -1, max_dist);
    int ryp = walk_y(m, i, j, pz, s0, dl, dr, +1, max_dist);
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

// Shared memory of one CTA for a tile of kThreads * kPerThread fragments.
template <int kThreads>
struct TileSmem {
    static constexpr int kTile = kThreads * kPerThread;
    float x[kTile];
    float y[kTile];
    float z[kTile];
    float sil[kTile];
    float fil[kTile];
    uint16_t code[kTile];
    uint32_t queue[kTile];      // slot | bits << 16
    int queue_n;
};

// Output pointers of one tile's fragments.
struct TileIO {
    const float *x, *y, *z;
    float *sil, *fil;
    uint16_t *codes;
    long long n;                // fragments in the job
    long long first;            // first fragment of the tile
    bool vec;                   // all planes 16-byte aligned
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Append `want` to the CTA queue with one atomic per warp.
__device__ __forceinline__ void queue_push(int &queue_n, uint32_t *queue, bool want, uint32_t entry)
{
    unsigned mask = __ballot_sync(0xffffffffu, want);
    if (mask == 0)
        return;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if ((int)lane_id() == leader)
        base = atomicAdd(&queue_n, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want)
        queue[base + __popc(mask & ((1u << lane_id()) - 1u))] = entry;
}

// Process one tile (all threads of the CTA call this; ends with a barrier).
template <int MODE, bool CODES, int kThreads>
__device__ __forceinline__ void process_tile(const MapDev &m, const TileIO &io, int max_dist,
                                             TileSmem<kThreads> &sm)
{
    constexpr int kTile = TileSmem<kThreads>::kTile;
    const int t = threadIdx.x;
    if (t == 0)
        sm.queue_n = 0;
    __syncthreads();

    // --- 1. load.  Vector path: thread t owns slots 4t..4t+3.  Scalar path:
    // thread t owns slots t, t + kThreads, ... (coalesced either way).
    float xs[kPerThread], ys[kPerThread], zs[kPerThread];
    int slot[kPerThread];
    bool valid[kPerThread];
    const long long remain = io.n - io.first;
    if (io.vec && remain >= kTile) {
        const float4 vx = __ldcs(reinterpret_cast<const float4 *>(io.x + io.first) + t);
        const float4 vy = __ldcs(reinterpret_cast<const float4 *>(io.y + io.first) + t);
        const float4 vz = __ldcs(reinterpret_cast<const float4 *>(io.z + io.first) + t);
        xs[0] = vx.x; xs[1] = vx.y; xs[2] = vx.z; xs[3] = vx.w;
        ys[0] = vy.x; ys[1] = vy.y; ys[2] = vy.z; ys[3] = vy.w;
        zs[0] = vz.x; zs[1] = vz.y; zs[2] = vz.z; zs[3] = vz.w;
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            slot[e] = kPerThread * t + e;
            valid[e] = true;
        }
    } else {
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            slot[e] = t + e * kThreads;
            valid[e] = slot[e] < remain;
            long long g = io.first + slot[e];
            xs[e] = valid[e] ? __ldcs(io.x + g) : 0.0f;
            ys[e] = valid[e] ? __ldcs(io.y + g) : 0.0f;
            zs[e] = valid[e] ? __ldcs(io.z + g) : 0.0f;
        }
    }

    // --- 2. classify; finish off-edge fragments, queue edge fragments.
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
        FragResult r{0.0f, 0.0f, 0};
        uint32_t bits = 0;
        bool edge = false;
        if (valid[e])
            edge = classify<MODE, CODES>(m, xs[e], ys[e], zs[e], r, bits);
        const int s = slot[e];
        sm.x[s] = xs[e];
        sm.y[s] = ys[e];
        sm.z[s] = zs[e];
        if (MODE & 1) sm.sil[s] = r.sil;
        if (MODE & 2) sm.fil[s] = r.fil;
        if (CODES) sm.code[s] = r.code;
        queue_push(sm.queue_n, sm.queue, edge, (uint32_t)s | (bits << 16));
    }
    __syncthreads();

    // --- 3. drain the edge queue with converged lanes.
    const int qn = sm.queue_n;
    for (int q = t; q < qn; q += kThreads) {
        const uint32_t entry = sm.queue[q];
        const int s = entry & 0xffff;
        const uint32_t bits = entry >> 16;
        FragResult r;
        r.code = CODES ? sm.code[s] : 0;
        r.sil = 0.0f;
        r.fil = 0.0f;
        resolve_edge<MODE>(m, sm.x[s], sm.y[s], sm.z[s], bits, max_dist, r);
        if (MODE & 1) sm.sil[s] = r.sil;
        if (MODE & 2) sm.fil[s] = r.fil;
        if (CODES) sm.code[s] = r.code;
    }
    __syncthreads();

    // --- 4. store.
    if (io.vec && remain >= kTile) {
        if (MODE & 1)
            __stcs(reinterpret_cast<float4 *>(io.sil + io.first) + t,
                   reinterpret_cast<const float4 *>(sm.sil)[t]);
        if (MODE & 2)
            __stcs(reinterpret_cast<float4 *>(io.fil + io.first) + t,
                   reinterpret_cast<const float4 *>(sm.fil)[t]);
        if (CODES) {
            const uint2 c = reinterpret_cast<const uint2 *>(sm.code)[t];
            __stcs(reinterpret_cast<uint2 *>(io.codes + io.first) + t, c);
        }
    } else {
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            if (!valid[e])
                continue;
            const long long g = io.first + slot[e];
            if (MODE & 1) io.sil[g] = sm.sil[slot[e]];
            if (MODE & 2) io.fil[g] = sm.fil[slot[e]];
            if (CODES) io.codes[g] = sm.code[slot[e]];
        }
    }
    __syncthreads();
}

}  // namespace rbsm
