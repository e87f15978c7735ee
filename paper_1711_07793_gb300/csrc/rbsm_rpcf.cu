// RPCF: percentage-closer filtering over the RSMSS answer (§5.3 removes the
// skeleton artifacts of the filtered edges with PCF; the paper prints no
// kernel).  A fragment's answer is the mean Listing 5 answer of the k x k
// samples at its texel-space position shifted by whole texels, (u + a,
// v + b), each with the fragment's depth.
//
// Same warp-tile scheme as the other kernels, with the sample as the unit
// of deferred work: a lane classifies its fragments' samples (two texture
// gathers or five loads each); off-edge samples add their shadow test at
// once, edge samples go to the warp's queue (fragment and sample index; for
// k = 3 with the fragment's shadow tests, else the drain classifies the
// sample again) and are walked 32 at a time on full warps.  For k > 1 a
// fragment with edge samples keeps its sum in the output plane as a
// fixed-point integer (each sample answer rounded to 2^-F, F = 24 / 22 / 20
// for k = 3 / 5 / 7) below a count of its samples still to come; the adds
// commute, so the result does not depend on their order, and the add that
// takes the count to zero writes the mean in place.  A fragment without
// edge samples writes its mean at once, and one outside the shared block
// (below) walks its own samples, so no second pass is needed.  For k = 1
// there is nothing to add and the answers are stored as floats
// (rsmss_filter's bits).  Because the answers do not depend on the order of
// the work, rbsm_rpcf_ws can hand the tiles out from a counter (balance
// between warps) and give the same bits as rbsm_rpcf's fixed partition.
#include <cuda_runtime.h>

#include <cstdint>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_host.h"

namespace rbsm {
namespace {

constexpr int kRpcfThreads = 256;

// The fixed-point layout of a pending fragment: F fraction bits per sample
// answer, the sum (at most K^2 * 2^F) below bit kCount, and the number of
// samples still to be added at bits kCount..31 (at most K^2):
// k = 3: 9 * 2^24 < 2^28, 9 < 2^4;  k = 5: 25 * 2^22 < 2^27, 25 < 2^5;
// k = 7: 49 * 2^20 < 2^26, 49 < 2^6.  A sample answer is off by at most
// 2^-(F+1), far inside the 1e-5 bar.
template <int K>
struct FixLayout {
    static constexpr int kFrac = K == 3 ? 24 : K == 5 ? 22 : 20;
    static constexpr int kCount = K == 3 ? 28 : K == 5 ? 27 : 26;
    static_assert((unsigned long long)(K * K) << kFrac < (1ull << kCount), "sum overflows into the count");
    static_assert(K * K < (1 << (32 - kCount)), "count overflows");
};
// Edge samples are queued per fragment element: for k <= 3 all of a lane's
// edge samples at once (a warp prefix sum places them), so the queue holds
// < 32 left over + k^2 samples of every lane; for larger k each lane's
// lowest remaining one per round (a ballot each), < 32 + 32.
template <int K>
struct RpcfQueue {
    static constexpr int kCap = K <= 3 ? 32 * K * K + 32 : 64;
    EdgeEntry q[kCap];
};

// A queued sample's number: for k = 3 its bit in the packed 5 x 5 block
// word (row y at bits 5y..5y+4, sample (a, b) at block (a + 2, b + 2)), for
// larger k its index (b + R) * K + (a + R) among the k x k samples.  A k = 3
// entry holds the number in bits 0-4 and the fragment's block word above it.
template <int K>
__device__ __forceinline__ int sample_slot(int q)
{
    return K == 3 ? (q / 3 + 1) * 5 + q % 3 + 1 : q;
}

template <int K>
__device__ __forceinline__ int sample_dx(int slot)
{
    return K == 3 ? slot % 5 - 2 : slot % K - (K - 1) / 2;
}

template <int K>
__device__ __forceinline__ int sample_dy(int slot)
{
    return K == 3 ? slot / 5 - 2 : slot / K - (K - 1) / 2;
}

template <int K>
__device__ __forceinline__ uint32_t to_fix(float v)
{
    return (uint32_t)__float2uint_rn(__fmul_rn(v, (float)(1u << FixLayout<K>::kFrac)));
}

// The mean of k^2 sample answers from their fixed-point sum.
template <int K>
__device__ __forceinline__ float mean_of(uint32_t sum)
{
    return __fdiv_rn(__fmul_rn(__uint2float_rn(sum), 1.0f / (float)(1u << FixLayout<K>::kFrac)), (float)(K * K));
}

// The same for a fragment without edge samples, whose answers are its c lit
// samples: c / k^2.  For k = 3, c * RN(1/9) rounds to RN(c / 9) for every
// c in 0..9 (checked for each c), so a multiply gives the division's bits.
template <int K>
__device__ __forceinline__ float mean_of_lit(uint32_t c)
{
    if (K == 3)
        return __fmul_rn((float)c, 1.0f / 9.0f);
    return __fdiv_rn((float)c, (float)(K * K));
}

// The shared block.  Sample (a, b)'s texel is clamp(floor(u + a)) with u + a
// rounded to float; when every such floor is floor(u) + a (u + a can round
// up to the next integer where it crosses a power of two) and the (K + 2)^2
// block of texels around floor(u), floor(v) lies inside the map (no
// clamping), all K^2 samples' four-neighbourhoods come from that one block:
// 7 texture gathers for k = 3 and ceil((K + 2) / 2)^2 for larger k instead
// of 2 K^2, and one shadow test (Eq. 1) per texel.  Other fragments take the
// per-sample path.
template <int K>
__device__ __forceinline__ bool block_ok(float u, float v, float uhi, float vhi)
{
    constexpr int R = (K - 1) / 2;
    const float fu = floorf(u), fv = floorf(v);
    bool ok = fu >= (float)(R + 1) && fu <= uhi && fv >= (float)(R + 1) && fv <= vhi;    // false for NaN
    // Only the sums can round: for 2 <= u < 2^16 (maps are at most 65536
    // texels wide) and d <= R, u - d is exact (a result at or above the
    // binade of u keeps its spacing, one below it has a finer one), so
    // floor(u - d) is floor(u) - d.
#pragma unroll
    for (int d = 1; d <= R; ++d)
        ok = ok && floorf(__fadd_rn(u, (float)d)) == fu + (float)d && floorf(__fadd_rn(v, (float)d)) == fv + (float)d;
    return ok;
}

// Shadow tests (Eq. 1) of the four texels of the gather at block columns
// p, p + 1 and rows q, q + 1 into the row masks.  A gather at (X, Y) covers
// columns X - 1, X and rows Y - 1, Y; components x = (lo col, hi row),
// y = (hi, hi), z = (hi, lo), w = (lo, lo).
template <int K>
__device__ __forceinline__ void gather_bits(const MapDev &m, float gx, float gy, int p, int q, float pz,
                                            uint32_t (&rows)[K + 2])
{
    const float4 g = tex2Dgather<float4>(m.tex, gx + (float)p, gy + (float)q, 0);
    rows[q] |= ((uint32_t)!(pz > g.w) << p) | ((uint32_t)!(pz > g.z) << (p + 1));
    if (q + 1 < K + 2)
        rows[q + 1] |= ((uint32_t)!(pz > g.x) << p) | ((uint32_t)!(pz > g.y) << (p + 1));
}

// Bit x of rows[y]: texel (floor(u) - R - 1 + x, floor(v) - R - 1 + y) is
// lit for depth pz (Eq. 1).  The samples' classification reads the block
// without its four corners (each sample's texel and its four neighbours).
// For k = 3 that is 21 texels of the 5 x 5 block, which seven gathers cover
// (rows 0-1 at columns 0-3, rows 3-4 at columns 1-4, and three across the
// middle row); larger k take the whole block, ceil((K + 2) / 2)^2 gathers.
// Bits of the corners may be missing; nothing reads them.
template <int K>
__device__ __forceinline__ void block_bits(const MapDev &m, float u, float v, float pz, uint32_t (&rows)[K + 2])
{
    constexpr int R = (K - 1) / 2, B = K + 2, G = (B + 1) / 2;
    const float gx = floorf(u) - (float)R, gy = floorf(v) - (float)R;
#pragma unroll
    for (int y = 0; y < B; ++y)
        rows[y] = 0u;
    if constexpr (K == 3) {
        gather_bits<K>(m, gx, gy, 0, 0, pz, rows);
        gather_bits<K>(m, gx, gy, 2, 0, pz, rows);
        gather_bits<K>(m, gx, gy, 3, 1, pz, rows);
        gather_bits<K>(m, gx, gy, 1, 1, pz, rows);
        gather_bits<K>(m, gx, gy, 0, 2, pz, rows);
        gather_bits<K>(m, gx, gy, 1, 3, pz, rows);
        gather_bits<K>(m, gx, gy, 3, 3, pz, rows);
    } else {
#pragma unroll
        for (int n = 0; n < G; ++n) {
#pragma unroll
            for (int c = 0; c < G; ++c)
                gather_bits<K>(m, gx, gy, 2 * c, 2 * n, pz, rows);
        }
    }
}

template <int K, int kThreads>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads)
rpcf_kernel(const MapDev m, const float *__restrict__ x, const float *__restrict__ y,
            const float *__restrict__ z, long long n, float *__restrict__ vis, int max_dist, bool vec_planes,
            unsigned long long *next_tile)
{
    constexpr int kWarps = kThreads / 32;
    constexpr int R = (K - 1) / 2;
    __shared__ RpcfQueue<K> wq[kWarps];
    __shared__ float4 next[kWarps][3][32];     // the next tile's coordinates (cp.async)
    const unsigned lane = lane_id();
    const unsigned below = (1u << lane) - 1u;
    const int warp = threadIdx.x >> 5;
    const long long stride = (long long)gridDim.x * kWarps;
    const long long tiles = (n + kWarpTile - 1) / kWarpTile;
    long long tile = (long long)blockIdx.x * kWarps + warp;
    if (tile >= tiles)
        return;
    // schedule: every warp takes one tile of the first wave; after that
    // either the static stride or, with a counter (next_tile, k > 1), one
    // tile per claim, taken one tile ahead, so that warps whose tiles carry
    // many edge samples do not hold up the end of the launch
    const bool claims = K > 1 && next_tile != nullptr;
    unsigned long long claim = 0;
    if (claims && lane == 0)
        claim = atomicAdd(next_tile, 1ull);
    const float W = (float)m.width, H = (float)m.height;
    // the largest floor(u), floor(v) whose block lies inside the map
    const float uhi = (float)(m.width - R - 2), vhi = (float)(m.height - R - 2);
    const bool tex = K > 1 && m.tex != 0;
    uint32_t *acc = reinterpret_cast<uint32_t *>(vis);
    auto io_of = [&](long long tl) {
        WarpTileIO t;
        t.x = x; t.y = y; t.z = z; t.sil = nullptr; t.fil = vis; t.codes = nullptr;
        t.first = tl * kWarpTile;
        const long long left = n - t.first;
        t.count = left < kWarpTile ? (int)left : kWarpTile;
        t.job = 0;
        t.vec = vec_planes && t.count == kWarpTile;
        return t;
    };
    // drain rounds of 32 queued edge samples: walk, answer, add
    auto drain = [&](int &queued, bool all) {
        while (queued >= 32 || (all && queued > 0)) {
            __syncwarp();                  // entries and the fragments' base values are visible
            const int base = queued >= 32 ? queued - 32 : 0;
            const int q = base + (int)lane;
            if (q < queued) {
                const EdgeEntry e = wq[warp].q[q];
                const uint32_t i = e.idx;
                const int sample = K == 3 ? (int)(e.bits_job & 31u) : (int)e.bits_job;
                const float ua = __fadd_rn(__fmul_rn(__ldg(x + i), W), (float)sample_dx<K>(sample));
                const float vb = __fadd_rn(__fmul_rn(__ldg(y + i), H), (float)sample_dy<K>(sample));
                const float pz = __ldg(z + i);
                FragResult r{0.0f, 0.0f, 0};
                uint32_t bits;
                if (K == 3) {
                    // the entry carries the fragment's block word: the
                    // sample's shadow test and its four neighbours' (left,
                    // right one bit away, +y, -y five bits away) are bits of
                    // it, taken with the same depth from the same texels
                    const uint32_t P = e.bits_job >> 5;
                    const uint32_t s0 = (P >> sample) & 1u;
                    bits = s0 | ((((P >> (sample - 1)) & 1u) ^ s0) << 1) | ((((P >> (sample + 1)) & 1u) ^ s0) << 2) |
                           ((((P >> (sample + 5)) & 1u) ^ s0) << 3) | ((((P >> (sample - 5)) & 1u) ^ s0) << 4);
                } else {
                    classify_uv<2, false>(m, ua, vb, pz, r, bits);    // the sample's discontinuity again
                }
                // walks through the texture view (two steps per gather), except
                // for k = 3, where the scalar walk measured 1 % faster
                resolve_edge_uv<2, K == 3 ? 0 : 2>(m, ua, vb, pz, bits, max_dist, r);
                if (K == 1) {
                    vis[i] = r.fil;
                } else {
                    // queued samples come from fragments inside the shared
                    // block (finite coordinates), whose answers are finite
                    constexpr int C = FixLayout<K>::kCount;
                    const uint32_t add = to_fix<K>(r.fil) - (1u << C);    // one sample fewer to come
                    const uint32_t old = atomicAdd(acc + i, add);
                    if ((old >> C) == 1u)                                  // the fragment's last sample
                        vis[i] = mean_of<K>((old + add) & ((1u << C) - 1u));
                }
            }
            __syncwarp();                  // entries read before they are overwritten
            queued = base;
        }
    };
    WarpTileIO t = io_of(tile);
    float4 (&buf)[3][32] = next[warp];
    stage_tile(t, lane, buf);
    int queued = 0;
    for (;;) {
        long long nt = tile + stride;
        if (claims) {
            nt = stride + (long long)__shfl_sync(0xffffffffu, claim, 0);
            if (nt < tiles && lane == 0)
                claim = atomicAdd(next_tile, 1ull);
        }
        const bool more = nt < tiles;
        WarpTileIO tn;
        LaneCoords c;
        fetch_tile_strided(t, lane, buf, c);
        if (more) {
            tn = io_of(nt);
            stage_tile(tn, lane, buf);     // next tile's copies fly during this tile
        }
#pragma unroll 1
        for (int e = 0; e < kPerThread; ++e) {
            const int s = (int)lane + 32 * e;
            const bool valid = s < t.count;
            const float xe = e == 0 ? c.x[0] : e == 1 ? c.x[1] : e == 2 ? c.x[2] : c.x[3];
            const float ye = e == 0 ? c.y[0] : e == 1 ? c.y[1] : e == 2 ? c.y[2] : c.y[3];
            const float ze = e == 0 ? c.z[0] : e == 1 ? c.z[1] : e == 2 ? c.z[2] : c.z[3];
            const float u = __fmul_rn(xe, W), v = __fmul_rn(ye, H);
            // all samples' texel reads first; off-edge samples add their
            // shadow test to the base value, edge samples set their bit
            uint64_t edges = 0;
            uint32_t base = 0, block = 0;
            float single = 0.0f;
            const bool base_path = tex && valid && block_ok<K>(u, v, uhi, vhi);
            if (base_path) {
                uint32_t rows[K + 2];
                block_bits<K>(m, u, v, ze, rows);
                // a row of samples at once: sample (a, b)'s texel is block
                // (a + 1, b + 1); it is an edge sample where one of Listing
                // 2's four neighbours differs from it, else it adds its
                // shadow test
                if constexpr (K == 3) {
                    // the whole 5 x 5 block in one word, row y at bits 5y..5y+4:
                    // a sample differs from a neighbour one bit (left, right)
                    // or five bits (below, above) away, so the four
                    // comparisons of Listing 2 cover all nine samples at once
                    const uint32_t P = rows[0] | (rows[1] << 5) | (rows[2] << 10) | (rows[3] << 15) | (rows[4] << 20);
                    constexpr uint32_t kSamples = (7u << 6) | (7u << 11) | (7u << 16);   // rows 1-3, columns 1-3
                    const uint32_t e = ((P ^ (P >> 1)) | (P ^ (P << 1)) | (P ^ (P >> 5)) | (P ^ (P << 5))) & kSamples;
                    edges = e;
                    block = P;
                    base = (uint32_t)__popc(P & ~e & kSamples) << FixLayout<K>::kFrac;
                } else {
                    constexpr uint32_t mk = (1u << K) - 1u;
#pragma unroll
                    for (int b = 0; b < K; ++b) {
                        const uint32_t c = (rows[b + 1] >> 1) & mk;
                        const uint32_t e = (c ^ (rows[b + 1] & mk)) | (c ^ ((rows[b + 1] >> 2) & mk)) |
                                           (c ^ ((rows[b + 2] >> 1) & mk)) | (c ^ ((rows[b] >> 1) & mk));
                        edges |= (uint64_t)e << (K * b);
                        base += (uint32_t)__popc(c & ~e) << FixLayout<K>::kFrac;
                    }
                }
            } else if (K == 1) {
                FragResult r{0.0f, 0.0f, 0};
                uint32_t bits = 0;
                if (valid && classify_uv<2, false>(m, u, v, ze, r, bits))
                    edges = 1ull << sample_slot<K>(0);
                single = r.fil;
            } else if (valid) {
                // outside the shared block (the map's border rows and
                // columns, or a non-finite coordinate): the lane walks its
                // own edge samples and writes the mean (rare, so the
                // divergence costs little)
                uint32_t sum = 0;
                bool nan = false;
#pragma unroll 1
                for (int q = 0; q < K * K; ++q) {
                    FragResult r{0.0f, 0.0f, 0};
                    uint32_t bits = 0;
                    const float ua = __fadd_rn(u, (float)(q % K - R)), vb = __fadd_rn(v, (float)(q / K - R));
                    if (classify_uv<2, false>(m, ua, vb, ze, r, bits))
                        resolve_edge_uv<2, K == 3 ? 0 : 2>(m, ua, vb, ze, bits, max_dist, r);
                    if (r.fil != r.fil)
                        nan = true;               // a NaN answer (NaN or infinite coordinates)
                    else
                        sum += to_fix<K>(r.fil);
                }
                vis[t.first + s] = nan ? __int_as_float(0x7fc00000) : mean_of<K>(sum);
            }
            // the base value is stored before any deferred sample of this
            // fragment can add to it ...
            const uint32_t ne = (uint32_t)__popcll(edges);
            if (valid) {
                if (K == 1)
                    vis[t.first + s] = single;
                else if (ne != 0)
                    acc[t.first + s] = (ne << FixLayout<K>::kCount) | base;
                else if (base_path)
                    vis[t.first + s] = mean_of_lit<K>(base >> FixLayout<K>::kFrac);
            }
            // ... then the edge samples are queued and walked whenever 32
            // are waiting
            if (K <= 3) {
                // all of the lane's edge samples, placed by a prefix sum
                uint32_t incl = ne, total = 0;
                if (__any_sync(0xffffffffu, ne != 0)) {      // about one element in five has none
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t t2 = __shfl_up_sync(0xffffffffu, incl, off);
                        if ((int)lane >= off)
                            incl += t2;
                    }
                    total = __shfl_sync(0xffffffffu, incl, 31);
                }
                if (total != 0u) {
                    int pos = queued + (int)(incl - ne);
                    uint64_t rest = edges;
                    while (rest) {
                        const int q = __ffsll((long long)rest) - 1;
                        rest &= rest - 1;
                        wq[warp].q[pos++] = EdgeEntry{(uint32_t)(t.first + s), K == 3 ? (block << 5) | (uint32_t)q : (uint32_t)q};
                    }
                    queued += (int)total;
                    drain(queued, false);
                }
            } else {
                // each lane's lowest remaining edge sample per round: as many
                // rounds as the most edge samples of any lane's fragment
                uint64_t rest = edges;
                while (__any_sync(0xffffffffu, rest != 0)) {
                    const bool has = rest != 0;
                    const unsigned mask = __ballot_sync(0xffffffffu, has);
                    if (has) {
                        const int q = __ffsll((long long)rest) - 1;
                        rest &= rest - 1;
                        wq[warp].q[queued + __popc(mask & below)] = EdgeEntry{(uint32_t)(t.first + s), (uint32_t)q};
                    }
                    queued += __popc(mask);
                    drain(queued, false);
                }
            }
        }
        if (!more)
            break;
        tile = nt;
        t = tn;
    }
    drain(queued, true);
}

template <int K>
int launch_rpcf(const rbsm_map &map, const rbsm_frags &f, float *vis, int max_dist, unsigned long long *ctr,
                cudaStream_t stream)
{
    auto kern = rpcf_kernel<K, kRpcfThreads>;
    static KernelSetup setup;
    int occupancy = 0;
    int rc = setup.get(kern, kRpcfThreads, 0, &occupancy);
    if (rc != RBSM_OK)
        return rc;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    const long long warp_tiles = (f.n + kWarpTile - 1) / kWarpTile;
    const long long blocks_needed = (warp_tiles + kRpcfThreads / 32 - 1) / (kRpcfThreads / 32);
    long long grid = (long long)sms * occupancy;
    if (grid > blocks_needed)
        grid = blocks_needed;
    const bool vec = aligned16(f.x) && aligned16(f.y) && aligned16(f.z);
    if (K > 1 && ctr) {
        const cudaError_t ez = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), stream);
        if (ez != cudaSuccess)
            return cuda_fail(ez);
    }
    kern<<<(unsigned)grid, kRpcfThreads, 0, stream>>>(to_dev(map), f.x, f.y, f.z, f.n, vis, max_dist, vec,
                                                      K > 1 ? ctr : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}

}  // namespace
}  // namespace rbsm

namespace rbsm {
namespace {

int rpcf_entry(const rbsm_map *map, const rbsm_frags *frags, float *vis, int32_t k, const rbsm_params *params,
               unsigned long long *ctr, void *stream)
{
    int rc, max_dist;
    if ((rc = check_map(map)) != RBSM_OK) return rc;
    if ((rc = check_frags(frags)) != RBSM_OK) return rc;
    if ((rc = check_params(params, &max_dist)) != RBSM_OK) return rc;
    if (k < 1 || k > RBSM_RPCF_MAX_K || (k & 1) == 0)
        return RBSM_ERR_ARG;
    if (frags->n > 0 && !vis)
        return RBSM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(vis) & 3u) != 0)
        return RBSM_ERR_ARG;
    if (frags->n == 0)
        return RBSM_OK;
    // vis holds partial sums while the kernel runs: it must not overlap an input
    if (overlaps_inputs(*map, *frags, vis, (size_t)frags->n * 4u))
        return RBSM_ERR_ARG;
    if (ctr && (overlaps_inputs(*map, *frags, ctr, 8) ||
                (reinterpret_cast<uintptr_t>(ctr) < reinterpret_cast<uintptr_t>(vis) + (uintptr_t)frags->n * 4u &&
                 reinterpret_cast<uintptr_t>(vis) < reinterpret_cast<uintptr_t>(ctr) + 8u)))
        return RBSM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (k) {
    case 1: return launch_rpcf<1>(*map, *frags, vis, max_dist, ctr, s);
    case 3: return launch_rpcf<3>(*map, *frags, vis, max_dist, ctr, s);
    case 5: return launch_rpcf<5>(*map, *frags, vis, max_dist, ctr, s);
    default: return launch_rpcf<7>(*map, *frags, vis, max_dist, ctr, s);
    }
}

}  // namespace
}  // namespace rbsm

extern "C" int rbsm_rpcf(const rbsm_map *map, const rbsm_frags *frags, float *vis, int32_t k,
                         const rbsm_params *params, void *stream)
{
    return rbsm::rpcf_entry(map, frags, vis, k, params, nullptr, stream);
}

extern "C" int rbsm_rpcf_ws(const rbsm_map *map, const rbsm_frags *frags, float *vis, int32_t k,
                            const rbsm_params *params, void *workspace, void *stream)
{
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 7u) != 0)
        return RBSM_ERR_ARG;
    return rbsm::rpcf_entry(map, frags, vis, k, params, reinterpret_cast<unsigned long long *>(workspace), stream);
}
