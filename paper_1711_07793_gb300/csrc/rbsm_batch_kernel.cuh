// Device side of the batched launch: descriptors, per-warp queues, the
// learned drain and the batch_kernel template.  Its instantiations are
// spread over rbsm_batch_inst_*.cu so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_mlp.cuh"

namespace rbsm {

struct BatchJobDev {
    const float *x, *y, *z;
    float *sil, *fil;
    uint16_t *codes;
    long long n;
    long long tile_start;        // first work item of the job
    int map;
    int mode;                    // 1, 2, 3
    int vec;                     // all planes 16-byte aligned
    int codes_on;
};

// Passed by value as a __grid_constant__ kernel parameter (about 21 KB,
// inside the 32 KB parameter space), so no descriptor copy to the device
// is needed and the launch can be captured into a CUDA graph as is.
struct BatchArgs {
    MapDev maps[RBSM_BATCH_MAX_MAPS];
    BatchJobDev jobs[RBSM_BATCH_MAX_JOBS];
    int n_jobs;
    int max_dist;
    long long total_tiles;
    unsigned long long *counter;
    int *status;
    const void *mlp;                 // surrogate state block or nullptr
    float tau;                       // guard: largest accepted error estimate
    unsigned long long *stats;       // [0] surrogate answers, [1] fallbacks
    int chunk_tiles;                 // warp tiles per claim of the work counter, 1..kMaxChunkTiles
};

constexpr size_t kWorkspaceBytes = 256;
constexpr int kMaxChunkTiles = 8;

__device__ __forceinline__ int find_job(const BatchArgs &a, long long tile)
{
    int lo = 0, hi = a.n_jobs - 1;    // last job whose first tile <= tile
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.jobs[mid].tile_start <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ WarpTileIO job_tile(const BatchJobDev &J, int job, long long tile)
{
    WarpTileIO t;
    t.x = J.x; t.y = J.y; t.z = J.z; t.sil = J.sil; t.fil = J.fil; t.codes = J.codes;
    t.first = (tile - J.tile_start) * kWarpTile;
    const long long left = J.n - t.first;
    t.count = left < kWarpTile ? (int)left : kWarpTile;
    t.job = job;
    t.vec = J.vec && t.count == kWarpTile;
    return t;
}

// Job table of a batched launch, for the deferred edge answers.
struct BatchJobs {
    const BatchArgs *a;
    __device__ __forceinline__ JobOut operator()(int j) const
    {
        const BatchJobDev &J = a->jobs[j];
        return JobOut{a->maps[J.map], J.x, J.y, J.z, J.sil, J.fil, J.codes_on ? J.codes : nullptr, J.mode};
    }
};

// Shared memory of the learned variant: the network's biases and weight
// pointers and, per warp, the 32 input rows and 32 outputs of one round of
// edge fragments.
template <int kThreads>
struct LearnedSmem {
    mlp::InferWeights w;
    uint16_t feat[kThreads / 32][32 * mlp::kIn];
    float out[kThreads / 32][32 * mlp::kOut];
    EdgeEntry fallback[kThreads / 32][64];      // guard-tripped fragments: < 32 left over + one round
    const uint32_t *trust;                      // trusted-pattern bitmap, or nullptr (none in force)
};

// Drain rounds of up to 32 queued edge fragments with the surrogate: each
// lane gathers its fragment's 5x5 features; the fragments whose walks stop
// inside the window and whose pattern is trusted are packed into input rows
// and the warp runs the network on as many m16 tiles as they fill (0, 1 or
// 2, on the tensor cores); each of them whose error estimate is within the
// guard takes the estimate, clamped to [0, 1]; the others (and every fragment of a job that is not in FILTER
// mode) go to the warp's fallback queue, whose exact walks run in
// rounds of 32 like the exact path's (walked in place, a round's few
// fallbacks would keep most lanes idle through the walk).
template <typename Jobs, int kThreads>
__device__ __forceinline__ void drain_queue_learned(const Jobs &jobs, WarpQueue &wq, int &count, int &fb_count,
                                                    int max_dist, bool all, LearnedSmem<kThreads> &ls, int warp,
                                                    float tau, unsigned long long *stats)
{
    const unsigned lane = lane_id();
    const unsigned below = (1u << lane) - 1u;
    const int g = lane >> 2, t = lane & 3;
    uint16_t *feat = ls.feat[warp];
    float *yout = ls.out[warp];
    EdgeEntry *fbq = ls.fallback[warp];
    auto drain_fallback = [&](bool every) {
        while (fb_count >= 32 || (every && fb_count > 0)) {
            __syncwarp();
            const int base = fb_count >= 32 ? fb_count - 32 : 0;
            const int k = base + (int)lane;
            if (k < fb_count) {
                const EdgeEntry q = fbq[k];
                resolve_entry(jobs((int)(q.bits_job >> 8)), q, max_dist);
            }
            __syncwarp();
            fb_count = base;
        }
    };
    while (count >= 32 || (all && count > 0)) {
        __syncwarp();
        const int base = count >= 32 ? count - 32 : 0;
        const int k = base + (int)lane;
        const bool valid = k < count;
        EdgeEntry q{0u, 0u};
        JobOut o{};
        if (valid) {
            q = wq.q[k];
            o = jobs((int)(q.bits_job >> 8));
        }
        const bool use_net = valid && o.mode == 2;
        // the structural guard and the trusted-pattern bitmap need only the
        // window pattern: fragments they turn down skip the network, and
        // the others are packed into the first rows of the round
        bool eligible = false;
        uint32_t bits = 0;
        float fx = 0.0f, fy = 0.0f, gap = 0.0f;
        if (use_net) {
            fragment_features(o.map, __ldg(o.x + q.idx), __ldg(o.y + q.idx), __ldg(o.z + q.idx), bits, fx, fy, gap);
            eligible = walks_inside_window(bits, max_dist) && mlp::pattern_trusted(ls.trust, bits);
        }
        const unsigned elig_mask = __ballot_sync(0xffffffffu, eligible);
        const int row = __popc(elig_mask & below);
        if (eligible)
            mlp::write_input_row(feat + row * mlp::kIn, bits, fx, fy, gap);
        __syncwarp();
        const int tiles = (__popc(elig_mask) + 15) >> 4;     // m16 tiles with rows in use (0..2)
        for (int mt = 0; mt < tiles; ++mt) {
            uint32_t xa[2][4];
            mlp::load_a(feat, mlp::kIn, mt * 16, 0, lane, xa[0]);
            mlp::load_a(feat, mlp::kIn, mt * 16, 1, lane, xa[1]);
            mlp::HiddenFrags h1, h2;
            uint32_t m1, m2;
            mlp::layer(xa, 2, ls.w.w1t, mlp::kIn, ls.w.b1, lane, h1, m1);
            mlp::layer(h1.a, 4, ls.w.w2t, mlp::kHid, ls.w.b2, lane, h2, m2);
            float y[4];
            mlp::output_layer(h2, ls.w.w3t, ls.w.b3, lane, y);
            if (t == 0) {
                yout[(mt * 16 + g) * 2] = y[0];
                yout[(mt * 16 + g) * 2 + 1] = y[1];
                yout[(mt * 16 + g + 8) * 2] = y[2];
                yout[(mt * 16 + g + 8) * 2 + 1] = y[3];
            }
        }
        __syncwarp();
        bool accepted = false;
        if (eligible) {
            const float v = yout[row * 2], e = yout[row * 2 + 1];
            // the network's own error estimate (a NaN never passes)
            accepted = e <= tau && v == v;
            if (accepted) {
                const float vc = v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v);
                o.fil[q.idx] = vc;
                if (o.codes) {
                    const uint32_t cb = q.bits_job & 0x1fu;
                    o.codes[q.idx] = (uint16_t)((cb >> 1) | ((1u - (cb & 1u)) << 4) | (1u << 10));
                }
            }
        }
        const bool walk = valid && !accepted;
        const unsigned walk_mask = __ballot_sync(0xffffffffu, walk);
        if (walk)
            fbq[fb_count + __popc(walk_mask & below)] = q;
        const unsigned acc_mask = __ballot_sync(0xffffffffu, accepted);
        const unsigned fb_mask = __ballot_sync(0xffffffffu, use_net && !accepted);
        if (lane == 0 && (acc_mask | fb_mask)) {
            atomicAdd(&stats[0], (unsigned long long)__popc(acc_mask));
            atomicAdd(&stats[1], (unsigned long long)__popc(fb_mask));
        }
        __syncwarp();
        fb_count += __popc(walk_mask);
        count = base;
        drain_fallback(false);
    }
    drain_fallback(all);
}

template <int kThreads, bool LEARNED>
struct BatchSmem {
    WarpQueue queue[kThreads / 32];
    float4 next[kThreads / 32][3][32];   // each warp's next tile: x, y, z, one float4 per lane and plane
};

template <int kThreads, bool LEARNED>
constexpr size_t batch_smem_bytes()
{
    return sizeof(BatchSmem<kThreads, LEARNED>) + (LEARNED ? sizeof(LearnedSmem<kThreads>) : 0);
}

// Persistent warps claim chunks of chunk_tiles warp tiles from the work
// counter, except that the last tiles of the launch (two per warp) go out
// one per claim, so that warps finish together instead of some running a
// whole chunk past the others.  The claim of the next chunk is issued when
// the current one starts, and its value is read only when the warp gets
// there, so the atomic's latency hides behind a chunk of work.  While a warp works on one
// tile, the asynchronous copies of its next tile's coordinates into the
// warp's shared-memory buffer are in flight: the tile is read out of the
// buffer into registers, the buffer is refilled with the next tile, and the
// registers are classified (the prefetch holds no registers, which makes
// room for 5 CTAs of 256 threads per SM).  Consecutive claims are
// consecutive tiles of the job list, so warps working at the same time
// share the L2 footprint of one region of one map.
//
// UMODE 0: each job's mode and codes flag are read at run time; UMODE
// 2 * mode + codes - 1 (1..6): every job of the launch has that pair, which
// keeps one specialisation of the classification in the loop (the run-time
// dispatch inlines all six and costs registers).
template <int kThreads, bool LEARNED, int kMinBlocks, int UMODE>
__global__ void __launch_bounds__(kThreads, kMinBlocks) batch_kernel(const __grid_constant__ BatchArgs a)
{
    constexpr int kFixedMode = (UMODE + 1) / 2;
    constexpr bool kFixedCodes = ((UMODE + 1) % 2) == 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &bs = *reinterpret_cast<BatchSmem<kThreads, LEARNED> *>(smem_raw);
    auto &ls = *reinterpret_cast<LearnedSmem<kThreads> *>(smem_raw + sizeof(BatchSmem<kThreads, LEARNED>));
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    if (LEARNED) {
        const mlp::State st = mlp::state_of(const_cast<void *>(a.mlp));
        if (threadIdx.x == 0) {
            ls.w.w1t = st.w1t;
            ls.w.w2t = st.w2t;
            ls.w.w3t = st.w3t;
        }
        for (int k = threadIdx.x; k < mlp::kHid; k += kThreads) {
            ls.w.b1[k] = st.master[mlp::kOffB1 + k];
            ls.w.b2[k] = st.master[mlp::kOffB2 + k];
        }
        for (int k = threadIdx.x; k < mlp::kOutPad; k += kThreads)
            ls.w.b3[k] = k < mlp::kOut ? st.master[mlp::kOffB3 + k] : 0.0f;
        if (threadIdx.x == 0)
            ls.trust = *st.trust_on ? st.trust : nullptr;
        __syncthreads();
    }
    WarpQueue &wq = bs.queue[warp];
    const long long total = a.total_tiles;
    unsigned long long claim = 0;
    if (lane == 0)
        claim = atomicAdd(a.counter, 1ull);
    const int chunk = a.chunk_tiles;
    // claims below c1 take `chunk` tiles, later ones a single tile, so the
    // last tiles (about two per warp) are spread one at a time
    const long long tail = 2ll * gridDim.x * (kThreads / 32);
    const long long c1 = total > tail ? (total - tail) / chunk : 0;
    long long c0 = (long long)__shfl_sync(0xffffffffu, claim, 0);
    long long tile = c0 < c1 ? c0 * chunk : c1 * chunk + (c0 - c1);
    int csz = c0 < c1 ? chunk : 1;
    if (tile >= total)
        return;
    if (lane == 0)
        claim = atomicAdd(a.counter, 1ull);      // next chunk, read later
    int in_chunk = 0;
    int job = find_job(a, tile);
    // tiles [job_lo, job_hi) belong to `job`: the search runs only when a
    // tile falls outside the current job
    long long job_lo = a.jobs[job].tile_start;
    long long job_hi = job + 1 < a.n_jobs ? a.jobs[job + 1].tile_start : total;
    WarpTileIO t = job_tile(a.jobs[job], job, tile);
    float4 (&buf)[3][32] = bs.next[warp];
    stage_tile(t, lane, buf);
    const BatchJobs jobs{&a};
    // the current job's map: in the 48-register variant (5 CTAs per SM) a
    // copy read again only when the job changes, elsewhere read per tile
    // (measured: the copy helps the former by 2.6 % on C5 and slows the
    // 3-CTA variant by 5 % on C4)
    constexpr bool kCopyMap = kMinBlocks >= 5;
    MapDev map = a.maps[a.jobs[job].map];
    int queued = 0;
    int fb_queued = 0;                         // learned variant: guard-tripped fragments waiting to walk
    for (;;) {
        long long nt;
        if (in_chunk + 1 < csz) {
            nt = tile + 1;
            in_chunk += 1;
        } else {
            const long long c = (long long)__shfl_sync(0xffffffffu, claim, 0);
            nt = c < c1 ? c * chunk : c1 * chunk + (c - c1);
            csz = c < c1 ? chunk : 1;
            in_chunk = 0;
            if (nt < total && lane == 0)
                claim = atomicAdd(a.counter, 1ull);
        }
        const bool more = nt < total;
        int njob = job;
        WarpTileIO tn;
        LaneCoords c;
        fetch_tile(t, lane, buf, c);
        if (more) {
            if (nt < job_lo || nt >= job_hi) {
                njob = find_job(a, nt);
                job_lo = a.jobs[njob].tile_start;
                job_hi = njob + 1 < a.n_jobs ? a.jobs[njob + 1].tile_start : total;
                tn = job_tile(a.jobs[njob], njob, nt);
            } else {
                // same job: only the position, the count and the vector flag move
                tn = t;
                tn.first = (nt - job_lo) * kWarpTile;
                const long long left = a.jobs[job].n - tn.first;
                tn.count = left < kWarpTile ? (int)left : kWarpTile;
                tn.vec = a.jobs[job].vec && tn.count == kWarpTile;
            }
            stage_tile(tn, lane, buf);         // next tile's copies fly during this tile
        }
        const BatchJobDev &J = a.jobs[job];
        if (UMODE == 0)
            classify_warp_tile_rt(J.mode, J.codes_on != 0, kCopyMap ? map : a.maps[J.map], t, c, wq, queued);
        else
            classify_warp_tile<kFixedMode ? kFixedMode : 1, kFixedCodes>(kCopyMap ? map : a.maps[J.map], t, c, wq,
                                                                         queued);
        if (LEARNED)
            drain_queue_learned<BatchJobs, kThreads>(jobs, wq, queued, fb_queued, a.max_dist, false, ls, warp, a.tau,
                                                     a.stats);
        else
            drain_queue<BatchJobs, kFixedMode>(jobs, wq, queued, a.max_dist, false);
        if (!more)
            break;
        tile = nt;
        if (kCopyMap && njob != job)
            map = a.maps[a.jobs[njob].map];
        job = njob;
        t = tn;
    }
    if (LEARNED)
        drain_queue_learned<BatchJobs, kThreads>(jobs, wq, queued, fb_queued, a.max_dist, true, ls, warp, a.tau,
                                                 a.stats);
    else
        drain_queue<BatchJobs, kFixedMode>(jobs, wq, queued, a.max_dist, true);
}

using BatchKernelFn = void (*)(BatchArgs);

// Kernel pointers of the instantiations (one function per translation unit).
BatchKernelFn batch_kernel_256_4(bool learned, int umode);
BatchKernelFn batch_kernel_256_3(int umode);
BatchKernelFn batch_kernel_256_5(int umode);
BatchKernelFn batch_kernel_misc(int threads, bool learned);

}  // namespace rbsm
