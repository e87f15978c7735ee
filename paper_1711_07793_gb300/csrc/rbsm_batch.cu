// Batched evaluation: many shadow maps x many fragment sets in one
// persistent launch.  CTAs take (job, tile) work items from an atomic
// counter in the caller's workspace, so maps of very different sizes and
// views of very different resolutions share the GPU without a launch per
// pair and without idle SMs at the end of small jobs.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_host.h"
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
};

constexpr size_t kWorkspaceBytes = 256;
constexpr int kChunkTiles = 8;       // warp tiles per claim of the work counter

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
        return JobOut{a->maps[J.map], J.sil, J.fil, J.codes_on ? J.codes : nullptr, J.mode};
    }
};

// Shared memory of the learned variant: the network's weights and, per
// warp, the 32 input rows and 32 outputs of one round of edge fragments.
template <int kThreads>
struct LearnedSmem {
    mlp::SmemWeights w;
    uint16_t feat[kThreads / 32][32 * mlp::kIn];
    float out[kThreads / 32][32 * mlp::kOut];
};

// Drain rounds of up to 32 queued edge fragments with the surrogate: each
// lane gathers its fragment's 5x5 features into one input row, the warp runs
// the network on the 32 rows (two m16 tiles on the tensor cores), and each
// fragment whose error estimate is within the guard takes the estimate,
// clamped to [0, 1]; the others (and every fragment of a job that is not in
// FILTER mode) take the exact walk.
template <typename Jobs, int kThreads>
__device__ __forceinline__ void drain_queue_learned(const Jobs &jobs, WarpQueue &wq, int &count, int max_dist,
                                                    bool all, LearnedSmem<kThreads> &ls, int warp, float tau,
                                                    unsigned long long *stats)
{
    const unsigned lane = lane_id();
    const int g = lane >> 2, t = lane & 3;
    uint16_t *feat = ls.feat[warp];
    float *yout = ls.out[warp];
    while (count >= 32 || (all && count > 0)) {
        __syncwarp();
        const int base = count >= 32 ? count - 32 : 0;
        const int k = base + (int)lane;
        const bool valid = k < count;
        EdgeEntry q{0.0f, 0.0f, 0.0f, 0u, 0};
        JobOut o{};
        if (valid) {
            q = wq.q[k];
            o = jobs((int)(q.bits_job >> 8));
        }
        const bool use_net = valid && o.mode == 2;
        if (use_net) {
            uint32_t bits;
            float fx, fy, gap;
            fragment_features(o.map, q.x, q.y, q.z, bits, fx, fy, gap);
            mlp::write_input_row(feat + lane * mlp::kIn, bits, fx, fy, gap);
        } else {
            uint4 *row = reinterpret_cast<uint4 *>(feat + lane * mlp::kIn);
#pragma unroll
            for (int w4 = 0; w4 < mlp::kIn / 8; ++w4)
                row[w4] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncwarp();
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            uint32_t xa[2][4];
            mlp::load_a(feat, mlp::kIn, mt * 16, 0, lane, xa[0]);
            mlp::load_a(feat, mlp::kIn, mt * 16, 1, lane, xa[1]);
            mlp::HiddenFrags h1, h2;
            uint32_t m1, m2;
            mlp::layer(xa, 2, ls.w.w1t, mlp::kIn, ls.w.b1, lane, h1, m1);
            mlp::layer(h1.a, 4, ls.w.w2t, mlp::kHid, ls.w.b2, lane, h2, m2);
            float y[4];
            mlp::output_layer(h2, ls.w, lane, y);
            if (t == 0) {
                yout[(mt * 16 + g) * 2] = y[0];
                yout[(mt * 16 + g) * 2 + 1] = y[1];
                yout[(mt * 16 + g + 8) * 2] = y[2];
                yout[(mt * 16 + g + 8) * 2 + 1] = y[3];
            }
        }
        __syncwarp();
        bool accepted = false;
        if (use_net) {
            const float v = yout[lane * 2], e = yout[lane * 2 + 1];
            accepted = e <= tau && v == v;          // a NaN estimate never passes
            if (accepted) {
                const float vc = v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v);
                o.fil[q.idx] = vc;
                if (o.codes) {
                    const uint32_t bits = q.bits_job & 0x1fu;
                    o.codes[q.idx] = (uint16_t)((bits >> 1) | ((1u - (bits & 1u)) << 4) | (1u << 10));
                }
            }
        }
        if (valid && !accepted)
            resolve_entry(o, q, max_dist);
        const unsigned acc_mask = __ballot_sync(0xffffffffu, accepted);
        const unsigned fb_mask = __ballot_sync(0xffffffffu, use_net && !accepted);
        if (lane == 0 && (acc_mask | fb_mask)) {
            atomicAdd(&stats[0], (unsigned long long)__popc(acc_mask));
            atomicAdd(&stats[1], (unsigned long long)__popc(fb_mask));
        }
        __syncwarp();
        count = base;
    }
}

// Persistent warps claim chunks of kChunkTiles warp tiles from the work
// counter (one atomic per 1024 fragments).  The claim of the next chunk is
// issued when the current one starts, and its value is read only when the
// warp gets there, so the atomic's latency hides behind eight tiles of work.
// Consecutive claims are consecutive tiles of the job list, so warps working
// at the same time share the L2 footprint of one region of one map.
// kMinBlocks: CTAs per SM the register allocation is sized for (64
// registers per thread at 1024 threads per SM, 48 at 1280, 40 at 1536).
template <int kThreads, bool LEARNED, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) batch_kernel(const __grid_constant__ BatchArgs a)
{
    constexpr int kWarps = kThreads / 32;
    __shared__ WarpQueue wq[kWarps];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &ls = *reinterpret_cast<LearnedSmem<kThreads> *>(smem_raw);
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    if (LEARNED) {
        const mlp::State st = mlp::state_of(const_cast<void *>(a.mlp));
        for (int k = threadIdx.x; k < mlp::kW1tElems; k += kThreads) ls.w.w1t[k] = st.w1t[k];
        for (int k = threadIdx.x; k < mlp::kW2tElems; k += kThreads) ls.w.w2t[k] = st.w2t[k];
        for (int k = threadIdx.x; k < mlp::kW3tElems; k += kThreads) ls.w.w3t[k] = st.w3t[k];
        for (int k = threadIdx.x; k < mlp::kHid; k += kThreads) {
            ls.w.b1[k] = st.master[mlp::kOffB1 + k];
            ls.w.b2[k] = st.master[mlp::kOffB2 + k];
        }
        for (int k = threadIdx.x; k < mlp::kOutPad; k += kThreads)
            ls.w.b3[k] = k < mlp::kOut ? st.master[mlp::kOffB3 + k] : 0.0f;
        __syncthreads();
    }
    const long long total = a.total_tiles;
    unsigned long long claim = 0;
    if (lane == 0)
        claim = atomicAdd(a.counter, 1ull);
    long long tile = (long long)__shfl_sync(0xffffffffu, claim, 0) * kChunkTiles;
    if (tile >= total)
        return;
    if (lane == 0)
        claim = atomicAdd(a.counter, 1ull);      // next chunk, read later
    int in_chunk = 0;
    int job = find_job(a, tile);
    WarpTileIO t = job_tile(a.jobs[job], job, tile);
    LaneCoords c;
    load_tile(t, lane, c);
    const BatchJobs jobs{&a};
    int queued = 0;
    for (;;) {
        long long nt;
        if (in_chunk + 1 < kChunkTiles) {
            nt = tile + 1;
            in_chunk += 1;
        } else {
            nt = (long long)__shfl_sync(0xffffffffu, claim, 0) * kChunkTiles;
            in_chunk = 0;
            if (nt < total && lane == 0)
                claim = atomicAdd(a.counter, 1ull);
        }
        const bool more = nt < total;
        int njob = job;
        WarpTileIO tn;
        LaneCoords cn;
        if (more) {
            njob = find_job(a, nt);
            tn = job_tile(a.jobs[njob], njob, nt);
            load_tile(tn, lane, cn);           // next tile's loads fly during this tile
        }
        const BatchJobDev &J = a.jobs[job];
        classify_warp_tile_rt(J.mode, J.codes_on != 0, a.maps[J.map], t, c, wq[warp], queued);
        if (LEARNED)
            drain_queue_learned<BatchJobs, kThreads>(jobs, wq[warp], queued, a.max_dist, false, ls, warp, a.tau,
                                                     a.stats);
        else
            drain_queue(jobs, wq[warp], queued, a.max_dist, false);
        if (!more)
            break;
        tile = nt;
        job = njob;
        t = tn;
        c = cn;
    }
    if (LEARNED)
        drain_queue_learned<BatchJobs, kThreads>(jobs, wq[warp], queued, a.max_dist, true, ls, warp, a.tau, a.stats);
    else
        drain_queue(jobs, wq[warp], queued, a.max_dist, true);
}

// Launch shape of a batched launch: grid and dynamic shared memory.  Kept
// apart from the launch itself so that it runs before any stream capture
// (it sets a function attribute and queries occupancy).
struct LaunchShape {
    int threads;
    unsigned grid;
    size_t smem;
    bool learned;
    int min_blocks;
};

template <int kThreads, bool LEARNED, int kMinBlocks>
int shape_for(const BatchArgs &args, int ctas_per_sm, LaunchShape *out)
{
    // the warp queues are static shared memory; the learned variant adds
    // its weights and input rows as dynamic shared memory
    const size_t smem = LEARNED ? sizeof(LearnedSmem<kThreads>) : 0;
    static KernelSetup setup;
    int occ = 0;
    int rc = setup.get(batch_kernel<kThreads, LEARNED, kMinBlocks>, kThreads, smem, &occ);
    if (rc != RBSM_OK)
        return rc;
    if (ctas_per_sm > 0 && ctas_per_sm < occ)
        occ = ctas_per_sm;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    const long long chunks = (args.total_tiles + kChunkTiles - 1) / kChunkTiles;
    const long long blocks_needed = (chunks + kThreads / 32 - 1) / (kThreads / 32);
    long long grid = (long long)sms * occ;
    if (grid > blocks_needed)
        grid = blocks_needed;
    if (grid < 1)
        grid = 1;
    *out = LaunchShape{kThreads, (unsigned)grid, smem, LEARNED, kMinBlocks};
    return RBSM_OK;
}

// Kernel variant for a launch request.  At 256 threads, asking for 5 or 6
// CTAs per SM selects the variant whose registers are sized for that many
// (fewer registers per thread, more warps to hide gather latency).
int launch_shape(const BatchArgs &args, int threads, int ctas_per_sm, LaunchShape *out)
{
    const bool learned = args.mlp != nullptr;
    if (learned) {
        switch (threads) {
        case 128: return shape_for<128, true, 8>(args, ctas_per_sm, out);
        case 512: return shape_for<512, true, 2>(args, ctas_per_sm, out);
        default: return shape_for<256, true, 4>(args, ctas_per_sm, out);
        }
    }
    switch (threads) {
    case 128: return shape_for<128, false, 8>(args, ctas_per_sm, out);
    case 512: return shape_for<512, false, 2>(args, ctas_per_sm, out);
    default:
        if (ctas_per_sm >= 6) return shape_for<256, false, 6>(args, ctas_per_sm, out);
        if (ctas_per_sm == 5) return shape_for<256, false, 5>(args, ctas_per_sm, out);
        return shape_for<256, false, 4>(args, ctas_per_sm, out);
    }
}

int launch_kernel(const BatchArgs &args, const LaunchShape &sh, cudaStream_t stream)
{
    const unsigned g = sh.grid;
    const size_t m = sh.smem;
    if (sh.learned) {
        switch (sh.threads) {
        case 128: batch_kernel<128, true, 8><<<g, 128, m, stream>>>(args); break;
        case 512: batch_kernel<512, true, 2><<<g, 512, m, stream>>>(args); break;
        default: batch_kernel<256, true, 4><<<g, 256, m, stream>>>(args); break;
        }
    } else {
        switch (sh.threads * 16 + sh.min_blocks) {
        case 128 * 16 + 8: batch_kernel<128, false, 8><<<g, 128, m, stream>>>(args); break;
        case 512 * 16 + 2: batch_kernel<512, false, 2><<<g, 512, m, stream>>>(args); break;
        case 256 * 16 + 6: batch_kernel<256, false, 6><<<g, 256, m, stream>>>(args); break;
        case 256 * 16 + 5: batch_kernel<256, false, 5><<<g, 256, m, stream>>>(args); break;
        default: batch_kernel<256, false, 4><<<g, 256, m, stream>>>(args); break;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}

// Validate a batch and fill the kernel arguments (everything but the
// workspace pointers).  Returns RBSM_OK or RBSM_ERR_ARG.
int prepare_batch(const rbsm_batch *b, BatchArgs &a, int *threads)
{
    if (!b || !b->maps || !b->jobs)
        return RBSM_ERR_ARG;
    if (b->n_maps < 1 || b->n_maps > RBSM_BATCH_MAX_MAPS || b->n_jobs < 1 || b->n_jobs > RBSM_BATCH_MAX_JOBS)
        return RBSM_ERR_ARG;
    int th = b->tile_threads == 0 ? 256 : b->tile_threads;   // CTA size (warps per CTA)
    if (th != 128 && th != 256 && th != 512)
        return RBSM_ERR_ARG;
    if (b->ctas_per_sm < 0 || b->ctas_per_sm > 8)
        return RBSM_ERR_ARG;
    int rc, max_dist;
    if ((rc = check_params(&b->params, &max_dist)) != RBSM_OK)
        return rc;
    for (int k = 0; k < b->n_maps; ++k) {
        if ((rc = check_map(&b->maps[k])) != RBSM_OK)
            return rc;
        a.maps[k] = to_dev(b->maps[k]);
    }
    const long long tile = kWarpTile;
    long long tiles = 0;
    for (int k = 0; k < b->n_jobs; ++k) {
        const rbsm_job &j = b->jobs[k];
        if (j.map < 0 || j.map >= b->n_maps)
            return RBSM_ERR_ARG;
        if (j.mode < RBSM_MODE_SILHOUETTE || j.mode > RBSM_MODE_BOTH)
            return RBSM_ERR_ARG;
        if ((rc = check_frags(&j.frags)) != RBSM_OK)
            return rc;
        const bool want_sil = (j.mode & 1) != 0, want_fil = (j.mode & 2) != 0;
        if (j.frags.n > 0 && ((want_sil && !j.vis_silhouette) || (want_fil && !j.vis_filter)))
            return RBSM_ERR_ARG;
        if ((reinterpret_cast<uintptr_t>(j.vis_silhouette) & 3u) || (reinterpret_cast<uintptr_t>(j.vis_filter) & 3u) ||
            (reinterpret_cast<uintptr_t>(j.codes) & 1u))
            return RBSM_ERR_ARG;
        BatchJobDev &d = a.jobs[k];
        d.x = j.frags.x;
        d.y = j.frags.y;
        d.z = j.frags.z;
        d.sil = want_sil ? j.vis_silhouette : nullptr;
        d.fil = want_fil ? j.vis_filter : nullptr;
        d.codes = j.codes;
        d.n = j.frags.n;
        d.tile_start = tiles;
        d.map = j.map;
        d.mode = j.mode;
        d.codes_on = j.codes ? 1 : 0;
        bool vec = aligned16(j.frags.x) && aligned16(j.frags.y) && aligned16(j.frags.z);
        if (want_sil) vec = vec && aligned16(j.vis_silhouette);
        if (want_fil) vec = vec && aligned16(j.vis_filter);
        if (j.codes) vec = vec && aligned16(j.codes);
        d.vec = vec ? 1 : 0;
        tiles += (j.frags.n + tile - 1) / tile;
    }
    if (b->surrogate) {
        if ((reinterpret_cast<uintptr_t>(b->surrogate) & 255u) != 0 || !(b->guard_tau >= 0.0f) ||
            !(b->guard_tau < 1e30f))
            return RBSM_ERR_ARG;
    }
    a.mlp = b->surrogate;
    a.tau = b->guard_tau;
    a.n_jobs = b->n_jobs;
    a.max_dist = max_dist;
    a.total_tiles = tiles;
    *threads = th;
    return RBSM_OK;
}

int check_workspace(const void *ws, size_t bytes)
{
    if (!ws || bytes < kWorkspaceBytes || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
        return RBSM_ERR_WORKSPACE;
    return RBSM_OK;
}

// Workspace layout: [0] work counter (u64), [8] status word (int),
// [16] surrogate answers (u64), [24] surrogate fallbacks (u64).
void bind_workspace(BatchArgs &a, void *ws)
{
    a.counter = reinterpret_cast<unsigned long long *>(ws);
    a.status = reinterpret_cast<int *>(reinterpret_cast<char *>(ws) + 8);
    a.stats = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(ws) + 16);
}

// Enqueue the memset of the work counter / status word and the kernel.
int enqueue_batch(const BatchArgs &a, const LaunchShape &sh, void *ws, cudaStream_t s)
{
    if (a.total_tiles == 0)
        return RBSM_OK;
    cudaError_t e = cudaMemsetAsync(ws, 0, 32, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    return launch_kernel(a, sh, s);
}

}  // namespace rbsm

struct rbsm_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace rbsm {
}  // namespace rbsm

extern "C" {

int rbsm_batch_workspace_size(const rbsm_batch *batch, size_t *bytes)
{
    if (!batch || !bytes)
        return RBSM_ERR_ARG;
    *bytes = rbsm::kWorkspaceBytes;
    return RBSM_OK;
}

int rbsm_batch_run(const rbsm_batch *batch, void *workspace, size_t workspace_bytes, void *stream)
{
    static thread_local rbsm::BatchArgs args;   // ~22 KB: kept off the stack
    int threads = 0;
    int rc = rbsm::prepare_batch(batch, args, &threads);
    if (rc != RBSM_OK)
        return rc;
    if ((rc = rbsm::check_workspace(workspace, workspace_bytes)) != RBSM_OK)
        return rc;
    rbsm::bind_workspace(args, workspace);
    if (args.total_tiles == 0)
        return RBSM_OK;
    rbsm::LaunchShape sh;
    if ((rc = rbsm::launch_shape(args, threads, batch->ctas_per_sm, &sh)) != RBSM_OK)
        return rc;
    return rbsm::enqueue_batch(args, sh, workspace, reinterpret_cast<cudaStream_t>(stream));
}

int rbsm_batch_graph_create(const rbsm_batch *batch, void *workspace, size_t workspace_bytes,
                            rbsm_graph *graph)
{
    if (!graph)
        return RBSM_ERR_ARG;
    *graph = nullptr;
    static thread_local rbsm::BatchArgs args;
    int threads = 0;
    int rc = rbsm::prepare_batch(batch, args, &threads);
    if (rc != RBSM_OK)
        return rc;
    if ((rc = rbsm::check_workspace(workspace, workspace_bytes)) != RBSM_OK)
        return rc;
    rbsm::bind_workspace(args, workspace);
    rbsm::LaunchShape sh{256, 1, 0};
    if (args.total_tiles > 0 && (rc = rbsm::launch_shape(args, threads, batch->ctas_per_sm, &sh)) != RBSM_OK)
        return rc;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = rbsm::enqueue_batch(args, sh, workspace, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);   // always end the capture
        if (rc == RBSM_OK && e2 != cudaSuccess)
            rc = rbsm::cuda_fail(e2);
    } else {
        rc = rbsm::cuda_fail(e);
    }
    cudaStreamDestroy(s);
    if (rc != RBSM_OK) {
        if (g)
            cudaGraphDestroy(g);
        return rc;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return rbsm::cuda_fail(e);
    }
    *graph = new rbsm_graph_s{g, exec};
    return RBSM_OK;
}

int rbsm_batch_graph_launch(rbsm_graph graph, void *stream)
{
    if (!graph)
        return RBSM_ERR_ARG;
    cudaError_t e = cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    return RBSM_OK;
}

int rbsm_batch_graph_destroy(rbsm_graph graph)
{
    if (!graph)
        return RBSM_OK;
    cudaError_t e1 = cudaGraphExecDestroy(graph->exec);
    cudaError_t e2 = cudaGraphDestroy(graph->graph);
    delete graph;
    if (e1 != cudaSuccess)
        return rbsm::cuda_fail(e1);
    if (e2 != cudaSuccess)
        return rbsm::cuda_fail(e2);
    return RBSM_OK;
}

int rbsm_batch_autotune(const rbsm_batch *batch, void *workspace, size_t workspace_bytes, void *stream,
                        int32_t repeats, rbsm_tuning *best)
{
    if (!best || repeats < 1 || repeats > 1000)
        return RBSM_ERR_ARG;
    static thread_local rbsm::BatchArgs args;
    int threads = 0;
    int rc = rbsm::prepare_batch(batch, args, &threads);
    if (rc != RBSM_OK)
        return rc;
    if ((rc = rbsm::check_workspace(workspace, workspace_bytes)) != RBSM_OK)
        return rc;
    rbsm::bind_workspace(args, workspace);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    best->tile_threads = 256;
    best->ctas_per_sm = 0;
    best->ms = -1.0f;
    best->candidates = 0;
    if (args.total_tiles == 0)
        return RBSM_OK;
    cudaEvent_t t0, t1;
    cudaError_t e = cudaEventCreate(&t0);
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        cudaEventDestroy(t0);
        return rbsm::cuda_fail(e);
    }
    // candidate (CTA size, CTAs per SM); 0 = the variant's occupancy limit
    const int cand[][2] = {{128, 0}, {256, 2}, {256, 3}, {256, 0}, {256, 5}, {256, 6}, {512, 1}, {512, 0}};
    const int n_cand = (int)(sizeof(cand) / sizeof(cand[0]));
    for (int ci = 0; ci < n_cand && rc == RBSM_OK; ++ci) {
        {
            rbsm::LaunchShape sh;
            if ((rc = rbsm::launch_shape(args, cand[ci][0], cand[ci][1], &sh)) != RBSM_OK)
                break;
            if ((rc = rbsm::enqueue_batch(args, sh, workspace, s)) != RBSM_OK)   // warm-up
                break;
            if ((e = cudaEventRecord(t0, s)) != cudaSuccess) { rc = rbsm::cuda_fail(e); break; }
            for (int r = 0; r < repeats && rc == RBSM_OK; ++r)
                rc = rbsm::enqueue_batch(args, sh, workspace, s);
            if (rc != RBSM_OK)
                break;
            if ((e = cudaEventRecord(t1, s)) != cudaSuccess || (e = cudaEventSynchronize(t1)) != cudaSuccess) {
                rc = rbsm::cuda_fail(e);
                break;
            }
            float ms = 0.0f;
            if ((e = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess) { rc = rbsm::cuda_fail(e); break; }
            ms /= (float)repeats;
            best->candidates += 1;
            if (best->ms < 0.0f || ms < best->ms) {
                best->ms = ms;
                best->tile_threads = cand[ci][0];
                best->ctas_per_sm = cand[ci][1];
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return rc;
}

int rbsm_batch_surrogate_counts(const void *workspace, uint64_t *accepted, uint64_t *fallback)
{
    if (!workspace || !accepted || !fallback)
        return RBSM_ERR_ARG;
    unsigned long long v[2] = {0, 0};
    cudaError_t e = cudaMemcpy(v, reinterpret_cast<const char *>(workspace) + 16, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    *accepted = v[0];
    *fallback = v[1];
    return RBSM_OK;
}

int rbsm_batch_status(const void *workspace, int *status)
{
    if (!workspace || !status)
        return RBSM_ERR_ARG;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, reinterpret_cast<const char *>(workspace) + 8, sizeof(int),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    *status = v;
    return RBSM_OK;
}

}  // extern "C"

// ----------------------------------------------------- allocation-free run --
//
// rbsm_batch_run_noalloc: the batched launch for callers that cannot
// allocate device memory (see include/rbsm.h).  Its scratch, the same
// work counter / status word / surrogate counters rbsm_batch_run keeps in a
// caller-allocated workspace, lives in this file-scope device array instead.
// Every GPU that loads the library holds the array until the process exits.
// On the host, `g_noalloc_scratch` only names a host-side stand-in: the
// kernel is given the device address cudaGetSymbolAddress reports, looked up
// once per device (with that device current) on the first call there.

static __device__ __align__(256) unsigned char g_noalloc_scratch[RBSM_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[rbsm::KernelSetup::kMaxDevices] = {};

int noalloc_scratch_for_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    if (dev < 0 || dev >= rbsm::KernelSetup::kMaxDevices)
        return rbsm::cuda_fail(cudaErrorInvalidDevice);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return rbsm::cuda_fail(e);
        if (!p)
            return rbsm::cuda_fail(cudaErrorInvalidSymbol);
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return RBSM_OK;
}

}  // namespace

extern "C" int rbsm_batch_run_noalloc(const rbsm_batch *batch, void *stream)
{
    size_t need = 0;
    int rc = rbsm_batch_workspace_size(batch, &need);
    if (rc != RBSM_OK)
        return rc;
    if (need > (size_t)RBSM_NOALLOC_SCRATCH_BYTES)
        return RBSM_ERR_WORKSPACE;           // this batch needs more scratch than the array holds
    static thread_local rbsm::BatchArgs args;
    int threads = 0;
    if ((rc = rbsm::prepare_batch(batch, args, &threads)) != RBSM_OK)
        return rc;
    void *scratch = nullptr;
    if ((rc = noalloc_scratch_for_current_device(&scratch)) != RBSM_OK)
        return rc;
    rbsm::bind_workspace(args, scratch);
    if (args.total_tiles == 0)
        return RBSM_OK;
    rbsm::LaunchShape sh;
    if ((rc = rbsm::launch_shape(args, threads, batch->ctas_per_sm, &sh)) != RBSM_OK)
        return rc;
    // enqueue_batch clears the counters that must start at zero (a memset of
    // the array's first 32 bytes, stream-ordered before the kernel)
    return rbsm::enqueue_batch(args, sh, scratch, reinterpret_cast<cudaStream_t>(stream));
}
