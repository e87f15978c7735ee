// Batched evaluation: many shadow maps x many fragment sets in one
// persistent launch (host side; the kernel is in rbsm_batch_kernel.cuh).  CTAs take (job, tile) work items from an atomic
// counter in the caller's workspace, so maps of very different sizes and
// views of very different resolutions share the GPU without a launch per
// pair and without idle SMs at the end of small jobs.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_batch_kernel.cuh"
#include "rbsm_batch_host.h"
#include "rbsm_host.h"
#include "rbsm_mlp.cuh"

namespace rbsm {

// Per-kernel, per-device cache of "dynamic shared memory attribute set +
// occupancy" (the attribute is a per-device property of each kernel).
struct KernelCache {
    static constexpr int kMax = 64;
    BatchKernelFn fn[kMax] = {};
    int occ[kMax][KernelSetup::kMaxDevices] = {};
    int n = 0;
    std::mutex mu;
};

int occupancy_of(BatchKernelFn fn, int threads, size_t smem, int *occ)
{
    static KernelCache cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if (dev < 0 || dev >= KernelSetup::kMaxDevices)
        return cuda_fail(cudaErrorInvalidDevice);
    std::lock_guard<std::mutex> lock(cache.mu);
    int k = 0;
    while (k < cache.n && cache.fn[k] != fn)
        ++k;
    if (k == cache.n) {
        if (cache.n == KernelCache::kMax)
            return cuda_fail(cudaErrorInvalidConfiguration);
        cache.fn[cache.n++] = fn;
    }
    if (cache.occ[k][dev] == 0) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return cuda_fail(e);
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, threads, smem);
        if (e != cudaSuccess)
            return cuda_fail(e);
        if (o < 1)
            return cuda_fail(cudaErrorInvalidConfiguration);
        cache.occ[k][dev] = o;
    }
    *occ = cache.occ[k][dev];
    return RBSM_OK;
}

template <int kThreads, bool LEARNED, int kMinBlocks>
BatchKernelFn kernel_for(int umode)
{
    if (kThreads == 256 && kMinBlocks == 4)
        return batch_kernel_256_4(LEARNED, umode);
    if (kThreads == 256 && kMinBlocks == 3)
        return batch_kernel_256_3(umode);
    if (kThreads == 256 && kMinBlocks == 5)
        return batch_kernel_256_5(umode);
    return batch_kernel_misc(kThreads, LEARNED);
}

template <int kThreads, bool LEARNED, int kMinBlocks>
int shape_for(const BatchArgs &args, int ctas_per_sm, int chunk_req, int umode, LaunchShape *out)
{
    const size_t smem = batch_smem_bytes<kThreads, LEARNED>();
    const BatchKernelFn fn = kernel_for<kThreads, LEARNED, kMinBlocks>(umode);
    int occ = 0;
    int rc = occupancy_of(fn, kThreads, smem, &occ);
    if (rc != RBSM_OK)
        return rc;
    if (ctas_per_sm > 0 && ctas_per_sm < occ)
        occ = ctas_per_sm;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    // about 8 claims per warp: chunks of 8 tiles when there is work enough,
    // smaller ones (a power of two, down to 1) for launches of a few tiles
    // per warp, where the last chunks would otherwise leave warps idle
    long long grid = (long long)sms * occ;
    const long long warps = grid * (kThreads / 32);
    int chunk = kMaxChunkTiles;
    while (chunk > 1 && args.total_tiles < 8LL * chunk * warps)
        chunk >>= 1;
    if (chunk_req > 0)
        chunk = chunk_req;
    const long long chunks = (args.total_tiles + chunk - 1) / chunk;
    const long long blocks_needed = (chunks + kThreads / 32 - 1) / (kThreads / 32);
    if (grid > blocks_needed)
        grid = blocks_needed;
    if (grid < 1)
        grid = 1;
    *out = LaunchShape{fn, kThreads, (unsigned)grid, smem, chunk};
    return RBSM_OK;
}

// The (mode, codes) pair shared by every job, as UMODE, or 0 when they differ.
int uniform_mode(const BatchArgs &a)
{
    const int m = a.jobs[0].mode, c = a.jobs[0].codes_on;
    for (int k = 1; k < a.n_jobs; ++k)
        if (a.jobs[k].mode != m || a.jobs[k].codes_on != c)
            return 0;
    return 2 * m + c - 1;
}

// Kernel variant for a launch request.  At 256 threads the exact path has
// variants with registers sized for 3, 4 and 5 CTAs per SM (80, 64, 48 per
// thread): asking for 3 selects the first, 5 or the occupancy limit (0) the
// last, 1, 2 and 4 the middle one; the specialisations for a batch-uniform
// mode exist for the 256-thread shapes.
int launch_shape(const BatchArgs &args, int threads, int ctas_per_sm, int chunk, LaunchShape *out)
{
    if (chunk != 0 && chunk != 1 && chunk != 2 && chunk != 4 && chunk != kMaxChunkTiles)
        return RBSM_ERR_ARG;
    const bool learned = args.mlp != nullptr;
    const int um = uniform_mode(args);
    if (learned) {
        switch (threads) {
        case 128: return shape_for<128, true, 8>(args, ctas_per_sm, chunk, 0, out);
        case 512: return shape_for<512, true, 2>(args, ctas_per_sm, chunk, 0, out);
        default: return shape_for<256, true, 4>(args, ctas_per_sm, chunk, um, out);
        }
    }
    switch (threads) {
    case 128: return shape_for<128, false, 8>(args, ctas_per_sm, chunk, 0, out);
    case 512: return shape_for<512, false, 2>(args, ctas_per_sm, chunk, 0, out);
    default:
        if (ctas_per_sm == 3) return shape_for<256, false, 3>(args, ctas_per_sm, chunk, um, out);
        if (ctas_per_sm == 0 || ctas_per_sm >= 5)
            return shape_for<256, false, 5>(args, ctas_per_sm, chunk, um, out);
        return shape_for<256, false, 4>(args, ctas_per_sm, chunk, um, out);
    }
}

int launch_kernel(BatchArgs &args, const LaunchShape &sh, cudaStream_t stream)
{
    args.chunk_tiles = sh.chunk;
    sh.kernel<<<sh.grid, sh.threads, sh.smem, stream>>>(args);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}

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
    if ((b->chunk_tiles != 0 && b->chunk_tiles != 1 && b->chunk_tiles != 2 && b->chunk_tiles != 4 &&
         b->chunk_tiles != kMaxChunkTiles) ||
        (b->flags & ~RBSM_BATCH_PLAIN_LOADS))
        return RBSM_ERR_ARG;
    int rc, max_dist;
    if ((rc = check_params(&b->params, &max_dist)) != RBSM_OK)
        return rc;
    for (int k = 0; k < b->n_maps; ++k) {
        if ((rc = check_map(&b->maps[k])) != RBSM_OK)
            return rc;
        a.maps[k] = to_dev(b->maps[k]);
        if (b->flags & RBSM_BATCH_PLAIN_LOADS)
            a.maps[k].tex = 0;
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
int enqueue_batch(BatchArgs &a, const LaunchShape &sh, void *ws, cudaStream_t s)
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
    if ((rc = rbsm::launch_shape(args, threads, batch->ctas_per_sm, batch->chunk_tiles, &sh)) != RBSM_OK)
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
    rbsm::LaunchShape sh{nullptr, 256, 1, 0, 1};
    if (args.total_tiles > 0 &&
        (rc = rbsm::launch_shape(args, threads, batch->ctas_per_sm, batch->chunk_tiles, &sh)) != RBSM_OK)
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
    best->chunk_tiles = 0;
    best->flags = 0;
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
    const int cand[][2] = {{128, 0}, {256, 2}, {256, 3}, {256, 4}, {256, 0}, {512, 1}, {512, 0}};
    const int n_cand = (int)(sizeof(cand) / sizeof(cand[0]));
    const int chunks[] = {1, 2, 4, rbsm::kMaxChunkTiles};
    // the maps' textures as given, and (when any map has one) plain loads
    cudaTextureObject_t tex[RBSM_BATCH_MAX_MAPS];
    bool any_tex = false;
    for (int k = 0; k < batch->n_maps; ++k) {
        tex[k] = args.maps[k].tex;
        any_tex = any_tex || tex[k] != 0;
    }
    const int n_tex = any_tex ? 2 : 1;
    for (int ti = 0; ti < n_tex && rc == RBSM_OK; ++ti) {
        for (int k = 0; k < batch->n_maps; ++k)
            args.maps[k].tex = ti == 0 ? tex[k] : 0;
        for (int ci = 0; ci < n_cand && rc == RBSM_OK; ++ci) {
            for (int ch = 0; ch < 4 && rc == RBSM_OK; ++ch) {
                rbsm::LaunchShape sh;
                if ((rc = rbsm::launch_shape(args, cand[ci][0], cand[ci][1], chunks[ch], &sh)) != RBSM_OK)
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
                    best->chunk_tiles = chunks[ch];
                    best->flags = ti == 0 ? (batch->flags & RBSM_BATCH_PLAIN_LOADS) : RBSM_BATCH_PLAIN_LOADS;
                }
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
    if ((rc = rbsm::launch_shape(args, threads, batch->ctas_per_sm, batch->chunk_tiles, &sh)) != RBSM_OK)
        return rc;
    // enqueue_batch clears the counters that must start at zero (a memset of
    // the array's first 32 bytes, stream-ordered before the kernel)
    return rbsm::enqueue_batch(args, sh, scratch, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int rbsm_batch_noalloc_counts(uint64_t *accepted, uint64_t *fallback)
{
    if (!accepted || !fallback)
        return RBSM_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (dev >= 0 && dev < rbsm::KernelSetup::kMaxDevices)
            scratch = g_noalloc_ptr[dev];
    }
    if (!scratch)
        return rbsm::cuda_fail(cudaErrorInvalidResourceHandle);   // no call has run on this device
    return rbsm_batch_surrogate_counts(scratch, accepted, fallback);
}
