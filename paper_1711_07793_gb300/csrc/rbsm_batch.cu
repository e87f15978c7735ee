// Batched evaluation: many shadow maps x many fragment sets in one
// persistent launch.  CTAs take (job, tile) work items from an atomic
// counter in the caller's workspace, so maps of very different sizes and
// views of very different resolutions share the GPU without a launch per
// pair and without idle SMs at the end of small jobs.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_host.h"

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
};

constexpr size_t kWorkspaceBytes = 256;

template <int kThreads>
__device__ __forceinline__ void run_item(const BatchArgs &a, const BatchJobDev &J, long long first,
                                         TileSmem<kThreads> &sm)
{
    const MapDev m = a.maps[J.map];
    TileIO io{J.x, J.y, J.z, J.sil, J.fil, J.codes, J.n, first, J.vec != 0};
    switch (J.mode * 2 + J.codes_on) {
    case 2: process_tile<1, false, kThreads>(m, io, a.max_dist, sm); break;
    case 3: process_tile<1, true, kThreads>(m, io, a.max_dist, sm); break;
    case 4: process_tile<2, false, kThreads>(m, io, a.max_dist, sm); break;
    case 5: process_tile<2, true, kThreads>(m, io, a.max_dist, sm); break;
    case 6: process_tile<3, false, kThreads>(m, io, a.max_dist, sm); break;
    default: process_tile<3, true, kThreads>(m, io, a.max_dist, sm); break;
    }
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads) batch_kernel(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<TileSmem<kThreads> *>(smem_raw);
    __shared__ long long item;
    constexpr long long kTile = TileSmem<kThreads>::kTile;
    for (;;) {
        if (threadIdx.x == 0)
            item = (long long)atomicAdd(a.counter, 1ull);
        __syncthreads();
        const long long t = item;          // read before process_tile's first barrier
        if (t >= a.total_tiles)
            break;
        int lo = 0, hi = a.n_jobs - 1;     // last job whose first item <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.jobs[mid].tile_start <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const BatchJobDev &J = a.jobs[lo];
        run_item<kThreads>(a, J, (t - J.tile_start) * kTile, sm);
    }
}

template <int kThreads>
int launch_batch(BatchArgs &args, int ctas_per_sm, cudaStream_t stream)
{
    const size_t smem = sizeof(TileSmem<kThreads>);
    auto kern = batch_kernel<kThreads>;
    static KernelSetup setup;
    int occ = 0;
    int rc = setup.get(kern, kThreads, smem, &occ);
    if (rc != RBSM_OK)
        return rc;
    if (ctas_per_sm > 0 && ctas_per_sm < occ)
        occ = ctas_per_sm;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    long long grid = (long long)sms * occ;
    if (grid > args.total_tiles)
        grid = args.total_tiles;
    kern<<<(unsigned)grid, kThreads, smem, stream>>>(args);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}

int tile_of(int threads) { return threads * kPerThread; }

// Validate a batch and fill the kernel arguments (everything but the
// workspace pointers).  Returns RBSM_OK or RBSM_ERR_ARG.
int prepare_batch(const rbsm_batch *b, BatchArgs &a, int *threads)
{
    if (!b || !b->maps || !b->jobs)
        return RBSM_ERR_ARG;
    if (b->n_maps < 1 || b->n_maps > RBSM_BATCH_MAX_MAPS || b->n_jobs < 1 || b->n_jobs > RBSM_BATCH_MAX_JOBS)
        return RBSM_ERR_ARG;
    int th = b->tile_threads == 0 ? 256 : b->tile_threads;
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
    const long long tile = tile_of(th);
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

// Enqueue the memset of the work counter / status word and the kernel.
int enqueue_batch(BatchArgs &a, int threads, int ctas_per_sm, void *ws, cudaStream_t s)
{
    a.counter = reinterpret_cast<unsigned long long *>(ws);
    a.status = reinterpret_cast<int *>(reinterpret_cast<char *>(ws) + 8);
    if (a.total_tiles == 0)
        return RBSM_OK;
    cudaError_t e = cudaMemsetAsync(ws, 0, 16, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    switch (threads) {
    case 128: return launch_batch<128>(a, ctas_per_sm, s);
    case 512: return launch_batch<512>(a, ctas_per_sm, s);
    default: return launch_batch<256>(a, ctas_per_sm, s);
    }
}

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
    static thread_local rbsm::BatchArgs args;   // ~21 KB: kept off the stack
    int threads = 0;
    int rc = rbsm::prepare_batch(batch, args, &threads);
    if (rc != RBSM_OK)
        return rc;
    if ((rc = rbsm::check_workspace(workspace, workspace_bytes)) != RBSM_OK)
        return rc;
    return rbsm::enqueue_batch(args, threads, batch->ctas_per_sm, workspace,
                               reinterpret_cast<cudaStream_t>(stream));
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
