// Single-map entry points rbsm_visibility and rsmss_filter, plus the shared
// host helpers of the C ABI (argument checks, status strings, device facts).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_host.h"

namespace rbsm {

thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int)e;
    return RBSM_ERR_CUDA;
}

int check_map(const rbsm_map *m)
{
    if (!m || !m->depth)
        return RBSM_ERR_ARG;
    if (m->width < 1 || m->height < 1 || m->width > RBSM_MAX_EXTENT || m->height > RBSM_MAX_EXTENT)
        return RBSM_ERR_ARG;
    if (m->pitch < m->width)
        return RBSM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(m->depth) & 3u) != 0)
        return RBSM_ERR_ARG;
    return RBSM_OK;
}

int check_frags(const rbsm_frags *f)
{
    if (!f || f->n < 0 || f->n > RBSM_MAX_FRAGMENTS)
        return RBSM_ERR_ARG;
    if (f->n > 0 && (!f->x || !f->y || !f->z))
        return RBSM_ERR_ARG;
    const uintptr_t a = reinterpret_cast<uintptr_t>(f->x) | reinterpret_cast<uintptr_t>(f->y) |
                        reinterpret_cast<uintptr_t>(f->z);
    if (f->n > 0 && (a & 3u) != 0)
        return RBSM_ERR_ARG;
    return RBSM_OK;
}

int check_params(const rbsm_params *p, int *max_dist)
{
    if (!p) {
        *max_dist = RBSM_MAXDIST_DEFAULT;
        return RBSM_OK;
    }
    if (p->max_dist < 1 || p->max_dist > RBSM_MAXDIST_LIMIT || p->flags != 0)
        return RBSM_ERR_ARG;
    *max_dist = p->max_dist;
    return RBSM_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int device_sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

MapDev to_dev(const rbsm_map &m)
{
    return MapDev{m.depth, m.width, m.height, (long long)m.pitch, (cudaTextureObject_t)m.texture};
}

// ---------------------------------------------------------------- kernel --

// The single job of a plain launch, for the deferred edge answers.
struct PlainJobs {
    JobOut out;
    __device__ __forceinline__ const JobOut &operator()(int) const { return out; }
};

// Persistent warps walk the warp tiles of one fragment set statically
// (tile = global warp id + k * warps in the grid): consecutive warps hold
// consecutive tiles, so the warps resident at one time gather from one
// compact region of the shadow map.
// The next tile waits in shared memory (cp.async), not in registers, which
// leaves room for 5 CTAs of 256 threads per SM.
template <int MODE, bool CODES, int kThreads>
__global__ void __launch_bounds__(kThreads, 1280 / kThreads)
plain_kernel(const MapDev m, const float *__restrict__ x, const float *__restrict__ y,
             const float *__restrict__ z, long long n, float *__restrict__ sil,
             float *__restrict__ fil, uint16_t *__restrict__ codes, int max_dist, bool vec_planes)
{
    constexpr int kWarps = kThreads / 32;
    __shared__ WarpQueue wq[kWarps];
    __shared__ float4 next[kWarps][3][32];
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const long long stride = (long long)gridDim.x * kWarps;
    const long long tiles = (n + kWarpTile - 1) / kWarpTile;
    long long tile = (long long)blockIdx.x * kWarps + warp;
    if (tile >= tiles)
        return;
    const PlainJobs jobs{JobOut{m, x, y, z, sil, fil, CODES ? codes : nullptr, MODE}};
    auto io_of = [&](long long tl) {
        WarpTileIO t;
        t.x = x; t.y = y; t.z = z; t.sil = sil; t.fil = fil; t.codes = codes;
        t.first = tl * kWarpTile;
        const long long left = n - t.first;
        t.count = left < kWarpTile ? (int)left : kWarpTile;
        t.job = 0;
        t.vec = vec_planes && t.count == kWarpTile;
        return t;
    };
    WarpTileIO t = io_of(tile);
    float4 (&buf)[3][32] = next[warp];
    stage_tile(t, lane, buf);
    int queued = 0;
    for (;;) {
        const long long nt = tile + stride;
        const bool more = nt < tiles;
        WarpTileIO tn;
        LaneCoords c;
        fetch_tile(t, lane, buf, c);
        if (more) {
            tn = io_of(nt);
            stage_tile(tn, lane, buf);     // next tile's copies fly during this tile
        }
        classify_warp_tile<MODE, CODES>(m, t, c, wq[warp], queued);
        drain_queue(jobs, wq[warp], queued, max_dist, false);
        if (!more)
            break;
        tile = nt;
        t = tn;
    }
    drain_queue(jobs, wq[warp], queued, max_dist, true);
}

template <int MODE, bool CODES>
int launch_plain(const rbsm_map &map, const rbsm_frags &f, float *sil, float *fil, uint16_t *codes,
                 int max_dist, cudaStream_t stream)
{
    constexpr int kThreads = 256;
    auto kern = plain_kernel<MODE, CODES, kThreads>;
    static KernelSetup setup;
    int occupancy = 0;
    int rc = setup.get(kern, kThreads, 0, &occupancy);
    if (rc != RBSM_OK)
        return rc;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    const long long warp_tiles = (f.n + kWarpTile - 1) / kWarpTile;
    const long long blocks_needed = (warp_tiles + kThreads / 32 - 1) / (kThreads / 32);
    long long grid = (long long)sms * occupancy;
    if (grid > blocks_needed)
        grid = blocks_needed;
    bool vec = aligned16(f.x) && aligned16(f.y) && aligned16(f.z);
    if (MODE & 1) vec = vec && aligned16(sil);
    if (MODE & 2) vec = vec && aligned16(fil);
    if (CODES) vec = vec && aligned16(codes);
    kern<<<(unsigned)grid, kThreads, 0, stream>>>(to_dev(map), f.x, f.y, f.z, f.n, sil, fil, codes,
                                                  max_dist, vec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}

bool overlaps_inputs(const rbsm_map &m, const rbsm_frags &f, const void *out, size_t bytes)
{
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(out), o1 = o0 + bytes;
    auto hit = [&](const void *p, uintptr_t n) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p);
        return a < o1 && o0 < a + n;
    };
    const uintptr_t plane = (uintptr_t)f.n * 4u;
    const uintptr_t map_bytes = ((uintptr_t)(m.height - 1) * (uintptr_t)m.pitch + (uintptr_t)m.width) * 4u;
    return hit(f.x, plane) || hit(f.y, plane) || hit(f.z, plane) || hit(m.depth, map_bytes);
}

int plain_entry(int mode, const rbsm_map *map, const rbsm_frags *frags, float *vis, uint16_t *codes,
                const rbsm_params *params, void *stream)
{
    int rc, max_dist;
    if ((rc = check_map(map)) != RBSM_OK) return rc;
    if ((rc = check_frags(frags)) != RBSM_OK) return rc;
    if ((rc = check_params(params, &max_dist)) != RBSM_OK) return rc;
    if (frags->n > 0 && !vis)
        return RBSM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(vis) & 3u) != 0 || (reinterpret_cast<uintptr_t>(codes) & 1u) != 0)
        return RBSM_ERR_ARG;
    if (frags->n == 0)
        return RBSM_OK;
    if (overlaps_inputs(*map, *frags, vis, (size_t)frags->n * 4u) ||
        (codes && overlaps_inputs(*map, *frags, codes, (size_t)frags->n * 2u)))
        return RBSM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (mode == RBSM_MODE_SILHOUETTE)
        return codes ? launch_plain<1, true>(*map, *frags, vis, nullptr, codes, max_dist, s)
                     : launch_plain<1, false>(*map, *frags, vis, nullptr, nullptr, max_dist, s);
    return codes ? launch_plain<2, true>(*map, *frags, nullptr, vis, codes, max_dist, s)
                 : launch_plain<2, false>(*map, *frags, nullptr, vis, nullptr, max_dist, s);
}

}  // namespace rbsm

extern "C" {

int rbsm_visibility(const rbsm_map *map, const rbsm_frags *frags, float *vis, uint16_t *codes,
                    const rbsm_params *params, void *stream)
{
    return rbsm::plain_entry(RBSM_MODE_SILHOUETTE, map, frags, vis, codes, params, stream);
}

int rsmss_filter(const rbsm_map *map, const rbsm_frags *frags, float *vis, uint16_t *codes,
                 const rbsm_params *params, void *stream)
{
    return rbsm::plain_entry(RBSM_MODE_FILTER, map, frags, vis, codes, params, stream);
}

const char *rbsm_status_string(int code)
{
    switch (code) {
    case RBSM_OK: return "ok";
    case RBSM_ERR_ARG: return "invalid argument";
    case RBSM_ERR_CUDA: return "CUDA error";
    case RBSM_ERR_TIMEOUT: return "device-side wait timed out";
    case RBSM_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    default: return "unknown status";
    }
}

int rbsm_last_cuda_error(void) { return rbsm::g_last_cuda_error; }

int rbsm_map_texture_create(const rbsm_map *map, uint64_t *texture)
{
    if (!texture)
        return RBSM_ERR_ARG;
    *texture = 0;
    int rc = rbsm::check_map(map);
    if (rc != RBSM_OK)
        return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return rbsm::cuda_fail(e);
    int align = 0, pitch_align = 0, max_w = 0, max_h = 0, max_pitch = 0;
    if ((e = cudaDeviceGetAttribute(&align, cudaDevAttrTextureAlignment, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&pitch_align, cudaDevAttrTexturePitchAlignment, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxTexture2DLinearWidth, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&max_h, cudaDevAttrMaxTexture2DLinearHeight, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxTexture2DLinearPitch, dev)) != cudaSuccess)
        return rbsm::cuda_fail(e);
    const long long pitch_bytes = map->pitch * 4;
    if (align <= 0 || pitch_align <= 0 || (reinterpret_cast<uintptr_t>(map->depth) % (uintptr_t)align) != 0 ||
        pitch_bytes % pitch_align != 0 || map->width > max_w || map->height > max_h || pitch_bytes > max_pitch)
        return RBSM_ERR_ARG;
    cudaResourceDesc res;
    std::memset(&res, 0, sizeof(res));
    res.resType = cudaResourceTypePitch2D;
    res.res.pitch2D.devPtr = const_cast<float *>(map->depth);
    res.res.pitch2D.desc = cudaCreateChannelDesc<float>();
    res.res.pitch2D.width = (size_t)map->width;
    res.res.pitch2D.height = (size_t)map->height;
    res.res.pitch2D.pitchInBytes = (size_t)pitch_bytes;
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof(td));
    td.addressMode[0] = cudaAddressModeClamp;
    td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    cudaTextureObject_t tex = 0;
    if ((e = cudaCreateTextureObject(&tex, &res, &td, nullptr)) != cudaSuccess)
        return rbsm::cuda_fail(e);
    *texture = (uint64_t)tex;
    return RBSM_OK;
}

int rbsm_map_texture_destroy(uint64_t texture)
{
    if (texture == 0)
        return RBSM_OK;
    cudaError_t e = cudaDestroyTextureObject((cudaTextureObject_t)texture);
    return e == cudaSuccess ? RBSM_OK : rbsm::cuda_fail(e);
}

int rbsm_version(void) { return 100; }

}  // extern "C"
