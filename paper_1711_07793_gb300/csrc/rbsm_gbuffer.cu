// Visibility straight from depth buffers (rbsm_visibility_gbuffer): the
// fragment's light-space position p, Listing 1's varying, is formed in the
// kernel from the pixel's depth and a screen-to-light-clip matrix, so a
// fragment costs 4 bytes of input instead of 12.  Everything after the
// projection is the path of the other kernels: warp tiles with the next
// tile's loads in flight, classification, the deferred edge queue.  The
// drain forms p again from the pixel's depth.  A call takes many (map,
// buffer) jobs and launches one kernel per job.
#include <cuda_runtime.h>

#include <cstdint>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_host.h"

namespace rbsm {
namespace {

struct GBufDev {
    const float *d;
    int width, height;
    long long pitch;
    float m[16];
};

// p of pixel (px, py) with depth d: M (px + 0.5, py + 0.5, d, 1), each row
// summed left to right, then the perspective divide (all float32).
// px as a float for 0 <= px < 2^23, from the bit pattern of 2^23 + px.
__device__ __forceinline__ float pixel_float(int px)
{
    return __fsub_rn(__int_as_float(0x4B000000 | px), 8388608.0f);
}

__device__ __forceinline__ void project(const float (&m)[16], int px, int py, float d, float &x, float &y, float &z)
{
    const float sx = __fadd_rn(pixel_float(px), 0.5f), sy = __fadd_rn(pixel_float(py), 0.5f);
    float v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        v[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[4 * r], sx), __fmul_rn(m[4 * r + 1], sy)),
                                   __fmul_rn(m[4 * r + 2], d)),
                         m[4 * r + 3]);
    x = __fdiv_rn(v[0], v[3]);
    y = __fdiv_rn(v[1], v[3]);
    z = __fdiv_rn(v[2], v[3]);
}

// Pixel of fragment f (f < width * height <= 2^32: a 32-bit division).
__device__ __forceinline__ void pixel_of(const GBufDev &g, long long f, int &px, int &py)
{
    const unsigned fu = (unsigned)f, w = (unsigned)g.width;
    const unsigned q = fu / w;
    py = (int)q;
    px = (int)(fu - q * w);
}

// One job per launch: the map, the buffer (with its matrix) and the answer
// planes are kernel parameters, so the hot loop takes them from the
// constant bank instead of holding them in registers (a launch over many
// jobs, indexing a job table at run time, measured 35 % slower).
template <int MODE, bool CODES, int kThreads>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads)
gbuffer_kernel(const MapDev m, const GBufDev g, float *__restrict__ sil, float *__restrict__ fil,
               uint16_t *__restrict__ codes, int max_dist, bool vec_planes)
{
    constexpr int kWarps = kThreads / 32;
    __shared__ WarpQueue wq[kWarps];
    // the next job's kernel (launched as a programmatic dependent when the
    // jobs share no output) may take SMs as this one's CTAs finish
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const long long n = (long long)g.width * g.height;
    const long long stride = (long long)gridDim.x * kWarps;
    const long long tiles = (n + kWarpTile - 1) / kWarpTile;
    long long tile = (long long)blockIdx.x * kWarps + warp;
    if (tile >= tiles)
        return;
    auto io_of = [&](long long tl) {
        WarpTileIO t;
        t.x = nullptr; t.y = nullptr; t.z = nullptr; t.sil = sil; t.fil = fil; t.codes = codes;
        t.first = tl * kWarpTile;
        const long long left = n - t.first;
        t.count = left < kWarpTile ? (int)left : kWarpTile;
        t.job = 0;
        t.vec = vec_planes && t.count == kWarpTile;
        return t;
    };
    // the depths of a tile: lane l holds fragments 4l..4l+3 (vector path,
    // contiguous rows) or l, l+32, l+64, l+96
    auto load = [&](const WarpTileIO &t, float (&d)[kPerThread]) {
        if (t.vec) {
            const float4 v = __ldcs(reinterpret_cast<const float4 *>(g.d + t.first) + lane);
            d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
        } else {
#pragma unroll
            for (int e = 0; e < kPerThread; ++e) {
                const long long f = t.first + lane + 32 * e;
                d[e] = 0.0f;
                if (f < n) {
                    int px, py;
                    pixel_of(g, f, px, py);
                    d[e] = __ldcs(g.d + (long long)py * g.pitch + px);
                }
            }
        }
    };
    auto drain = [&](int &queued, bool all) {
        while (queued >= 32 || (all && queued > 0)) {
            __syncwarp();                  // queue entries and provisional stores are visible
            const int base = queued >= 32 ? queued - 32 : 0;
            const int k = base + (int)lane;
            if (k < queued) {
                const EdgeEntry q = wq[warp].q[k];
                const uint32_t bits = q.bits_job & 0x1fu;
                const uint32_t d4 = bits >> 1, s0 = bits & 1u;
                FragResult r{0.0f, 0.0f, (uint16_t)(d4 | ((1u - s0) << 4))};
                int px, py;
                pixel_of(g, q.idx, px, py);
                float x, y, z;
                project(g.m, px, py, __ldg(g.d + (long long)py * g.pitch + px), x, y, z);
                resolve_edge<MODE>(m, x, y, z, bits, max_dist, r);
                if (MODE & 1) sil[q.idx] = r.sil;
                if (MODE & 2) fil[q.idx] = r.fil;
                if (CODES) codes[q.idx] = r.code;
            }
            __syncwarp();                  // entries read before they are overwritten
            queued = base;
        }
    };
    WarpTileIO t = io_of(tile);
    float d[kPerThread];
    load(t, d);
    int queued = 0;
    for (;;) {
        const long long nt = tile + stride;
        const bool more = nt < tiles;
        WarpTileIO tn;
        float dn[kPerThread];
        if (more) {
            tn = io_of(nt);
            load(tn, dn);                  // next tile's loads fly during this tile
        }
        LaneCoords c;
        // the vector path's 4 fragments are consecutive pixels: one division
        // for the first, then steps along the row (one wrap at most when the
        // buffer is at least 4 pixels wide)
        const bool steps = t.vec && g.width >= kPerThread;
        int px = 0, py = 0;
        if (steps)
            pixel_of(g, t.first + 4 * (long long)lane, px, py);
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            const long long f = t.first + (t.vec ? 4 * (long long)lane + e : (long long)lane + 32 * e);
            c.x[e] = c.y[e] = c.z[e] = 0.0f;
            if (steps) {
                if (e > 0 && ++px == g.width) {
                    px = 0;
                    ++py;
                }
                project(g.m, px, py, d[e], c.x[e], c.y[e], c.z[e]);
            } else if (f < n) {
                int qx, qy;
                pixel_of(g, f, qx, qy);
                project(g.m, qx, qy, d[e], c.x[e], c.y[e], c.z[e]);
            }
        }
        classify_warp_tile<MODE, CODES>(m, t, c, wq[warp], queued);
        drain(queued, false);
        if (!more)
            break;
        tile = nt;
        t = tn;
#pragma unroll
        for (int e = 0; e < kPerThread; ++e)
            d[e] = dn[e];
    }
    drain(queued, true);
}

template <int MODE, bool CODES>
int launch_gbuffer(const MapDev &map, const GBufDev &g, float *sil, float *fil, uint16_t *codes, bool vec,
                   int max_dist, bool overlap, cudaStream_t stream)
{
    constexpr int kThreads = 256;
    auto kern = gbuffer_kernel<MODE, CODES, kThreads>;
    static KernelSetup setup;
    int occupancy = 0;
    int rc = setup.get(kern, kThreads, 0, &occupancy);
    if (rc != RBSM_OK)
        return rc;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    const long long n = (long long)g.width * g.height;
    const long long warp_tiles = (n + kWarpTile - 1) / kWarpTile;
    const long long blocks_needed = (warp_tiles + kThreads / 32 - 1) / (kThreads / 32);
    long long grid = (long long)sms * occupancy;
    if (grid > blocks_needed)
        grid = blocks_needed;
    cudaError_t e;
    if (overlap) {
        // a programmatic dependent of the previous job's kernel: it starts as
        // that kernel's CTAs finish instead of after its last one, and does
        // not wait for it (the jobs share no output, and everything before
        // the call is complete before the first job's kernel starts)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, map, g, sil, fil, codes, max_dist, vec);
    } else {
        kern<<<(unsigned)grid, kThreads, 0, stream>>>(map, g, sil, fil, codes, max_dist, vec);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return cuda_fail(e);
    return RBSM_OK;
}

struct Span {
    uintptr_t lo, hi;    // [lo, hi) bytes
};

bool spans_meet(const Span &a, const Span &b) { return a.lo < b.hi && b.lo < a.hi; }

// Whether the jobs' outputs are pairwise disjoint and disjoint from every
// job's inputs (depth buffer, map), so that the jobs' kernels may overlap.
bool jobs_independent(const rbsm_gbuffer_job *jobs, int n_jobs, int mode, bool codes)
{
    Span out[RBSM_GBUFFER_MAX_JOBS * 3], in[RBSM_GBUFFER_MAX_JOBS * 2];
    int n_out = 0, n_in = 0, owner[RBSM_GBUFFER_MAX_JOBS * 3];
    for (int k = 0; k < n_jobs; ++k) {
        const rbsm_gbuffer_job &j = jobs[k];
        const uintptr_t n = (uintptr_t)j.gbuffer.width * (uintptr_t)j.gbuffer.height;
        const uintptr_t d = reinterpret_cast<uintptr_t>(j.gbuffer.depth);
        in[n_in++] = Span{d, d + ((uintptr_t)j.gbuffer.pitch * (uintptr_t)(j.gbuffer.height - 1) +
                                  (uintptr_t)j.gbuffer.width) * 4u};
        const uintptr_t md = reinterpret_cast<uintptr_t>(j.map.depth);
        in[n_in++] = Span{md, md + ((uintptr_t)j.map.pitch * (uintptr_t)(j.map.height - 1) +
                                    (uintptr_t)j.map.width) * 4u};
        if (mode & 1) {
            const uintptr_t p = reinterpret_cast<uintptr_t>(j.vis_silhouette);
            owner[n_out] = k;
            out[n_out++] = Span{p, p + n * 4u};
        }
        if (mode & 2) {
            const uintptr_t p = reinterpret_cast<uintptr_t>(j.vis_filter);
            owner[n_out] = k;
            out[n_out++] = Span{p, p + n * 4u};
        }
        if (codes) {
            const uintptr_t p = reinterpret_cast<uintptr_t>(j.codes);
            owner[n_out] = k;
            out[n_out++] = Span{p, p + n * 2u};
        }
    }
    for (int a = 0; a < n_out; ++a) {
        for (int b = a + 1; b < n_out; ++b)
            if (owner[a] != owner[b] && spans_meet(out[a], out[b]))
                return false;
        for (int b = 0; b < n_in; ++b)
            if (spans_meet(out[a], in[b]))
                return false;
    }
    return true;
}

}  // namespace
}  // namespace rbsm

extern "C" int rbsm_visibility_gbuffer(const rbsm_gbuffer_job *jobs, int32_t n_jobs, int32_t mode,
                                       const rbsm_params *params, void *stream)
{
    using namespace rbsm;
    int rc, max_dist;
    if (!jobs || n_jobs < 1 || n_jobs > RBSM_GBUFFER_MAX_JOBS)
        return RBSM_ERR_ARG;
    if ((rc = check_params(params, &max_dist)) != RBSM_OK) return rc;
    if (mode < RBSM_MODE_SILHOUETTE || mode > RBSM_MODE_BOTH)
        return RBSM_ERR_ARG;
    const bool codes = jobs[0].codes != nullptr;
    // every job is checked before the first launch
    for (int k = 0; k < n_jobs; ++k) {
        const rbsm_gbuffer_job &j = jobs[k];
        const rbsm_gbuffer &gb = j.gbuffer;
        if ((rc = check_map(&j.map)) != RBSM_OK) return rc;
        if (!gb.depth || gb.width < 1 || gb.width > RBSM_MAX_EXTENT || gb.height < 1 ||
            gb.height > RBSM_MAX_EXTENT || gb.pitch < gb.width)
            return RBSM_ERR_ARG;
        if (((mode & 1) && !j.vis_silhouette) || ((mode & 2) && !j.vis_filter) || (j.codes != nullptr) != codes)
            return RBSM_ERR_ARG;
        if ((reinterpret_cast<uintptr_t>(j.vis_silhouette) & 3u) || (reinterpret_cast<uintptr_t>(j.vis_filter) & 3u) ||
            (reinterpret_cast<uintptr_t>(j.codes) & 1u) || (reinterpret_cast<uintptr_t>(gb.depth) & 3u))
            return RBSM_ERR_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool independent = n_jobs > 1 && jobs_independent(jobs, n_jobs, mode, codes);
    for (int k = 0; k < n_jobs; ++k) {
        const bool overlap = independent && k > 0;
        const rbsm_gbuffer_job &j = jobs[k];
        const rbsm_gbuffer &gb = j.gbuffer;
        GBufDev g;
        g.d = gb.depth;
        g.width = gb.width;
        g.height = gb.height;
        g.pitch = gb.pitch;
        for (int q = 0; q < 16; ++q)
            g.m[q] = gb.m[q];
        float *sil = (mode & 1) ? j.vis_silhouette : nullptr;
        float *fil = (mode & 2) ? j.vis_filter : nullptr;
        bool vec = gb.pitch == gb.width && aligned16(gb.depth);
        if (mode & 1) vec = vec && aligned16(sil);
        if (mode & 2) vec = vec && aligned16(fil);
        if (codes) vec = vec && aligned16(j.codes);
        const MapDev map = to_dev(j.map);
        switch (mode) {
        case RBSM_MODE_SILHOUETTE:
            rc = codes ? launch_gbuffer<1, true>(map, g, sil, fil, j.codes, vec, max_dist, overlap, s)
                       : launch_gbuffer<1, false>(map, g, sil, fil, nullptr, vec, max_dist, overlap, s);
            break;
        case RBSM_MODE_FILTER:
            rc = codes ? launch_gbuffer<2, true>(map, g, sil, fil, j.codes, vec, max_dist, overlap, s)
                       : launch_gbuffer<2, false>(map, g, sil, fil, nullptr, vec, max_dist, overlap, s);
            break;
        default:
            rc = codes ? launch_gbuffer<3, true>(map, g, sil, fil, j.codes, vec, max_dist, overlap, s)
                       : launch_gbuffer<3, false>(map, g, sil, fil, nullptr, vec, max_dist, overlap, s);
        }
        if (rc != RBSM_OK)
            return rc;
    }
    return RBSM_OK;
}
