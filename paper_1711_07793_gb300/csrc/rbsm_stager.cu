// Host-resident batches (rbsm_stager_*).  Per map: copy the fragment planes
// of the map's jobs in, find the texel bounds of those fragments on the
// device, copy in only the window of the map the path can read (the bounds
// grown by max_dist + 1), run the batched kernel on the staged copies and
// copy the answers out.  A ring of device slots and four streams (in,
// window, kernel, out) let consecutive maps overlap; no step waits on the
// host.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "rbsm.h"
#include "rbsm_batch_host.h"
#include "rbsm_batch_kernel.cuh"
#include "rbsm_device.cuh"
#include "rbsm_host.h"

namespace rbsm {
namespace {

constexpr int kMaxSlots = 4;
constexpr int kDefaultSlots = 3;
constexpr int kBoundsThreads = 256;
constexpr int kWindowThreads = 256;
constexpr long long kJobAlign = 32;           // floats: job offsets inside a slot are 128-byte aligned
constexpr size_t kSubAlign = 4096;            // bytes: alignment of the buffers carved from a slot

// ---------------------------------------------------------------- kernels --

// Texel bounds of staged fragments, with the kernels' own texel arithmetic
// (texel_coord: clamp(floor(x * size))).  win[0] / win[2] collect the maximum
// of ~i / ~j (so ~win[0] is the smallest i), win[1] / win[3] the maximum of
// i + 1 / j + 1; all four start at 0, and win[1] == 0 afterwards means no
// fragment.  x and y are 16-byte aligned (the slot layout).
__global__ void __launch_bounds__(kBoundsThreads) texel_bounds(const float *__restrict__ x,
                                                               const float *__restrict__ y, long long n,
                                                               int width, int height, unsigned *win)
{
    unsigned lo_i = 0, hi_i = 0, lo_j = 0, hi_j = 0;
    auto take = [&](float xv, float yv) {
        int i, j;
        float f;
        texel_coord(xv, width, i, f);
        texel_coord(yv, height, j, f);
        lo_i = max(lo_i, ~(unsigned)i);
        hi_i = max(hi_i, (unsigned)i + 1u);
        lo_j = max(lo_j, ~(unsigned)j);
        hi_j = max(hi_j, (unsigned)j + 1u);
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n4 = n / 4;
    for (long long k = t0; k < n4; k += stride) {
        const float4 a = reinterpret_cast<const float4 *>(x)[k];
        const float4 b = reinterpret_cast<const float4 *>(y)[k];
        take(a.x, b.x);
        take(a.y, b.y);
        take(a.z, b.z);
        take(a.w, b.w);
    }
    for (long long k = n4 * 4 + t0; k < n; k += stride)
        take(x[k], y[k]);
    lo_i = __reduce_max_sync(0xffffffffu, lo_i);
    hi_i = __reduce_max_sync(0xffffffffu, hi_i);
    lo_j = __reduce_max_sync(0xffffffffu, lo_j);
    hi_j = __reduce_max_sync(0xffffffffu, hi_j);
    if ((threadIdx.x & 31) == 0 && hi_i != 0) {
        atomicMax(&win[0], lo_i);
        atomicMax(&win[1], hi_i);
        atomicMax(&win[2], lo_j);
        atomicMax(&win[3], hi_j);
    }
}

// Copy the window of a host map (page-locked, read through its device
// mapping) into the same texels of the slot's map: the texel bounds in win
// grown by `halo`, clipped to the map and widened to columns 4k .. 4k+3
// (also clipped), so that rows move in 16-byte pieces when both maps allow
// it (`vec`: 16-byte aligned base and a pitch of a multiple of 4 floats on
// both sides).  One warp per row.  Block 0 adds the window's bytes to
// *bytes_in.
__global__ void __launch_bounds__(kWindowThreads) stage_window(const float *__restrict__ src, long long src_pitch,
                                                               int width, int height, int halo,
                                                               float *__restrict__ dst, long long dst_pitch,
                                                               int vec, const unsigned *win,
                                                               unsigned long long *bytes_in)
{
    const unsigned hi_i = win[1], hi_j = win[3];
    if (hi_i == 0)
        return;
    const int i0 = max((int)~win[0] - halo, 0) & ~3;
    const int i1 = min(min((int)(hi_i - 1u) + halo, width - 1) | 3, width - 1);
    const int j0 = max((int)~win[2] - halo, 0);
    const int j1 = min((int)(hi_j - 1u) + halo, height - 1);
    const int cols = i1 - i0 + 1, rows = j1 - j0 + 1;
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < rows; r += gridDim.x * warps) {
        const float *s = src + (long long)(j0 + r) * src_pitch + i0;
        float *d = dst + (long long)(j0 + r) * dst_pitch + i0;
        int c = 0;
        if (vec) {
            const int n4 = cols >> 2;
            const float4 *s4 = reinterpret_cast<const float4 *>(s);
            float4 *d4 = reinterpret_cast<float4 *>(d);
            int q = lane;
            for (; q + 32 < n4; q += 64) {
                const float4 a = s4[q], b = s4[q + 32];
                d4[q] = a;
                d4[q + 32] = b;
            }
            for (; q < n4; q += 32)
                d4[q] = s4[q];
            c = n4 << 2;
        }
        for (c += lane; c < cols; c += 32)
            d[c] = s[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(bytes_in, (unsigned long long)rows * (unsigned long long)cols * sizeof(float));
}

// ------------------------------------------------------------------ host --

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Slot {
    unsigned char *block = nullptr;   // one allocation per slot
    float *map = nullptr;
    float *x = nullptr, *y = nullptr, *z = nullptr, *sil = nullptr, *fil = nullptr;
    uint16_t *codes = nullptr;
    unsigned *win = nullptr;
    void *ws = nullptr;
    uint64_t tex = 0;                 // texture of `map` for (tex_w, tex_h, tex_pitch)
    int tex_w = 0, tex_h = 0;
    long long tex_pitch = 0;
    cudaEvent_t bounds_done = nullptr, in_done = nullptr, cmp_done = nullptr, free_ = nullptr;
    bool used = false;                // cmp_done / free_ recorded at least once
};

int host_plane(const void *p, const void **dev_view)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RBSM_ERR_ARG;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer)
        return RBSM_ERR_ARG;
    if (dev_view)
        *dev_view = at.devicePointer;
    return RBSM_OK;
}

}  // namespace
}  // namespace rbsm

struct rbsm_stager_s {
    rbsm_stager_desc desc;
    int device = 0;
    int n_slots = 0;
    long long plane_cap = 0;          // floats per plane in a slot
    long long map_pitch_align = 1;    // floats
    int sms = 1;
    rbsm::Slot slot[rbsm::kMaxSlots];
    cudaStream_t s_in = nullptr, s_win = nullptr, s_cmp = nullptr, s_out = nullptr;
    cudaEvent_t start = nullptr, end = nullptr;
    unsigned long long *window_bytes = nullptr;   // device counter
    long long host_bytes_in = 0, bytes_out = 0;
    unsigned long long next = 0;      // slot of the next map
};

namespace rbsm {
namespace {

void release(rbsm_stager_s *st)
{
    for (int k = 0; k < kMaxSlots; ++k) {
        Slot &s = st->slot[k];
        if (s.tex)
            rbsm_map_texture_destroy(s.tex);
        if (s.block)
            cudaFree(s.block);
        if (s.bounds_done)
            cudaEventDestroy(s.bounds_done);
        if (s.in_done)
            cudaEventDestroy(s.in_done);
        if (s.cmp_done)
            cudaEventDestroy(s.cmp_done);
        if (s.free_)
            cudaEventDestroy(s.free_);
    }
    if (st->window_bytes)
        cudaFree(st->window_bytes);
    for (cudaStream_t s : {st->s_in, st->s_win, st->s_cmp, st->s_out})
        if (s)
            cudaStreamDestroy(s);
    for (cudaEvent_t e : {st->start, st->end})
        if (e)
            cudaEventDestroy(e);
    delete st;
}

// The slot's texture for a map of this shape (created on first use; a new
// shape waits for the slot's last kernel before the old texture goes).
int slot_texture(Slot &s, int w, int h, long long pitch, uint64_t *tex)
{
    if (s.tex && s.tex_w == w && s.tex_h == h && s.tex_pitch == pitch) {
        *tex = s.tex;
        return RBSM_OK;
    }
    if (s.tex) {
        if (s.used) {
            cudaError_t e = cudaEventSynchronize(s.cmp_done);
            if (e != cudaSuccess)
                return cuda_fail(e);
        }
        rbsm_map_texture_destroy(s.tex);
        s.tex = 0;
    }
    rbsm_map m{s.map, w, h, pitch, 0};
    int rc = rbsm_map_texture_create(&m, &s.tex);
    if (rc != RBSM_OK) {
        s.tex = 0;
        *tex = 0;             // the device refused: plain loads (same answers)
        return rc == RBSM_ERR_ARG ? RBSM_OK : rc;
    }
    s.tex_w = w;
    s.tex_h = h;
    s.tex_pitch = pitch;
    *tex = s.tex;
    return RBSM_OK;
}

#define RBSM_CK(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess)                          \
            return cuda_fail(e_);                       \
    } while (0)

// Enqueue one map: its jobs are jobs[idx[0..count)] of the batch.
int run_map(rbsm_stager_s *st, const rbsm_batch *b, int map_index, const int *idx, int count,
            const void *map_view)
{
    const rbsm_map &hm = b->maps[map_index];
    const int k = (int)(st->next++ % (unsigned long long)st->n_slots);
    Slot &s = st->slot[k];
    int max_dist = 0;
    int rc = check_params(&b->params, &max_dist);
    if (rc != RBSM_OK)
        return rc;
    const long long pitch = (long long)align_up((size_t)hm.width, (size_t)st->map_pitch_align);

    // in: fragment planes, texel bounds, map window
    RBSM_CK(cudaStreamWaitEvent(st->s_in, s.free_, 0));
    long long off[RBSM_BATCH_MAX_JOBS];
    long long at = 0;
    for (int q = 0; q < count; ++q) {
        const rbsm_job &j = b->jobs[idx[q]];
        const size_t bytes = (size_t)j.frags.n * sizeof(float);
        off[q] = at;
        at += (long long)align_up((size_t)j.frags.n, (size_t)kJobAlign);
        RBSM_CK(cudaMemcpyAsync(s.x + off[q], j.frags.x, bytes, cudaMemcpyHostToDevice, st->s_in));
        RBSM_CK(cudaMemcpyAsync(s.y + off[q], j.frags.y, bytes, cudaMemcpyHostToDevice, st->s_in));
        RBSM_CK(cudaMemcpyAsync(s.z + off[q], j.frags.z, bytes, cudaMemcpyHostToDevice, st->s_in));
        st->host_bytes_in += 3 * (long long)bytes;
    }
    RBSM_CK(cudaMemsetAsync(s.win, 0, 4 * sizeof(unsigned), st->s_in));
    for (int q = 0; q < count; ++q) {
        const long long n = b->jobs[idx[q]].frags.n;
        long long blocks = (n + 4LL * kBoundsThreads - 1) / (4LL * kBoundsThreads);
        if (blocks > 8LL * st->sms)
            blocks = 8LL * st->sms;
        texel_bounds<<<(unsigned)blocks, kBoundsThreads, 0, st->s_in>>>(s.x + off[q], s.y + off[q], n, hm.width,
                                                                        hm.height, s.win);
        RBSM_CK(cudaGetLastError());
    }
    // the window copy runs on its own stream, beside the next map's
    // fragment copies
    RBSM_CK(cudaEventRecord(s.bounds_done, st->s_in));
    RBSM_CK(cudaStreamWaitEvent(st->s_win, s.bounds_done, 0));
    const int vec = (reinterpret_cast<uintptr_t>(map_view) & 15u) == 0 && hm.pitch % 4 == 0 && pitch % 4 == 0;
    stage_window<<<(unsigned)(2 * st->sms), kWindowThreads, 0, st->s_win>>>(
        static_cast<const float *>(map_view), hm.pitch, hm.width, hm.height, max_dist + 1, s.map, pitch, vec, s.win,
        st->window_bytes);
    RBSM_CK(cudaGetLastError());
    RBSM_CK(cudaEventRecord(s.in_done, st->s_win));

    // kernel: the batch of this map's jobs on the staged copies
    uint64_t tex = 0;
    if (st->desc.texture && (rc = slot_texture(s, hm.width, hm.height, pitch, &tex)) != RBSM_OK)
        return rc;
    rbsm_map dm{s.map, hm.width, hm.height, pitch, tex};
    rbsm_job dj[RBSM_BATCH_MAX_JOBS];
    for (int q = 0; q < count; ++q) {
        const rbsm_job &j = b->jobs[idx[q]];
        dj[q].map = 0;
        dj[q].mode = j.mode;
        dj[q].frags = rbsm_frags{s.x + off[q], s.y + off[q], s.z + off[q], j.frags.n};
        dj[q].vis_silhouette = (j.mode & 1) ? s.sil + off[q] : nullptr;
        dj[q].vis_filter = (j.mode & 2) ? s.fil + off[q] : nullptr;
        dj[q].codes = j.codes ? s.codes + off[q] : nullptr;
    }
    rbsm_batch db = *b;
    db.maps = &dm;
    db.n_maps = 1;
    db.jobs = dj;
    db.n_jobs = count;
    static thread_local BatchArgs args;
    int threads = 0;
    if ((rc = prepare_batch(&db, args, &threads)) != RBSM_OK)
        return rc;
    bind_workspace(args, s.ws);
    LaunchShape sh;
    if ((rc = launch_shape(args, threads, db.ctas_per_sm, db.chunk_tiles, &sh)) != RBSM_OK)
        return rc;
    RBSM_CK(cudaStreamWaitEvent(st->s_cmp, s.in_done, 0));
    if ((rc = enqueue_batch(args, sh, s.ws, st->s_cmp)) != RBSM_OK)
        return rc;
    RBSM_CK(cudaEventRecord(s.cmp_done, st->s_cmp));

    // out: the answers
    RBSM_CK(cudaStreamWaitEvent(st->s_out, s.cmp_done, 0));
    for (int q = 0; q < count; ++q) {
        const rbsm_job &j = b->jobs[idx[q]];
        const size_t n = (size_t)j.frags.n;
        if (j.mode & 1) {
            RBSM_CK(cudaMemcpyAsync(j.vis_silhouette, s.sil + off[q], n * sizeof(float), cudaMemcpyDeviceToHost,
                                    st->s_out));
            st->bytes_out += (long long)(n * sizeof(float));
        }
        if (j.mode & 2) {
            RBSM_CK(cudaMemcpyAsync(j.vis_filter, s.fil + off[q], n * sizeof(float), cudaMemcpyDeviceToHost,
                                    st->s_out));
            st->bytes_out += (long long)(n * sizeof(float));
        }
        if (j.codes) {
            RBSM_CK(cudaMemcpyAsync(j.codes, s.codes + off[q], n * sizeof(uint16_t), cudaMemcpyDeviceToHost,
                                    st->s_out));
            st->bytes_out += (long long)(n * sizeof(uint16_t));
        }
    }
    RBSM_CK(cudaEventRecord(s.free_, st->s_out));
    s.used = true;
    return RBSM_OK;
}

// Arguments of a run: the batch checks of rbsm_batch_run, then the stager's
// own (no map textures, sizes within the slots, page-locked host planes).
// Fills the device view of every map.
int check_run(const rbsm_stager_s *st, const rbsm_batch *b, const void **map_view)
{
    static thread_local BatchArgs args;
    int threads = 0;
    int rc = prepare_batch(b, args, &threads);
    if (rc != RBSM_OK)
        return rc;
    long long per_map[RBSM_BATCH_MAX_MAPS] = {};      // fragments of each map's jobs
    long long padded[RBSM_BATCH_MAX_MAPS] = {};       // the same with the slot's job alignment
    for (int m = 0; m < b->n_maps; ++m) {
        const rbsm_map &hm = b->maps[m];
        if (hm.texture || hm.width > st->desc.max_width || hm.height > st->desc.max_height)
            return RBSM_ERR_ARG;
        map_view[m] = nullptr;
    }
    for (int k = 0; k < b->n_jobs; ++k) {
        const rbsm_job &j = b->jobs[k];
        if (j.frags.n == 0)
            continue;
        per_map[j.map] += j.frags.n;
        padded[j.map] += (long long)align_up((size_t)j.frags.n, (size_t)kJobAlign);
        if (per_map[j.map] > st->desc.max_fragments || padded[j.map] > st->plane_cap)
            return RBSM_ERR_ARG;
        const void *planes[6] = {j.frags.x, j.frags.y, j.frags.z, (j.mode & 1) ? j.vis_silhouette : nullptr,
                                 (j.mode & 2) ? j.vis_filter : nullptr, j.codes};
        for (const void *p : planes)
            if (p && (rc = host_plane(p, nullptr)) != RBSM_OK)
                return rc;
        if (!map_view[j.map] && (rc = host_plane(b->maps[j.map].depth, &map_view[j.map])) != RBSM_OK)
            return rc;
    }
    return RBSM_OK;
}

}  // namespace
}  // namespace rbsm

extern "C" {

int rbsm_stager_create(const rbsm_stager_desc *desc, rbsm_stager *out)
{
    using namespace rbsm;
    if (!desc || !out)
        return RBSM_ERR_ARG;
    *out = nullptr;
    const int slots = desc->slots == 0 ? kDefaultSlots : desc->slots;
    if (desc->max_fragments < 1 || desc->max_fragments > RBSM_MAX_FRAGMENTS || desc->max_width < 1 ||
        desc->max_width > RBSM_MAX_EXTENT || desc->max_height < 1 || desc->max_height > RBSM_MAX_EXTENT ||
        slots < 2 || slots > kMaxSlots || (desc->texture != 0 && desc->texture != 1) || desc->flags != 0)
        return RBSM_ERR_ARG;
    auto *st = new rbsm_stager_s();
    st->desc = *desc;
    st->n_slots = slots;
    auto fail = [&](cudaError_t e) {
        release(st);
        return cuda_fail(e);
    };
    cudaError_t e = cudaGetDevice(&st->device);
    if (e != cudaSuccess)
        return fail(e);
    int pitch_align = 0;
    if ((e = cudaDeviceGetAttribute(&pitch_align, cudaDevAttrTexturePitchAlignment, st->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&st->sms, cudaDevAttrMultiProcessorCount, st->device)) != cudaSuccess)
        return fail(e);
    // device map pitch: the texture pitch alignment, and at least 4 floats
    // (16-byte rows for the window copy)
    st->map_pitch_align = pitch_align > 16 ? pitch_align / 4 : 4;
    // plane capacity: max_fragments plus the alignment gap of every job
    st->plane_cap = (long long)align_up((size_t)desc->max_fragments, (size_t)kJobAlign) +
                    (long long)kJobAlign * RBSM_BATCH_MAX_JOBS;
    const size_t plane = align_up((size_t)st->plane_cap * sizeof(float), kSubAlign);
    const size_t codes = align_up((size_t)st->plane_cap * sizeof(uint16_t), kSubAlign);
    const size_t map = align_up((size_t)desc->max_height *
                                    align_up((size_t)desc->max_width, (size_t)st->map_pitch_align) * sizeof(float),
                                kSubAlign);
    const size_t small = align_up(4 * sizeof(unsigned), 256) + align_up(kWorkspaceBytes, 256);
    const size_t total = map + 5 * plane + codes + small;
    for (int k = 0; k < slots; ++k) {
        Slot &s = st->slot[k];
        if ((e = cudaMalloc(&s.block, total)) != cudaSuccess)
            return fail(e);
        unsigned char *p = s.block;
        s.map = reinterpret_cast<float *>(p);            // first: the texture base alignment
        p += map;
        float **planes[5] = {&s.x, &s.y, &s.z, &s.sil, &s.fil};
        for (float **q : planes) {
            *q = reinterpret_cast<float *>(p);
            p += plane;
        }
        s.codes = reinterpret_cast<uint16_t *>(p);
        p += codes;
        s.win = reinterpret_cast<unsigned *>(p);
        p += align_up(4 * sizeof(unsigned), 256);
        s.ws = p;
        if ((e = cudaEventCreateWithFlags(&s.bounds_done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.cmp_done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.free_, cudaEventDisableTiming)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemset(s.ws, 0, kWorkspaceBytes)) != cudaSuccess)
            return fail(e);
    }
    if ((e = cudaMalloc(&st->window_bytes, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(st->window_bytes, 0, sizeof(unsigned long long))) != cudaSuccess)
        return fail(e);
    if ((e = cudaStreamCreateWithFlags(&st->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&st->s_win, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&st->s_cmp, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&st->s_out, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&st->start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&st->end, cudaEventDisableTiming)) != cudaSuccess)
        return fail(e);
    // every slot starts free: record its events once, in order
    for (int k = 0; k < slots; ++k)
        if ((e = cudaEventRecord(st->slot[k].free_, st->s_out)) != cudaSuccess)
            return fail(e);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess)
        return fail(e);
    *out = st;
    return RBSM_OK;
}

int rbsm_stager_run(rbsm_stager st, const rbsm_batch *batch, void *stream)
{
    using namespace rbsm;
    if (!st)
        return RBSM_ERR_ARG;
    const void *map_view[RBSM_BATCH_MAX_MAPS];
    int rc = check_run(st, batch, map_view);
    if (rc != RBSM_OK)
        return rc;
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    RBSM_CK(cudaEventRecord(st->start, caller));
    RBSM_CK(cudaStreamWaitEvent(st->s_in, st->start, 0));
    int idx[RBSM_BATCH_MAX_JOBS];
    for (int m = 0; m < batch->n_maps; ++m) {
        int count = 0;
        for (int k = 0; k < batch->n_jobs; ++k)
            if (batch->jobs[k].map == m && batch->jobs[k].frags.n > 0)
                idx[count++] = k;
        if (count == 0)
            continue;
        if ((rc = run_map(st, batch, m, idx, count, map_view[m])) != RBSM_OK)
            return rc;
    }
    // the caller's stream resumes after the last copy out (and, through the
    // events each stream waited on, after everything else of this run)
    RBSM_CK(cudaStreamWaitEvent(st->s_out, st->start, 0));
    RBSM_CK(cudaEventRecord(st->end, st->s_out));
    RBSM_CK(cudaStreamWaitEvent(caller, st->end, 0));
    return RBSM_OK;
}

int rbsm_stager_stats(rbsm_stager st, int64_t *bytes_in, int64_t *bytes_out)
{
    using namespace rbsm;
    if (!st || !bytes_in || !bytes_out)
        return RBSM_ERR_ARG;
    for (cudaStream_t s : {st->s_in, st->s_win, st->s_cmp, st->s_out})
        RBSM_CK(cudaStreamSynchronize(s));
    unsigned long long w = 0;
    RBSM_CK(cudaMemcpy(&w, st->window_bytes, sizeof w, cudaMemcpyDeviceToHost));
    *bytes_in = st->host_bytes_in + (int64_t)w;
    *bytes_out = st->bytes_out;
    return RBSM_OK;
}

int rbsm_stager_status(rbsm_stager st, int *status)
{
    using namespace rbsm;
    if (!st || !status)
        return RBSM_ERR_ARG;
    for (cudaStream_t s : {st->s_in, st->s_win, st->s_cmp, st->s_out})
        RBSM_CK(cudaStreamSynchronize(s));
    *status = RBSM_OK;
    for (int k = 0; k < st->n_slots; ++k) {
        int v = 0;
        RBSM_CK(cudaMemcpy(&v, static_cast<char *>(st->slot[k].ws) + 8, sizeof v, cudaMemcpyDeviceToHost));
        if (v != RBSM_OK && *status == RBSM_OK)
            *status = v;
    }
    return RBSM_OK;
}

int rbsm_stager_destroy(rbsm_stager st)
{
    using namespace rbsm;
    if (!st)
        return RBSM_ERR_ARG;
    cudaError_t first = cudaSuccess;
    for (cudaStream_t s : {st->s_in, st->s_win, st->s_cmp, st->s_out}) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (first == cudaSuccess)
            first = e;
    }
    release(st);
    return first == cudaSuccess ? RBSM_OK : cuda_fail(first);
}

}  // extern "C"
