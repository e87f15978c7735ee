/*
 * rbsm.h - C ABI of the GB300 revectorization-based shadow mapping (RBSM)
 * library: the per-fragment visibility of Macedo, Apolinario and Aguero,
 * "Optimized Visibility Functions for Revectorization-Based Shadow Mapping"
 * (TR-PGCOMP-007/2017).
 *
 * The problem as the paper states it (Listing 1, §3): a shadow map SM of
 * SMWIDTH x SMHEIGHT depths rendered from the light, a fragment p = (x, y, z)
 * in light space (x, y texture coordinates, z the fragment's depth as seen
 * from the light), the traversal cap MAXDIST (Listing 3, §3.1.3) and the
 * choice between silhouette recovery and filtering.  Each fragment's answer
 * is a visibility in [0, 1]: 1 lit, 0 shadowed (Eq. 1).
 *
 * Conventions shared by every entry point
 *   - Every data pointer is a DEVICE pointer into memory the caller owns
 *     (cudaMalloc, a torch tensor, ...).  The library never frees, keeps or
 *     allocates memory during a call, and never synchronises the stream: it
 *     enqueues work on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and returns.  Results are ready when that stream reaches them.
 *   - Shadow map: row-major float32, row j holds the texels with texture
 *     coordinate y in [j/height, (j+1)/height); texel (i, j) is at
 *     depth[j * pitch + i].  Lookups use the nearest texel, i = floor(x *
 *     width) formed in float32, and clamp to the edge outside the map.
 *   - Fragments: three float32 planes x[n], y[n], z[n] (structure of arrays).
 *     Any 4-byte alignment is accepted; 16-byte aligned planes and outputs
 *     take the vectorised path.
 *   - Outputs must not overlap the inputs: an edge fragment's coordinates
 *     are read again after the answers of its tile have been stored.  The
 *     single-map calls and rbsm_rpcf refuse an output that overlaps their
 *     fragment planes or map (RBSM_ERR_ARG).
 *   - Codes (optional uint16 per fragment):
 *       bits 0-3  discontinuity directions of Eq. 3: left, right, +y, -y
 *                 (+y = next row index)
 *       bit  4    d.z of Eq. 4: the fragment's own shadow test failed
 *       bits 5-6  number of edge ends the traversal found along x (0..2)
 *       bits 7-8  number of edge ends found along y (0..2)
 *       bit  9    the fragment went through the edge traversal
 *     The Eq. 5 code of an axis is (ends - 1).
 *   - Return value: RBSM_OK, or a negative RBSM_ERR_* code.  On an error
 *     nothing is enqueued unless the error is RBSM_ERR_CUDA, which means a
 *     launch failed; rbsm_last_cuda_error() then gives the CUDA error number.
 *
 * Floating point: depth comparisons, discontinuity codes and the silhouette
 * decision are exact float32 operations identical to the paper's GLSL
 * arithmetic; the normalised distances use one correctly rounded float32
 * add and divide per axis (no fast-math, no contraction).
 */
#ifndef RBSM_H
#define RBSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RBSM_OK 0
#define RBSM_ERR_ARG (-1)          /* a NULL pointer, a size out of range, a bad mode */
#define RBSM_ERR_CUDA (-2)         /* a CUDA call failed; see rbsm_last_cuda_error() */
#define RBSM_ERR_TIMEOUT (-3)      /* a bounded device-side wait gave up (the tensor-core
                                      surrogate kernels wait at most 1 s for their products;
                                      rbsm_mlp_read reports it) */
#define RBSM_ERR_WORKSPACE (-4)    /* workspace missing, too small or misaligned */

#define RBSM_MODE_SILHOUETTE 1     /* Listing 4, §4.1: hard shadows, revectorised */
#define RBSM_MODE_FILTER 2         /* Listing 5, §4.2: fake penumbra (RSMSS) */
#define RBSM_MODE_BOTH 3           /* both answers from one pass over the fragments */

#define RBSM_MAXDIST_DEFAULT 16    /* §3.1.3: the value the paper used */
#define RBSM_MAXDIST_LIMIT 255
#define RBSM_MAX_EXTENT 65536      /* width and height limit of a shadow map */
#define RBSM_MAX_FRAGMENTS 2147483647LL   /* fragments per fragment set (rbsm_frags.n) */

/* A shadow map (device memory, owned by the caller). */
typedef struct {
    const float *depth;
    int32_t width;
    int32_t height;
    int64_t pitch;                 /* floats between rows, >= width */
    uint64_t texture;              /* optional, 0 = none: a texture of this map from
                                    * rbsm_map_texture_create; when given, the four-
                                    * neighbourhood is read with two texture gathers */
} rbsm_map;

/*
 * Texture view of a shadow map for faster neighbourhood reads: a
 * cudaTextureObject_t over the map's own memory (no copy) with point
 * sampling, clamp-to-edge addressing and unnormalised coordinates, so two
 * 2x2 texture gathers return the fragment's texel and its four neighbours
 * (Listing 2) with the clamp of R2 done by the texture unit.  Answers are
 * identical with and without it.  Creation is a set-up call (it creates a
 * driver object, no device memory); destroy the texture with
 * rbsm_map_texture_destroy once every launch that reads it has completed.
 * Errors: RBSM_ERR_ARG for an invalid map, or for a base address or pitch
 * that the device's texture alignment rules reject (use the map without a
 * texture then); RBSM_ERR_CUDA when the driver refuses.
 */
int rbsm_map_texture_create(const rbsm_map *map, uint64_t *texture);
int rbsm_map_texture_destroy(uint64_t texture);

/* A set of light-space fragments (device memory, owned by the caller). */
typedef struct {
    const float *x;
    const float *y;
    const float *z;
    int64_t n;                     /* 0..RBSM_MAX_FRAGMENTS; n == 0 enqueues nothing */
} rbsm_frags;

typedef struct {
    int32_t max_dist;              /* MAXDIST of Listing 3, 1..RBSM_MAXDIST_LIMIT */
    int32_t flags;                 /* 0; rbsm_mlp_dataset also takes RBSM_DATASET_IN_WINDOW */
} rbsm_params;

/* rbsm_mlp_dataset: keep only edge fragments whose Listing 3 walks stop
 * inside the 5x5 window (the fragments the batch's surrogate may answer). */
#define RBSM_DATASET_IN_WINDOW 1

/*
 * Silhouette recovery (Listing 1 with Listings 2-4; §3.1 and §4.1).
 * For every fragment: shadow test (Eq. 1); shadowed fragments stay at 0;
 * lit fragments with a discontinuity (Eqs. 2-4) walk the shadow edge in the
 * four directions (Listing 3), normalise their position inside it (Eq. 5)
 * and take the optimized silhouette visibility: 0 in U and O shapes, 1 in I
 * shapes, and for L shapes 0 below the revectorisation line
 * nrd.y = 1 - nrd.x, 1 on or above it.
 *   map, frags, params: inputs (params NULL = MAXDIST 16).
 *   vis:   output, n floats, each 0.0 or 1.0.
 *   codes: optional output, n uint16 (see above); NULL to skip.
 * Errors: RBSM_ERR_ARG for NULL map/frags/vis, NULL planes with n > 0,
 * width or height outside 1..RBSM_MAX_EXTENT, pitch < width, n outside
 * 0..RBSM_MAX_FRAGMENTS,
 * max_dist outside 1..RBSM_MAXDIST_LIMIT, flags != 0; RBSM_ERR_CUDA when the
 * launch fails.
 */
int rbsm_visibility(const rbsm_map *map, const rbsm_frags *frags, float *vis,
                    uint16_t *codes, const rbsm_params *params, void *stream);

/*
 * Revectorization-based shadow filtering, RSMSS (Listing 1 with Listings 2,
 * 3 and 5; §3.2 and §4.2).  Every fragment with a discontinuity, on either
 * side of the edge, walks the edge and takes the optimized filtering
 * visibility: O shapes take the opposite of their shadow test, U shapes the
 * normalised distance along the open axis, I shapes the shadow test, L
 * shapes clamp(d.z +- nrd.x +- nrd.y, 0, 1); other fragments take the plain
 * shadow test.  Arguments and errors as for rbsm_visibility; vis holds
 * values in [0, 1].
 */
int rsmss_filter(const rbsm_map *map, const rbsm_frags *frags, float *vis,
                 uint16_t *codes, const rbsm_params *params, void *stream);

/*
 * Visibility straight from depth buffers: the fragment's light-space
 * position p (Listing 1's varying) is formed in the kernel instead of read.
 * Pixel (px, py) of a job's buffer holds depth d; (X, Y, Z, W) =
 * m (px + 0.5, py + 0.5, d, 1) with m its row-major 4 x 4
 * screen-to-light-clip matrix, each row summed left to right in float32,
 * and p = (X / W, Y / W, Z / W).  Fragment f = py * width + px then goes
 * through the path of rbsm_visibility / rsmss_filter against the job's map:
 * the answers are those of those calls on the projected planes, bit for
 * bit, and 4 bytes per fragment are read instead of 12.  Every job is
 * checked before the first launch; then each job runs as one launch, in
 * order, on `stream`.  When no job's outputs overlap another job's outputs
 * or any job's inputs (depth buffer, map), each job after the first is a
 * programmatic dependent launch: it takes SMs as the previous job's kernel
 * drains instead of after it ends.  Work after the call on `stream` still
 * follows all of them.  The kernels signal their dependents at their
 * start, so a caller's own programmatic dependent of this call must wait
 * for it (cudaGridDependencySynchronize) before reading its outputs.
 *   jobs: n_jobs (1..RBSM_GBUFFER_MAX_JOBS) descriptors, copied into the
 *   launch; mode: RBSM_MODE_SILHOUETTE, _FILTER or _BOTH for every job;
 *   vis_silhouette / vis_filter: width * height floats each as the mode
 *   asks; codes: width * height uint16 (filter-mode codes for BOTH), given
 *   for every job or for none.
 * Errors: RBSM_ERR_ARG as for rbsm_visibility for each map, for a NULL or
 * invalid depth buffer (width, height outside 1..RBSM_MAX_EXTENT,
 * pitch < width), a bad mode or job count, a missing output or codes given
 * for some jobs only; RBSM_ERR_CUDA when the launch fails.
 */
typedef struct {
    const float *depth;            /* device, height rows of width floats */
    int32_t width;
    int32_t height;
    int64_t pitch;                 /* floats between rows, >= width */
    float m[16];                   /* row-major screen-to-light-clip matrix */
} rbsm_gbuffer;

typedef struct {
    rbsm_map map;
    rbsm_gbuffer gbuffer;
    float *vis_silhouette;
    float *vis_filter;
    uint16_t *codes;
} rbsm_gbuffer_job;

#define RBSM_GBUFFER_MAX_JOBS 64
int rbsm_visibility_gbuffer(const rbsm_gbuffer_job *jobs, int32_t n_jobs, int32_t mode,
                            const rbsm_params *params, void *stream);

/*
 * RPCF: percentage-closer filtering over the RSMSS answer (§5.3: the
 * skeleton artifacts along filtered edges are suppressed with PCF; the
 * paper prints no kernel for it).  For every fragment: the mean of the
 * Listing 5 (RSMSS) answers of the k x k samples at its texel-space
 * position (x W, y H), shifted by whole texels (u + a, v + b) for a, b in
 * -(k-1)/2 .. (k-1)/2 (float32 adds), each with the fragment's depth,
 * summed with b outer and a inner.  k = 1 is rsmss_filter itself.
 *   k: odd, 1..RBSM_RPCF_MAX_K.  vis: output, n floats in [0, 1]; while
 *   the call runs it also holds the pending fragments' partial sums, so it
 *   must not overlap the fragment planes or the map.
 * For k > 1 the sample answers are added in fixed point, each rounded to
 * 2^-24, 2^-22 or 2^-20 (k = 3, 5, 7), so a result does not depend on the
 * order in which a fragment's samples are finished and lies within
 * k^2 * 2^-(F+1) of the exact mean of the sample answers.
 * Errors as for rsmss_filter, and RBSM_ERR_ARG for an even or out-of-range k.
 */
#define RBSM_RPCF_MAX_K 7
int rbsm_rpcf(const rbsm_map *map, const rbsm_frags *frags, float *vis, int32_t k,
              const rbsm_params *params, void *stream);

/*
 * rbsm_rpcf with an 8-byte device workspace (8-byte aligned, owned by the
 * caller, used by one call at a time: calls that overlap on the GPU need
 * workspaces of their own).  The answers are those of rbsm_rpcf bit for
 * bit.  For k > 1 the call first zeroes the workspace on `stream`, and the
 * warps then take the tiles after their first one from that counter, one
 * tile per claim, instead of a fixed partition, so that warps whose tiles
 * carry many edge samples do not hold up the end of the launch.  For k = 1
 * the workspace is not used.  Errors as for rbsm_rpcf, and RBSM_ERR_ARG
 * for a NULL or unaligned workspace or one that overlaps vis or an input.
 */
int rbsm_rpcf_ws(const rbsm_map *map, const rbsm_frags *frags, float *vis, int32_t k,
                 const rbsm_params *params, void *workspace, void *stream);

/*
 * Batched evaluation: many shadow maps (lights, cascades) against many
 * fragment sets (views) in ONE persistent kernel launch.  Not in the paper,
 * which evaluates one map per shader pass; every job's answers are
 * bit-identical to the single-map calls above on the same inputs.
 */
#define RBSM_BATCH_MAX_MAPS 64
#define RBSM_BATCH_MAX_JOBS 256

typedef struct {
    int32_t map;                   /* index into rbsm_batch.maps */
    int32_t mode;                  /* RBSM_MODE_SILHOUETTE / _FILTER / _BOTH */
    rbsm_frags frags;
    float *vis_silhouette;         /* n floats; required when mode has SILHOUETTE */
    float *vis_filter;             /* n floats; required when mode has FILTER */
    uint16_t *codes;               /* optional; filter-mode codes when mode is BOTH */
} rbsm_job;

typedef struct {
    const rbsm_map *maps;          /* host array of n_maps descriptors */
    int32_t n_maps;                /* 1..RBSM_BATCH_MAX_MAPS */
    const rbsm_job *jobs;          /* host array of n_jobs descriptors */
    int32_t n_jobs;                /* 1..RBSM_BATCH_MAX_JOBS */
    rbsm_params params;
    int32_t tile_threads;          /* CTA size: 128, 256 or 512 threads; 0 = default 256 */
    int32_t ctas_per_sm;           /* persistent CTAs per SM, 1..8; 0 = occupancy limit.  At
                                    * 256 threads the exact path has variants compiled for 3, 4
                                    * and 5 CTAs per SM (80, 64, 48 registers per thread): 3
                                    * selects the first, 1, 2 and 4 the second, 5 and up and 0
                                    * the third */
    /* Learned penumbra (not in the paper): NULL = exact everywhere.  Given a
     * network state block (rbsm_mlp_state_bytes), FILTER-mode jobs answer
     * an edge fragment with the surrogate when (1) its four Listing 3 walks
     * stop inside the 5x5 window the network sees (read from the window's
     * shadow-test pattern; otherwise the exact answer depends on texels the
     * network cannot see), (2) its pattern is trusted (rbsm_mlp_set_trust;
     * all are when no bitmap is in force) and (3) the network's own error
     * estimate is <= guard_tau (0 <= guard_tau < 1e30); every other edge
     * fragment falls back to the exact walk;
     * shadow tests, discontinuity codes and off-edge answers stay exact, and
     * SILHOUETTE / BOTH jobs are not touched.  A surrogate answer's code has
     * bit 10 set and no end counts (bits 5-9 clear). */
    const void *surrogate;
    float guard_tau;
    int32_t chunk_tiles;           /* 128-fragment warp tiles a warp claims at a time from the
                                    * work counter: 1, 2, 4 or 8; 0 = chosen from the batch size
                                    * (8 when every warp gets about eight claims, halved below) */
    int32_t flags;                 /* 0 or RBSM_BATCH_PLAIN_LOADS */
} rbsm_batch;

/* rbsm_batch.flags: read the four-neighbourhood with plain loads even where
 * a map carries a texture (answers are the same bits either way). */
#define RBSM_BATCH_PLAIN_LOADS 1

/*
 * Device workspace a batch needs (a work counter and a status word), in
 * bytes; the caller allocates it (256-byte aligned) and may reuse it for any
 * later batch that is not in flight at the same time.
 */
int rbsm_batch_workspace_size(const rbsm_batch *batch, size_t *bytes);

/*
 * Enqueue one batched launch: a memset of the workspace followed by one
 * persistent kernel whose warps take chunks of 1 to 8 tiles of 128
 * fragments (in job order; the chunk is as large as leaves every warp
 * about eight claims) from an atomic counter in the workspace.
 * The descriptors are copied into the launch parameters, so the host arrays
 * may be reused as soon as the call returns.  Errors: RBSM_ERR_ARG as for
 * rbsm_visibility applied to every map and job, or a map index out of range;
 * RBSM_ERR_WORKSPACE for a NULL, small or misaligned workspace;
 * RBSM_ERR_CUDA when a launch fails.
 */
int rbsm_batch_run(const rbsm_batch *batch, void *workspace, size_t workspace_bytes, void *stream);

/*
 * rbsm_batch_run without a workspace argument, for callers that cannot
 * allocate device memory: a plugin running inside a host application that
 * owns every device allocation, or a frame loop with a fixed memory footprint
 * that must not allocate while frames are in flight.  The paper has no
 * counterpart; this is a convenience of the library.
 *
 * The scratch rbsm_batch_run keeps in the caller's workspace (work counter,
 * status word, surrogate counters) lives instead in one device array
 * compiled into the library, RBSM_NOALLOC_SCRATCH_BYTES bytes, which every
 * GPU that loads the library holds until the process exits.  The call
 * allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine): it clears the counters with a stream-ordered memset and
 * launches the same kernel as rbsm_batch_run, so its answers are the same.
 *
 * The first call on each device looks up the array's device address (with
 * that device current), so make that first call before any stream capture
 * on the calling thread.  Every call shares the one array and the array
 * keeps the last call's contents: calls whose work overlaps on the GPU
 * (other streams, other threads) race on it, so order them on one stream
 * or use rbsm_batch_run with separate workspaces.  A batch whose workspace
 * (rbsm_batch_workspace_size) exceeds the array is rejected with
 * RBSM_ERR_WORKSPACE; other errors as for rbsm_batch_run.
 */
#define RBSM_NOALLOC_SCRATCH_BYTES 256
int rbsm_batch_run_noalloc(const rbsm_batch *batch, void *stream);

/* The surrogate counters (as rbsm_batch_surrogate_counts) of the last
 * rbsm_batch_run_noalloc launch on the current device, read from the
 * library's array once the stream has completed it (synchronous
 * device-to-host copy); RBSM_ERR_CUDA when no call has run on the device. */
int rbsm_batch_noalloc_counts(uint64_t *accepted, uint64_t *fallback);

/*
 * CUDA graph of one batched launch (the workspace memset and the persistent
 * kernel), built once and replayed with one cudaGraphLaunch per frame.  The
 * graph captures the descriptors, the device pointers and the workspace as
 * they are at creation: replaying it reads whatever those buffers then hold.
 * Creation allocates the graph (host and driver resources) and must not run
 * while the calling thread captures a stream; launching allocates nothing.
 * Errors as for rbsm_batch_run; rbsm_batch_graph_launch returns RBSM_ERR_ARG
 * for a NULL graph and RBSM_ERR_CUDA when the launch fails.
 */
typedef struct rbsm_graph_s *rbsm_graph;
int rbsm_batch_graph_create(const rbsm_batch *batch, void *workspace, size_t workspace_bytes,
                            rbsm_graph *graph);
int rbsm_batch_graph_launch(rbsm_graph graph, void *stream);
int rbsm_batch_graph_destroy(rbsm_graph graph);

/*
 * Autotuner of the batched launch.  Times every combination of
 *   - 7 (CTA size, CTAs per SM) pairs: 128 threads at its occupancy limit;
 *     256 threads at 2, 3, 4 and 5 (occupancy limit) CTAs per SM; 512
 *     threads at 1 and 2;
 *   - 4 claim sizes: 1, 2, 4 and 8 warp tiles per claim of the work counter;
 *   - when any map carries a texture: texture gathers or plain loads for the
 *     four-neighbourhood;
 * with `repeats` launches each after one warm-up, on `stream`, and returns
 * the fastest in *best (apply it through tile_threads, ctas_per_sm,
 * chunk_tiles and flags).  Every warp works on its own 128-fragment tiles
 * whatever the CTA size.  It writes the batch's outputs (the answers stay
 * correct) and waits for the stream (cudaEventSynchronize): a set-up call,
 * not for a frame loop.
 */
typedef struct {
    int32_t tile_threads;
    int32_t ctas_per_sm;           /* 0 = occupancy limit */
    float ms;                      /* mean time per launch of the winner */
    int32_t candidates;            /* combinations timed */
    int32_t chunk_tiles;           /* claim size of the winner */
    int32_t flags;                 /* RBSM_BATCH_PLAIN_LOADS when plain loads won */
} rbsm_tuning;
int rbsm_batch_autotune(const rbsm_batch *batch, void *workspace, size_t workspace_bytes, void *stream,
                        int32_t repeats, rbsm_tuning *best);

/*
 * After the stream has completed a batch: the number of edge fragments the
 * surrogate answered and the number it handed to the exact walk (guard
 * tripped) in its last launch (synchronous device-to-host copy).
 */
int rbsm_batch_surrogate_counts(const void *workspace, uint64_t *accepted, uint64_t *fallback);

/*
 * After the stream has completed a batch: read its device status word
 * (synchronously, with a device-to-host copy) into *status.  The word is
 * cleared before every launch and reserved: the batched kernel has no wait
 * and no condition to record (every argument is checked on the host before
 * the launch), so it reads RBSM_OK.
 */
int rbsm_batch_status(const void *workspace, int *status);

/*
 * Shadow maps of analytic occluders: the light pass that produces SM, the
 * input of Listing 1 (the paper rasterises it with the graphics pipeline;
 * this library writes it with a CUDA kernel, for maps generated per frame).
 * An orthographic light looks down the depth axis; texel (i, j) point-
 * samples (i + 0.5, j + 0.5) and stores the smallest depth of the occluders
 * covering that point, else `ground`:
 *   rectangle: with p = point - (cx, cy), covered when |p . (ux, uy)| <= ha
 *     and |p . (-uy, ux)| <= hb; its depth is `depth`;
 *   sphere: covered when |p|^2 <= radius^2 (p from its centre); depth
 *     centre_depth - sqrt(radius^2 - |p|^2) / zscale, rounded to float32.
 * Every operation is a separate IEEE double operation in the order written
 * (no fused multiply-add), so the map is bit-exact on any host.
 * Occluder arrays are device memory owned by the caller; depth is a device
 * map of width x height floats with `pitch` floats between rows.
 * Errors: RBSM_ERR_ARG for NULL pointers with counts > 0, counts < 0,
 * width or height outside 1..RBSM_MAX_EXTENT, pitch < width, zscale <= 0,
 * flags != 0; RBSM_ERR_CUDA when the launch fails.
 */
typedef struct {
    double cx, cy;                 /* centre, texel units */
    double ux, uy;                 /* axis (unit length) */
    double ha, hb;                 /* half extents along and across the axis */
    float depth;
    float reserved;                /* 0 */
} rbsm_rect;

typedef struct {
    double cx, cy, radius;         /* texel units */
    double centre_depth;
} rbsm_sphere;

typedef struct {
    const rbsm_rect *rects;
    int32_t n_rects;
    const rbsm_sphere *spheres;
    int32_t n_spheres;
    double zscale;                 /* depth units per texel for the sphere caps */
    float ground;                  /* depth of a texel nothing covers */
    int32_t flags;                 /* reserved, 0 */
} rbsm_occluders;

int rbsm_shadow_map(const rbsm_occluders *occ, float *depth, int32_t width, int32_t height, int64_t pitch,
                    void *stream);

/*
 * n_maps (1..RBSM_SHADOW_MAPS_MAX) shadow maps of the same size and pitch in
 * one call: map k from occluder set occ[k] (a host array of n_maps
 * descriptors) into depth[k] (a host array of n_maps device pointers), each
 * exactly as rbsm_shadow_map writes it, one launch per map, in order on
 * `stream`.  When no map's memory meets another map's or any occluder
 * array, each map after the first is a programmatic dependent launch that
 * takes SMs as the previous map's kernel drains; work after the call on
 * `stream` still follows all of them.  The kernels (of both calls) signal
 * their dependents at their start, so a caller's own programmatic
 * dependent must wait for them (cudaGridDependencySynchronize) before
 * reading the maps.  Every argument is checked before the first launch.
 * Errors: RBSM_ERR_ARG as rbsm_shadow_map for any map, NULL arrays, or
 * n_maps outside 1..RBSM_SHADOW_MAPS_MAX; RBSM_ERR_CUDA when a launch fails.
 */
#define RBSM_SHADOW_MAPS_MAX 256
int rbsm_shadow_maps(const rbsm_occluders *occ, float *const *depth, int32_t n_maps, int32_t width,
                     int32_t height, int64_t pitch, void *stream);

/*
 * Host-resident batches: the stager (this library's addition; the paper
 * evaluates fragments where the renderer produced them, on the GPU, and has
 * no host-side interface).
 *
 * rbsm_stager_run takes an rbsm_batch whose maps, fragment planes and
 * answer planes live in page-locked host memory (cudaHostAlloc or
 * cudaHostRegister; pageable memory is rejected) and returns the answers
 * to those host planes.  Per map (in index order) it moves to the device
 * only what the path can read: the fragment planes of the map's jobs and
 * the window of the map within h = max_dist + 1 texels of some fragment's
 * texel.  The shadow test and discontinuity check (Eq. 1, Listing 2) read
 * one texel around the fragment's texel, each edge traversal (Listing 3) at
 * most max_dist texels along one row or column and one across it, and the
 * learned surrogate's 5x5 window two; no read leaves the window, so the
 * answers are those rbsm_batch_run gives on device copies of the whole
 * batch, bit for bit.  The window is the bounding box of the jobs' texels
 * (computed on the device from the staged fragments, with the texel
 * arithmetic of the kernels) grown by h, its columns widened to multiples
 * of 4 texels (16-byte row pieces) and clipped to the map; the texels
 * outside it are never copied.
 *
 * Work per map, with no host wait anywhere: copies of the fragment planes
 * in, the texel bounds, a kernel that copies the window rows in from the
 * host map, the batched kernel, copies of the answers out.  These run on
 * the stager's own streams through a ring of device slots, so the copies
 * in of one map, the window and kernel of the previous ones and the
 * copies out of the one before overlap.  The call is ordered after the work already enqueued
 * on `stream`, and `stream` is ordered after the call's last copy out.
 *
 * desc: max_fragments = the largest sum of n over the jobs of one map;
 * max_width / max_height bound every map; slots = device slots in the ring,
 * 2..4 (0 = 3: in, kernel and out of three maps at once); texture = 1 to
 * read the staged maps through texture gathers; flags reserved (0).  A slot
 * holds 22 bytes per fragment (x, y, z, both answers, codes) and one map.
 * Creation allocates the slots and streams (device memory, driver objects)
 * and may not run during a stream capture; the calls of one stager must
 * come from one thread at a time, and a stager is not graph-capturable.
 *
 * rbsm_stager_run errors: RBSM_ERR_ARG as for rbsm_batch_run, or a map
 * descriptor with a texture, a map larger than max_width x max_height, the
 * jobs of one map holding more than max_fragments fragments, or a plane
 * that is not page-locked host memory; RBSM_ERR_CUDA when a copy or launch
 * fails (work already enqueued for earlier maps stays enqueued).
 * rbsm_stager_stats waits for the stager's work and returns the bytes its
 * runs copied in (fragment planes and map windows) and out (answers),
 * summed over every run since creation.  rbsm_stager_status waits for the
 * stager's work and returns the first RBSM_ERR_* code a kernel recorded in
 * any slot, or RBSM_OK.
 */
typedef struct rbsm_stager_s *rbsm_stager;
typedef struct {
    int64_t max_fragments;
    int32_t max_width;
    int32_t max_height;
    int32_t slots;
    int32_t texture;
    int32_t flags;
} rbsm_stager_desc;
int rbsm_stager_create(const rbsm_stager_desc *desc, rbsm_stager *stager);
int rbsm_stager_run(rbsm_stager stager, const rbsm_batch *batch, void *stream);
int rbsm_stager_stats(rbsm_stager stager, int64_t *bytes_in, int64_t *bytes_out);
int rbsm_stager_status(rbsm_stager stager, int *status);
int rbsm_stager_destroy(rbsm_stager stager);

/*
 * Learned penumbra surrogate (not in the paper; this library's addition).
 * A 32-64-64-2 perceptron estimates the Listing 5 answer of an edge
 * fragment from its 5x5 shadow-test pattern (bit (dy+2)*5 + (dx+2) set when
 * texel (i+dx, j+dy) is lit), its in-texel offsets and the depth gap to the
 * nearest blocker of the window, plus an estimate of its own absolute
 * error.  BF16 weights and activations, FP32 accumulation on the tensor
 * cores: training and rbsm_mlp_forward on tcgen05 (tiles of 128 samples,
 * accumulators in tensor memory), the guarded inference inside
 * rbsm_batch_run on warp-level tiles of the edge fragments of one warp.
 *
 * The state block (device, caller-allocated, 256-byte aligned,
 * rbsm_mlp_state_bytes() bytes, about 11 MB) holds the FP32 master
 * parameters, their gradient, the Adam moments, BF16 weight copies, a loss
 * accumulator, a status word, the per-CTA partial sums of the gradient
 * kernel and the trusted-pattern bitmap.  The FP32 parameter vector has
 * RBSM_MLP_PARAMS floats in the order W1 (32 x 64, row-major (in, out)),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (64 x 2), b3 (2).  Calls on one state block must be ordered (one
 * stream, or events); the gradient calls use the partials as scratch.
 */
#define RBSM_MLP_PARAMS 6402

/* One training sample: features of an edge fragment and its exact RSMSS answer. */
typedef struct {
    uint32_t bits;                 /* 25-bit 5x5 shadow-test pattern */
    float fx, fy;                  /* in-texel offsets */
    float gap;                     /* fragment depth - nearest blocker depth in the window */
    float label;                   /* Listing 5 visibility */
} rbsm_sample;

size_t rbsm_mlp_state_bytes(void);

/* Copy n = RBSM_MLP_PARAMS host floats in (stream-ordered; the host array
 * must stay valid until the stream reaches the copy), zero the gradient,
 * the Adam moments, the loss and the status word, build the BF16 copies. */
int rbsm_mlp_load(void *state, const float *params_host, void *stream);

/* Trusted patterns: a bitmap of RBSM_MLP_TRUST_WORDS host words (bit p & 31
 * of word p >> 5 for the 25-bit 5x5 pattern p), copied in stream-ordered;
 * from then on rbsm_batch_run lets the surrogate answer only fragments whose
 * pattern is trusted.  NULL switches the bitmap off (every pattern trusted,
 * the state after rbsm_mlp_load).  The bitmap comes from calibration: the
 * patterns on which the trained network's answers stayed within a stated
 * error over held-out calibration scenes. */
#define RBSM_MLP_TRUST_WORDS (1 << 20)
int rbsm_mlp_set_trust(void *state, const uint32_t *bitmap_host, void *stream);

/* Copy the FP32 master parameters out to host memory (stream-ordered). */
int rbsm_mlp_store(const void *state, float *params_host, void *stream);

/* Append every edge fragment of a fragment set (filtering mode) as a
 * training sample at the device counter *counter (which the caller zeroes
 * once); samples past `capacity` are counted but not written.  With
 * params->flags = RBSM_DATASET_IN_WINDOW only the fragments whose walks stop
 * inside the 5x5 window are kept.  The order of the samples is not fixed
 * (warps append as they finish). */
int rbsm_mlp_dataset(const rbsm_map *map, const rbsm_frags *frags, const rbsm_params *params,
                     rbsm_sample *samples, int64_t capacity, unsigned long long *counter, void *stream);

/* Add the loss gradient of one minibatch (samples[order[0..batch)], every
 * order entry a valid sample index) to the state's gradient, and the loss
 * sum to its loss accumulator: loss = mean (y0 - t)^2 + mean
 * (y1 - |clamp(y0,0,1) - t|)^2, the second target held constant.  Two
 * kernels: per-CTA sums over 128-sample tiles, then their sum in CTA order;
 * the result is the same bits on every run. */
int rbsm_mlp_grad(void *state, const rbsm_sample *samples, const int32_t *order, int32_t batch, void *stream);

/* One training step: rbsm_mlp_grad of the minibatch followed by
 * rbsm_mlp_adam(step, lr), with the reduction and the Adam update in one
 * kernel (the same bits as the two calls). */
int rbsm_mlp_step(void *state, const rbsm_sample *samples, const int32_t *order, int32_t batch, int32_t step,
                  float lr, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr;
 * `step` counts from 1; clears the gradient. */
int rbsm_mlp_adam(void *state, int32_t step, float lr, void *stream);

/* Synchronously read the accumulated gradient (RBSM_MLP_PARAMS floats) and/or
 * the loss sum since the last reset (either pointer may be NULL).  Returns
 * the RBSM_ERR_* code a surrogate kernel recorded in the state (a tensor-core
 * wait that gave up: RBSM_ERR_TIMEOUT; the outputs are then not valid), else
 * RBSM_OK. */
int rbsm_mlp_read(const void *state, float *grad_host, float *loss_host, void *stream);
int rbsm_mlp_reset_loss(void *state, void *stream);

/* Network outputs (n x 2 floats: estimate, error estimate) of n samples. */
int rbsm_mlp_forward(const void *state, const rbsm_sample *samples, int64_t n, float *out, void *stream);

/*
 * Diagnostic of the bounded waits.  Every tensor-core kernel of the library
 * waits for its products on mbarriers through one routine that gives up
 * after a time limit of the device's global timer; the kernel then records
 * RBSM_ERR_TIMEOUT and returns instead of hanging.  This call runs that routine in one thread of one CTA
 * on a barrier that nothing arrives at, with limit_ns (1e3 ... 1e9
 * nanoseconds), and then on the same barrier after one arrival.
 *
 *   out: device pointer to 3 uint64_t (8-byte aligned), written
 *     out[0] = 1 when the first wait gave up (expected), else 0;
 *     out[1] = 1 when the second wait completed (expected), else 0;
 *     out[2] = nanoseconds the first wait took (the device's global timer).
 *
 * Asynchronous on `stream`.  Returns RBSM_ERR_ARG for a null or unaligned
 * `out` or a limit outside the range, RBSM_ERR_CUDA when the launch fails.
 * Not part of the method; it lets a caller check the timeout path on its
 * own hardware without faulting or hanging the GPU.
 */
int rbsm_selftest_bounded_wait(uint64_t limit_ns, uint64_t *out, void *stream);

/* Text for a return code. */
const char *rbsm_status_string(int code);

/* The cudaError_t number behind the last RBSM_ERR_CUDA of this thread. */
int rbsm_last_cuda_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int rbsm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RBSM_H */
