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
#define RBSM_ERR_TIMEOUT (-3)      /* a bounded device-side wait gave up */
#define RBSM_ERR_WORKSPACE (-4)    /* workspace missing, too small or misaligned */

#define RBSM_MODE_SILHOUETTE 1     /* Listing 4, §4.1: hard shadows, revectorised */
#define RBSM_MODE_FILTER 2         /* Listing 5, §4.2: fake penumbra (RSMSS) */
#define RBSM_MODE_BOTH 3           /* both answers from one pass over the fragments */

#define RBSM_MAXDIST_DEFAULT 16    /* §3.1.3: the value the paper used */
#define RBSM_MAXDIST_LIMIT 255
#define RBSM_MAX_EXTENT 65536      /* width and height limit of a shadow map */

/* A shadow map (device memory, owned by the caller). */
typedef struct {
    const float *depth;
    int32_t width;
    int32_t height;
    int64_t pitch;                 /* floats between rows, >= width */
} rbsm_map;

/* A set of light-space fragments (device memory, owned by the caller). */
typedef struct {
    const float *x;
    const float *y;
    const float *z;
    int64_t n;                     /* >= 0; n == 0 enqueues nothing */
} rbsm_frags;

typedef struct {
    int32_t max_dist;              /* MAXDIST of Listing 3, 1..RBSM_MAXDIST_LIMIT */
    int32_t flags;                 /* reserved, must be 0 */
} rbsm_params;

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
 * width or height outside 1..RBSM_MAX_EXTENT, pitch < width, n < 0,
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
    int32_t tile_threads;          /* CTA size: 128, 256 or 512; 0 = default 256 */
    int32_t ctas_per_sm;           /* persistent CTAs per SM, 1..8; 0 = occupancy limit */
} rbsm_batch;

/*
 * Device workspace a batch needs (a work counter and a status word), in
 * bytes; the caller allocates it (256-byte aligned) and may reuse it for any
 * later batch that is not in flight at the same time.
 */
int rbsm_batch_workspace_size(const rbsm_batch *batch, size_t *bytes);

/*
 * Enqueue one batched launch: a memset of the workspace followed by one
 * persistent kernel whose CTAs take (job, tile) items from an atomic counter.
 * The descriptors are copied into the launch parameters, so the host arrays
 * may be reused as soon as the call returns.  Errors: RBSM_ERR_ARG as for
 * rbsm_visibility applied to every map and job, or a map index out of range;
 * RBSM_ERR_WORKSPACE for a NULL, small or misaligned workspace;
 * RBSM_ERR_CUDA when a launch fails.
 */
int rbsm_batch_run(const rbsm_batch *batch, void *workspace, size_t workspace_bytes, void *stream);

/*
 * After the stream has completed a batch: read its device status word
 * (synchronously, with a device-to-host copy) and return RBSM_OK or the
 * RBSM_ERR_* code the kernel recorded.
 */
int rbsm_batch_status(const void *workspace, int *status);

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
