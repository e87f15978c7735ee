// Learned penumbra surrogate: training data, training step, Adam, forward.
//
// Not in the paper.  The surrogate estimates the Listing 5 (RSMSS) answer of
// an edge fragment from its 5x5 shadow-test pattern, in-texel offsets and
// blocker-receiver depth gap.  Training data come from the plain RSMSS
// (this library's exact walk), so the plain method is the surrogate's
// teacher, its fallback and the measure of its error.
//
// The network state lives in one caller-allocated device block
// (rbsm_mlp_state_bytes): FP32 master parameters, their gradient, the two
// Adam moments, BF16 copies of the weights in the layouts the tensor-core
// tiles read, and a loss accumulator.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rbsm.h"
#include "rbsm_device.cuh"
#include "rbsm_host.h"
#include "rbsm_mlp.cuh"
#include "rbsm_tc.cuh"

namespace rbsm {
namespace mlp {

// Write parameter p's BF16 copy from its FP32 value (weights only; the
// copies are the forward layout [out][in], read by every kernel).
__device__ __forceinline__ void write_copies(const State &s, int p, float val)
{
    const uint16_t h = float_to_bf16(val);
    if (p < kOffB1) {
        const int i = (p - kOffW1) / kHid, o = (p - kOffW1) % kHid;
        s.w1t[o * kIn + i] = h;
    } else if (p >= kOffW2 && p < kOffB2) {
        const int i = (p - kOffW2) / kHid, o = (p - kOffW2) % kHid;
        s.w2t[o * kHid + i] = h;
    } else if (p >= kOffW3 && p < kOffB3) {
        const int i = (p - kOffW3) / kOut, o = (p - kOffW3) % kOut;
        s.w3t[o * kHid + i] = h;
    }
}

__global__ void refresh_kernel(void *base)
{
    const State s = state_of(base);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams; p += gridDim.x * blockDim.x) {
        write_copies(s, p, s.master[p]);
        s.grad[p] = 0.0f;
        s.m[p] = 0.0f;
        s.v[p] = 0.0f;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2)
        s.loss[threadIdx.x] = 0.0f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *s.status = 0u;
        *s.trust_on = 0u;
    }
}

// One Adam update (Kingma and Ba, Algorithm 1) of parameter p with gradient
// g; refreshes the BF16 copy.
__device__ __forceinline__ void adam_update(const State &s, int p, float g, float lr, float bc1, float bc2)
{
    constexpr float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m = b1 * s.m[p] + (1.0f - b1) * g;
    const float v = b2 * s.v[p] + (1.0f - b2) * g * g;
    s.m[p] = m;
    s.v[p] = v;
    const float val = s.master[p] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    s.master[p] = val;
    write_copies(s, p, val);
}

// One Adam step of every parameter from the accumulated gradient, which it
// clears.
__global__ void adam_kernel(void *base, float lr, float bc1, float bc2)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const State s = state_of(base);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams; p += gridDim.x * blockDim.x) {
        adam_update(s, p, s.grad[p], lr, bc1, bc2);
        s.grad[p] = 0.0f;
    }
}

// ------------------------------------------------------------- features --

// Training samples: every edge fragment (filtering mode) of a fragment set
// with its features and its exact RSMSS answer, appended at an atomic
// counter (warp-aggregated).  Samples past `capacity` are counted, not kept.
__global__ void dataset_kernel(const MapDev m, const float *__restrict__ x, const float *__restrict__ y,
                               const float *__restrict__ z, long long n, int max_dist, bool in_window_only,
                               rbsm_sample *out, long long capacity, unsigned long long *counter)
{
    const unsigned lane = lane_id();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
        const long long k = base + threadIdx.x;
        bool edge = false;
        FragResult r{0.0f, 0.0f, 0};
        uint32_t bits = 0;
        float xv = 0.0f, yv = 0.0f, zv = 0.0f;
        rbsm_sample smp;
        if (k < n) {
            xv = x[k];
            yv = y[k];
            zv = z[k];
            edge = classify<2, false>(m, xv, yv, zv, r, bits);
            if (edge) {
                fragment_features(m, xv, yv, zv, smp.bits, smp.fx, smp.fy, smp.gap);
                if (in_window_only && !walks_inside_window(smp.bits, max_dist))
                    edge = false;
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, edge);
        if (mask == 0)
            continue;
        unsigned long long slot0 = 0;
        const int leader = __ffs(mask) - 1;
        if ((int)lane == leader)
            slot0 = atomicAdd(counter, (unsigned long long)__popc(mask));
        slot0 = __shfl_sync(0xffffffffu, slot0, leader);
        if (!edge)
            continue;
        const unsigned long long slot = slot0 + __popc(mask & ((1u << lane) - 1u));
        if ((long long)slot >= capacity)
            continue;
        resolve_edge<2>(m, xv, yv, zv, bits, max_dist, r);
        smp.label = r.fil;
        out[slot] = smp;
    }
}

// ----------------------------------------------------------- training --
//
// Gradient and forward pass on the fifth-generation tensor cores.  A CTA of
// 128 threads takes tiles of 128 samples (M = 128, one TMEM lane and one
// thread per sample).  Per tile, with one thread issuing every product:
//
//   forward        a1 = X W1,  a2 = h1 W2,  y = h2 W3             (K-major A and B)
//   backward-data  dh2 = dY W3^T,  dh1 = dA2 W2^T                  (B: the forward
//                  weight copies read as MN-major operands)
//   weight grads   [dA1 | dA2]^T [X | H1]  -> dW1^T, dW2^T          (M = 128 units,
//                  [H1 | H2]^T dY          -> dW3                  K = samples; both
//                                                                  operands MN-major)
//
// Activations are written once per tile, in 8 x 8 core matrices, into two
// shared-memory buffers: act (X | H1 | H2, 160 units per sample) and grd
// (dA1 | dA2 | dY, 144 units per sample).  A K-major descriptor over a
// column range of a buffer is the next layer's A operand; an MN-major
// descriptor over the same bytes is that activation transposed (units
// along M or N, samples along K) for the weight-gradient products, which
// accumulate in TMEM across the CTA's tiles.  The epilogues (bias, ReLU
// and its mask, loss, BF16 rounding) are per thread on its own row.
//
// Bias gradients and the loss are FP32 column sums of unrounded values in a
// fixed order (a butterfly over the warp, then the four warps in order).
// Each CTA writes its sums to its row of the partials; the reduction kernel
// adds the rows in CTA order, so a gradient is bit-reproducible.

constexpr int kTcRows = 128;                       // samples per tile (M)
constexpr int kTcThreads = 128;
constexpr int kActCols = kIn + 2 * kHid;           // X | H1 | H2
constexpr int kGrdCols = 2 * kHid + 16;            // dA1 | dA2 | dY (padded to 16)
constexpr uint32_t kCore = 128;                    // bytes per core matrix = LBO of a K-major buffer
constexpr uint32_t kActSbo = kActCols * 16;        // bytes between 8-row groups of act
constexpr uint32_t kGrdSbo = kGrdCols * 16;
constexpr uint32_t kW1tSbo = kIn * 16;             // weights: rows = output unit, K = input unit
constexpr uint32_t kW2tSbo = kHid * 16;
constexpr uint32_t kW3tSbo = kHid * 16;
constexpr int kW3Rows = 16;                        // N of the output layer (2 used)
// column groups (8 units each) of the buffers
constexpr int kGX = 0, kGH1 = kIn / 8, kGH2 = kGH1 + kHid / 8;
constexpr int kGdA1 = 0, kGdA2 = kHid / 8, kGdY = 2 * kHid / 8;
// TMEM columns: weight-gradient accumulators, then two transient tiles
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColP1 = 0, kColP2 = 96, kColA = 128, kColB = 192;
constexpr uint64_t kWaitNs = 1000000000ull;       // a tensor-core wait gives up after 1 s

struct TcSmem {
    alignas(128) unsigned char act[kTcRows * kActCols * 2];
    alignas(128) unsigned char grd[kTcRows * kGrdCols * 2];
    alignas(128) unsigned char w1t[kHid * kIn * 2];
    alignas(128) unsigned char w2t[kHid * kHid * 2];
    alignas(128) unsigned char w3t[kW3Rows * kHid * 2];
    float b1[kHid], b2[kHid], b3[kOut];
    float red1[4][kHid], red2[4][kHid], red3[4][4];
    uint64_t bar;
    uint32_t tmem_base;
};

__device__ __forceinline__ unsigned char *group_ptr(unsigned char *buf, uint32_t sbo, int row, int group)
{
    return buf + (row >> 3) * sbo + group * kCore + (row & 7) * 16;
}

// Copy a row-major BF16 matrix (rows x cols, the first src_rows rows from
// global memory, the rest zero) into core matrices (rows along M/N).
__device__ __forceinline__ void stage_weights(unsigned char *dst, const uint16_t *src, int rows, int src_rows,
                                              int cols)
{
    const int groups = cols / 8;
    for (int c = threadIdx.x; c < rows * groups; c += blockDim.x) {
        const int r = c / groups, g = c % groups;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < src_rows)
            v = *reinterpret_cast<const uint4 *>(src + r * cols + g * 8);
        *reinterpret_cast<uint4 *>(dst + (r >> 3) * (cols * 16) + g * kCore + (r & 7) * 16) = v;
    }
}

// Column sums of v[0..64) over the warp's 32 lanes by halving exchanges:
// lane L returns the sums of columns 2L and 2L + 1.  v is consumed.
__device__ __forceinline__ float2 warp_column_sums(float (&v)[kHid], unsigned lane)
{
#pragma unroll
    for (int width = 32, bit = 16; bit >= 1; width >>= 1, bit >>= 1) {
        const bool upper = (lane & bit) != 0;
#pragma unroll
        for (int i = 0; i < width; ++i) {
            const float send = upper ? v[i] : v[i + width];
            const float keep = upper ? v[i + width] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    return make_float2(v[0], v[1]);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int bit = 16; bit >= 1; bit >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, bit);
    return v;
}

// Hand this thread's shared-memory writes to the tensor core and meet at a
// CTA barrier; returns whether any thread raised `flag`.
__device__ __forceinline__ bool sync_for_mma(bool flag)
{
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    const int any = __syncthreads_or(flag ? 1 : 0);
    tc::fence_after_sync();
    return any != 0;
}

// Wait for the products committed last; the outcome is uniform over the warp
// (the TMEM loads that follow are warp-collective).
__device__ __forceinline__ bool wait_products(uint64_t *bar, uint32_t &parity)
{
    const bool ok = tc::mbar_wait(bar, parity, kWaitNs);
    parity ^= 1u;
    const bool all = __all_sync(0xffffffffu, ok) != 0;
    if (all)
        tc::fence_after_sync();
    return all;
}

// Bias, ReLU and BF16 rounding of one hidden layer's row (FP32 accumulators
// a[64]); writes h into eight column groups of act and returns the ReLU mask
// (bit j: unit j positive).
__device__ __forceinline__ uint64_t hidden_epilogue(const float (&a)[kHid], const float *bias, unsigned char *act,
                                                    int row, int group0)
{
    uint64_t mask = 0;
#pragma unroll
    for (int g = 0; g < kHid / 8; ++g) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = g * 8 + 2 * q;
            const float v0 = a[j] + bias[j], v1 = a[j + 1] + bias[j + 1];
            mask |= (uint64_t)(v0 > 0.0f) << j;
            mask |= (uint64_t)(v1 > 0.0f) << (j + 1);
            w[q] = pack_bf16(fmaxf(v0, 0.0f), fmaxf(v1, 0.0f));
        }
        *reinterpret_cast<uint4 *>(group_ptr(act, kActSbo, row, group0 + g)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    return mask;
}

// Mask a backward row by the ReLU mask, write it (BF16) into eight column
// groups of grd, and leave this warp's FP32 column sums in red[warp].
__device__ __forceinline__ void backward_epilogue(float (&d)[kHid], uint64_t mask, unsigned char *grd, int row,
                                                  int group0, float (*red)[kHid], int warp, unsigned lane)
{
#pragma unroll
    for (int j = 0; j < kHid; ++j)
        d[j] = ((mask >> j) & 1u) ? d[j] : 0.0f;
#pragma unroll
    for (int g = 0; g < kHid / 8; ++g) {
        const int j = g * 8;
        *reinterpret_cast<uint4 *>(group_ptr(grd, kGrdSbo, row, group0 + g)) =
            make_uint4(pack_bf16(d[j], d[j + 1]), pack_bf16(d[j + 2], d[j + 3]), pack_bf16(d[j + 4], d[j + 5]),
                       pack_bf16(d[j + 6], d[j + 7]));
    }
    const float2 s = warp_column_sums(d, lane);
    red[warp][2 * lane] = s.x;
    red[warp][2 * lane + 1] = s.y;
}

// kTrain: gradient of the mean loss over samples[order[0..n)] into the
// partials row of this CTA (n = batch).  Otherwise: outputs out[2b], out[2b+1]
// of samples[0..n).  Launched as a programmatic dependent (it waits for the
// previous kernel before reading global memory).
template <bool kTrain>
__global__ void __launch_bounds__(kTcThreads)
surrogate_tc_kernel(void *base, const rbsm_sample *__restrict__ data, const int *__restrict__ order, long long n,
                    float inv_batch, float *__restrict__ out)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const unsigned lane = lane_id();

    if (tid == 0)
        tc::mbar_init(&sm.bar, 1);
    if (warp == 0)
        tc::tmem_alloc(&sm.tmem_base, kTmemCols);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const State st = state_of(base);
    const long long tiles = (n + kTcRows - 1) / kTcRows;
    // a tile's samples are gathered one tile ahead (the first before the
    // weights are staged), so the gather overlaps the previous tile's products
    auto gather = [&](long long tile) {
        rbsm_sample v{0u, 0.0f, 0.0f, 0.0f, 0.0f};
        const long long b = tile * kTcRows + tid;
        if (tile < tiles && b < n)
            v = data[kTrain ? (long long)order[b] : b];
        return v;
    };
    rbsm_sample smp = gather(blockIdx.x);
    stage_weights(sm.w1t, st.w1t, kHid, kHid, kIn);
    stage_weights(sm.w2t, st.w2t, kHid, kHid, kHid);
    stage_weights(sm.w3t, st.w3t, kW3Rows, kOutPad, kHid);
    for (int k = tid; k < kHid; k += kTcThreads) {
        sm.b1[k] = st.master[kOffB1 + k];
        sm.b2[k] = st.master[kOffB2 + k];
    }
    if (tid < kOut)
        sm.b3[tid] = st.master[kOffB3 + tid];
    if (kTrain)   // dY columns 8..15 stay zero
        *reinterpret_cast<uint4 *>(group_ptr(sm.grd, kGrdSbo, tid, kGdY + 1)) = make_uint4(0u, 0u, 0u, 0u);
    bool fail = sync_for_mma(false);

    const uint32_t tmem = sm.tmem_base;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const uint32_t tA = tmem + kColA, tB = tmem + kColB, tP1 = tmem + kColP1, tP2 = tmem + kColP2;
    const uint32_t act = tc::smem_addr(sm.act), grd = tc::smem_addr(sm.grd);
    const uint32_t w1t = tc::smem_addr(sm.w1t), w2t = tc::smem_addr(sm.w2t), w3t = tc::smem_addr(sm.w3t);
    constexpr uint32_t id64 = tc::idesc_bf16(kTcRows, kHid, false, false);
    constexpr uint32_t id16 = tc::idesc_bf16(kTcRows, kW3Rows, false, false);
    constexpr uint32_t id64_bmn = tc::idesc_bf16(kTcRows, kHid, false, true);
    constexpr uint32_t idP1 = tc::idesc_bf16(kTcRows, kIn + kHid, true, true);
    constexpr uint32_t idP2 = tc::idesc_bf16(kTcRows, kW3Rows, true, true);

    uint32_t parity = 0;
    bool first = true, p1_pending = false;
    float db1 = 0.0f, db2 = 0.0f, db3 = 0.0f, loss = 0.0f;    // thread t: column t of b1 / b2 (t < 64), b3 (t < 2)
    for (long long tile = blockIdx.x; tile < tiles && !fail; tile += gridDim.x) {
        const long long b = tile * kTcRows + tid;
        const bool valid = b < n;
        if (p1_pending) {       // the previous tile's weight-gradient products still read act and grd
            const bool ok = wait_products(&sm.bar, parity);
            p1_pending = false;
            tc::fence_smem_to_async();
            if ((fail = sync_for_mma(!ok)))
                break;
        }
        {   // input row: 25 pattern bits, fx, fy, gap, zeros (BF16)
            uint32_t w[16];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const uint32_t lo = (smp.bits >> (2 * k)) & 1u, hi = (smp.bits >> (2 * k + 1)) & 1u;
                w[k] = (lo ? 0x3F80u : 0u) | ((hi ? 0x3F80u : 0u) << 16);      // 1.0 in BF16 is 0x3F80
            }
            w[12] = (((smp.bits >> 24) & 1u) ? 0x3F80u : 0u) | ((uint32_t)float_to_bf16(smp.fx) << 16);
            w[13] = (uint32_t)float_to_bf16(smp.fy) | ((uint32_t)float_to_bf16(smp.gap) << 16);
            w[14] = 0u;
            w[15] = 0u;
#pragma unroll
            for (int g = 0; g < 4; ++g)
                *reinterpret_cast<uint4 *>(group_ptr(sm.act, kActSbo, tid, kGX + g)) =
                    make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
        }
        const float label = smp.label;
        smp = gather(tile + gridDim.x);
        if ((fail = sync_for_mma(false)))
            break;
        // ---- layer 1: a1 = X W1 (K = 32)
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < kIn / 16; ++k)
                tc::mma_bf16(tA, tc::smem_desc(act + kGX * kCore + k * 2 * kCore, kCore, kActSbo),
                             tc::smem_desc(w1t + k * 2 * kCore, kCore, kW1tSbo), id64, k > 0);
            tc::commit(&sm.bar);
        }
        bool ok = wait_products(&sm.bar, parity);
        uint64_t mask1 = 0, mask2 = 0;
        if (ok) {
            float a[kHid];
            tc::tmem_load_row<kHid>(tA + lane_off, a);
            mask1 = hidden_epilogue(a, sm.b1, sm.act, tid, kGH1);
        }
        if ((fail = sync_for_mma(!ok)))
            break;
        // ---- layer 2: a2 = h1 W2 (K = 64)
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < kHid / 16; ++k)
                tc::mma_bf16(tB, tc::smem_desc(act + kGH1 * kCore + k * 2 * kCore, kCore, kActSbo),
                             tc::smem_desc(w2t + k * 2 * kCore, kCore, kW2tSbo), id64, k > 0);
            tc::commit(&sm.bar);
        }
        ok = wait_products(&sm.bar, parity);
        if (ok) {
            float a[kHid];
            tc::tmem_load_row<kHid>(tB + lane_off, a);
            mask2 = hidden_epilogue(a, sm.b2, sm.act, tid, kGH2);
        }
        if ((fail = sync_for_mma(!ok)))
            break;
        // ---- layer 3: y = h2 W3 (N = 16, two columns used)
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < kHid / 16; ++k)
                tc::mma_bf16(tA, tc::smem_desc(act + kGH2 * kCore + k * 2 * kCore, kCore, kActSbo),
                             tc::smem_desc(w3t + k * 2 * kCore, kCore, kW3tSbo), id16, k > 0);
            tc::commit(&sm.bar);
        }
        ok = wait_products(&sm.bar, parity);
        if (ok) {
            uint32_t r[2];
            tc::tmem_ld2(tA + lane_off, r);
            const float y0 = __uint_as_float(r[0]) + sm.b3[0], y1 = __uint_as_float(r[1]) + sm.b3[1];
            if (!kTrain) {
                if (valid) {
                    out[2 * b] = y0;
                    out[2 * b + 1] = y1;
                }
            } else {
                // loss and output gradient: (y0 - t)^2 + (y1 - |clamp(y0) - t|)^2, the second target constant
                float dy0 = 0.0f, dy1 = 0.0f, l = 0.0f;
                if (valid) {
                    const float tl = label;
                    const float vc = fminf(fmaxf(y0, 0.0f), 1.0f);
                    const float et = fabsf(vc - tl);
                    const float rv = y0 - tl, re = y1 - et;
                    dy0 = 2.0f * rv * inv_batch;
                    dy1 = 2.0f * re * inv_batch;
                    l = __fadd_rn(__fmul_rn(rv, rv), __fmul_rn(re, re));
                }
                *reinterpret_cast<uint4 *>(group_ptr(sm.grd, kGrdSbo, tid, kGdY)) =
                    make_uint4(pack_bf16(dy0, dy1), 0u, 0u, 0u);
                const float s0 = warp_sum(dy0), s1 = warp_sum(dy1), sl = warp_sum(l);
                if (lane == 0) {
                    sm.red3[warp][0] = s0;
                    sm.red3[warp][1] = s1;
                    sm.red3[warp][2] = sl;
                }
            }
        }
        if (!kTrain) {
            if ((fail = sync_for_mma(!ok)))
                break;
            continue;
        }
        if ((fail = sync_for_mma(!ok)))
            break;
        if (tid < kOut)
            db3 += ((sm.red3[0][tid] + sm.red3[1][tid]) + sm.red3[2][tid]) + sm.red3[3][tid];
        if (tid == 0)
            loss += ((sm.red3[0][2] + sm.red3[1][2]) + sm.red3[2][2]) + sm.red3[3][2];
        // ---- dh2 = dY W3^T (K = 16) and dW3 += [H1 | H2]^T dY (K = the tile's 128 samples)
        if (tid == 0) {
            tc::mma_bf16(tB, tc::smem_desc(grd + kGdY * kCore, kCore, kGrdSbo),
                         tc::smem_desc(w3t, kW3tSbo, kCore), id64_bmn, false);
#pragma unroll
            for (int k = 0; k < kTcRows / 16; ++k)
                tc::mma_bf16(tP2, tc::smem_desc(act + kGH1 * kCore + k * 2 * kActSbo, kActSbo, kCore),
                             tc::smem_desc(grd + kGdY * kCore + k * 2 * kGrdSbo, kGrdSbo, kCore), idP2,
                             !(first && k == 0));
            tc::commit(&sm.bar);
        }
        ok = wait_products(&sm.bar, parity);
        if (ok) {
            float d[kHid];
            tc::tmem_load_row<kHid>(tB + lane_off, d);
            backward_epilogue(d, mask2, sm.grd, tid, kGdA2, sm.red2, warp, lane);
        }
        if ((fail = sync_for_mma(!ok)))
            break;
        // ---- dh1 = dA2 W2^T (K = 64)
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < kHid / 16; ++k)
                tc::mma_bf16(tA, tc::smem_desc(grd + kGdA2 * kCore + k * 2 * kCore, kCore, kGrdSbo),
                             tc::smem_desc(w2t + k * 2 * kW2tSbo, kW2tSbo, kCore), id64_bmn, k > 0);
            tc::commit(&sm.bar);
        }
        if (tid < kHid)
            db2 += ((sm.red2[0][tid] + sm.red2[1][tid]) + sm.red2[2][tid]) + sm.red2[3][tid];
        ok = wait_products(&sm.bar, parity);
        if (ok) {
            float d[kHid];
            tc::tmem_load_row<kHid>(tA + lane_off, d);
            backward_epilogue(d, mask1, sm.grd, tid, kGdA1, sm.red1, warp, lane);
        }
        if ((fail = sync_for_mma(!ok)))
            break;
        // ---- dW1^T, dW2^T += [dA1 | dA2]^T [X | H1] (M = 128 units, N = 96 units, K = 128 samples)
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < kTcRows / 16; ++k)
                tc::mma_bf16(tP1, tc::smem_desc(grd + kGdA1 * kCore + k * 2 * kGrdSbo, kGrdSbo, kCore),
                             tc::smem_desc(act + kGX * kCore + k * 2 * kActSbo, kActSbo, kCore), idP1,
                             !(first && k == 0));
            tc::commit(&sm.bar);
        }
        if (tid < kHid)
            db1 += ((sm.red1[0][tid] + sm.red1[1][tid]) + sm.red1[2][tid]) + sm.red1[3][tid];
        p1_pending = true;
        first = false;
    }

    if (kTrain && !fail && p1_pending) {
        const bool ok = wait_products(&sm.bar, parity);
        fail = !ok;
        if (ok) {
            // row r of the weight-gradient accumulators: r < 64 is unit r of dA1
            // (columns 0..31: dW1[i][r]); r >= 64 is unit r - 64 of dA2 (columns
            // 32..95: dW2[i][r - 64]) and of H2 in the dW3 product
            float *part = st.part + (size_t)blockIdx.x * kPartStride;
            float d[kIn + kHid];
            tc::tmem_load_row<kIn + kHid>(tP1 + lane_off, d);
            uint32_t r3[2];
            tc::tmem_ld2(tP2 + lane_off, r3);
            if (tid < kHid) {
#pragma unroll
                for (int i = 0; i < kIn; ++i)
                    part[kOffW1 + i * kHid + tid] = d[i];
                part[kOffB1 + tid] = db1;
                part[kOffB2 + tid] = db2;
            } else {
                const int o = tid - kHid;
#pragma unroll
                for (int i = 0; i < kHid; ++i)
                    part[kOffW2 + i * kHid + o] = d[kIn + i];
                part[kOffW3 + o * kOut] = __uint_as_float(r3[0]);
                part[kOffW3 + o * kOut + 1] = __uint_as_float(r3[1]);
            }
            if (tid < kOut)
                part[kOffB3 + tid] = db3;
            if (tid == 0)
                part[kParams] = loss;
        }
    }
    if (fail && lane == 0)
        atomicOr(st.status, (unsigned)(-RBSM_ERR_TIMEOUT));
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_free(tmem, kTmemCols);
    }
}

// Sum of the `parts` partial rows of every parameter (and the loss), in CTA
// order within each of 8 strided subsets, the 8 subset sums then combined
// by a fixed butterfly.  step = 0: added to the gradient.  step > 0: one Adam
// step with (gradient + sum), and the gradient cleared.
constexpr int kReduceLanes = 8;
__global__ void __launch_bounds__(256) reduce_kernel(void *base, int parts, int step, float lr, float bc1, float bc2)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const State s = state_of(base);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = gtid / kReduceLanes, q = gtid % kReduceLanes;
    float sum = 0.0f;
    if (p <= kParams)
        for (int c = q; c < parts; c += kReduceLanes)
            sum += s.part[(size_t)c * kPartStride + p];
#pragma unroll
    for (int bit = kReduceLanes / 2; bit >= 1; bit >>= 1)
        sum += __shfl_xor_sync(0xffffffffu, sum, bit);
    if (q != 0 || p > kParams)
        return;
    if (p == kParams) {
        s.loss[0] += sum;
        return;
    }
    const float g = s.grad[p] + sum;
    if (step > 0) {
        adam_update(s, p, g, lr, bc1, bc2);
        s.grad[p] = 0.0f;
    } else {
        s.grad[p] = g;
    }
}

// Launch of the tensor-core kernel (gradient or forward) as a programmatic
// dependent of the previous kernel in the stream; *ctas gets the grid size.
template <bool kTrain>
int launch_tc(void *state, const rbsm_sample *samples, const int32_t *order, long long n, float inv_batch,
              float *out, cudaStream_t stream, int *ctas)
{
    static KernelSetup setup;
    const size_t smem = sizeof(TcSmem) + 1024;      // + alignment slack of the dynamic block
    int occ = 0;
    int rc = setup.get(surrogate_tc_kernel<kTrain>, kTcThreads, smem, &occ);
    if (rc != RBSM_OK)
        return rc;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    const long long tiles = (n + kTcRows - 1) / kTcRows;
    long long grid = (long long)sms * occ;
    if (kTrain && grid > kMaxGradCtas)
        grid = kMaxGradCtas;
    if (grid > tiles)
        grid = tiles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, surrogate_tc_kernel<kTrain>, state, samples,
                                       reinterpret_cast<const int *>(order), n, inv_batch, out);
    if (e != cudaSuccess)
        return cuda_fail(e);
    *ctas = (int)grid;
    return RBSM_OK;
}

// The reduction of `parts` partial rows (step 0: into the gradient; step > 0:
// fused with that Adam step), a programmatic dependent of the gradient kernel.
int launch_reduce(void *state, int parts, int step, float lr, cudaStream_t stream)
{
    double bc1 = 1.0, bc2 = 1.0;
    if (step > 0) {
        bc1 = 1.0 - pow(0.9, (double)step);
        bc2 = 1.0 - pow(0.999, (double)step);
    }
    const int threads = 256;
    const int blocks = ((kParams + 1) * kReduceLanes + threads - 1) / threads;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, reduce_kernel, state, parts, step, lr, (float)bc1, (float)bc2);
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

}  // namespace mlp
}  // namespace rbsm

using namespace rbsm;

extern "C" {

size_t rbsm_mlp_state_bytes(void) { return mlp::kStateBytes; }

int rbsm_mlp_load(void *state, const float *params, void *stream)
{
    if (!state || !params || (reinterpret_cast<uintptr_t>(state) & 255u))
        return RBSM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const mlp::State st = mlp::state_of(state);
    cudaError_t e = cudaMemcpyAsync(st.master, params, mlp::kParams * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    e = cudaMemsetAsync(reinterpret_cast<char *>(state) + mlp::kByteBf16, 0, mlp::kBf16Bytes, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    mlp::refresh_kernel<<<26, 256, 0, s>>>(state);
    e = cudaGetLastError();
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

int rbsm_mlp_set_trust(void *state, const uint32_t *bitmap, void *stream)
{
    if (!state || (reinterpret_cast<uintptr_t>(state) & 255u))
        return RBSM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const mlp::State st = mlp::state_of(state);
    cudaError_t e = cudaSuccess;
    if (bitmap)
        e = cudaMemcpyAsync(st.trust, bitmap, (size_t)mlp::kTrustWords * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(st.trust_on, bitmap ? 1 : 0, sizeof(unsigned), s);
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

int rbsm_mlp_store(const void *state, float *params, void *stream)
{
    if (!state || !params)
        return RBSM_ERR_ARG;
    const mlp::State st = mlp::state_of(const_cast<void *>(state));
    cudaError_t e = cudaMemcpyAsync(params, st.master, mlp::kParams * sizeof(float), cudaMemcpyDeviceToHost,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

int rbsm_mlp_dataset(const rbsm_map *map, const rbsm_frags *frags, const rbsm_params *params,
                     rbsm_sample *samples, int64_t capacity, unsigned long long *counter, void *stream)
{
    int rc, max_dist;
    if ((rc = check_map(map)) != RBSM_OK) return rc;
    if ((rc = check_frags(frags)) != RBSM_OK) return rc;
    if (!params || (params->flags & ~RBSM_DATASET_IN_WINDOW))
        return RBSM_ERR_ARG;
    const rbsm_params plain{params->max_dist, 0};
    if ((rc = check_params(&plain, &max_dist)) != RBSM_OK) return rc;
    if (!counter || capacity < 0 || (capacity > 0 && !samples))
        return RBSM_ERR_ARG;
    const bool in_window_only = (params->flags & RBSM_DATASET_IN_WINDOW) != 0;
    if (frags->n == 0)
        return RBSM_OK;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    long long blocks = (frags->n + 255) / 256;
    if (blocks > (long long)sms * 8)
        blocks = (long long)sms * 8;
    mlp::dataset_kernel<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        to_dev(*map), frags->x, frags->y, frags->z, frags->n, max_dist, in_window_only, samples, capacity, counter);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

int rbsm_mlp_grad(void *state, const rbsm_sample *samples, const int32_t *order, int32_t batch, void *stream)
{
    if (!state || !samples || !order || batch < 1 || (reinterpret_cast<uintptr_t>(state) & 255u))
        return RBSM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int parts = 0;
    int rc = mlp::launch_tc<true>(state, samples, order, batch, 1.0f / (float)batch, nullptr, s, &parts);
    if (rc != RBSM_OK)
        return rc;
    return mlp::launch_reduce(state, parts, 0, 0.0f, s);
}

int rbsm_mlp_step(void *state, const rbsm_sample *samples, const int32_t *order, int32_t batch, int32_t step,
                  float lr, void *stream)
{
    if (!state || !samples || !order || batch < 1 || step < 1 || !(lr > 0.0f) ||
        (reinterpret_cast<uintptr_t>(state) & 255u))
        return RBSM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int parts = 0;
    int rc = mlp::launch_tc<true>(state, samples, order, batch, 1.0f / (float)batch, nullptr, s, &parts);
    if (rc != RBSM_OK)
        return rc;
    return mlp::launch_reduce(state, parts, step, lr, s);
}

int rbsm_mlp_adam(void *state, int32_t step, float lr, void *stream)
{
    if (!state || step < 1 || !(lr > 0.0f))
        return RBSM_ERR_ARG;
    const double bc1 = 1.0 - pow(0.9, (double)step), bc2 = 1.0 - pow(0.999, (double)step);
    mlp::adam_kernel<<<26, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(state, lr, (float)bc1, (float)bc2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

int rbsm_mlp_read(const void *state, float *grad, float *loss, void *stream)
{
    if (!state || (!grad && !loss))
        return RBSM_ERR_ARG;
    const mlp::State st = mlp::state_of(const_cast<void *>(state));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned status = 0;
    cudaError_t e = cudaSuccess;
    if (grad)
        e = cudaMemcpyAsync(grad, st.grad, mlp::kParams * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && loss)
        e = cudaMemcpyAsync(loss, st.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, st.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    return status ? -(int)status : RBSM_OK;
}

int rbsm_mlp_reset_loss(void *state, void *stream)
{
    if (!state)
        return RBSM_ERR_ARG;
    const mlp::State st = mlp::state_of(state);
    cudaError_t e = cudaMemsetAsync(st.loss, 0, 2 * sizeof(float), reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

int rbsm_mlp_forward(const void *state, const rbsm_sample *samples, int64_t n, float *out, void *stream)
{
    if (!state || n < 0 || (n > 0 && (!samples || !out)) || (reinterpret_cast<uintptr_t>(state) & 255u))
        return RBSM_ERR_ARG;
    if (n == 0)
        return RBSM_OK;
    int ctas = 0;
    return mlp::launch_tc<false>(const_cast<void *>(state), samples, nullptr, n, 0.0f, out,
                                 reinterpret_cast<cudaStream_t>(stream), &ctas);
}

}  // extern "C"
