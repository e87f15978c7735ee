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

namespace rbsm {
namespace mlp {

// Write parameter p's BF16 copies from its FP32 value.
__device__ __forceinline__ void write_copies(const State &s, int p, float val)
{
    const uint16_t h = float_to_bf16(val);
    if (p < kOffB1) {
        const int i = (p - kOffW1) / kHid, o = (p - kOffW1) % kHid;
        s.w1t[o * kIn + i] = h;
    } else if (p >= kOffW2 && p < kOffB2) {
        const int i = (p - kOffW2) / kHid, o = (p - kOffW2) % kHid;
        s.w2t[o * kHid + i] = h;
        s.w2[i * kHid + o] = h;
    } else if (p >= kOffW3 && p < kOffB3) {
        const int i = (p - kOffW3) / kOut, o = (p - kOffW3) % kOut;
        s.w3t[o * kHid + i] = h;
        s.w3[i * 16 + o] = h;
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
}

// One Adam step (Kingma and Ba, Algorithm 1) per parameter; clears the
// gradient for the next step and refreshes the BF16 copies.
__global__ void adam_kernel(void *base, float lr, float bc1, float bc2)
{
    const State s = state_of(base);
    constexpr float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams; p += gridDim.x * blockDim.x) {
        const float g = s.grad[p];
        const float m = b1 * s.m[p] + (1.0f - b1) * g;
        const float v = b2 * s.v[p] + (1.0f - b2) * g * g;
        s.m[p] = m;
        s.v[p] = v;
        const float val = s.master[p] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        s.master[p] = val;
        s.grad[p] = 0.0f;
        write_copies(s, p, val);
    }
}

// ------------------------------------------------------------- features --

// Training samples: every edge fragment (filtering mode) of a fragment set
// with its features and its exact RSMSS answer, appended at an atomic
// counter (warp-aggregated).  Samples past `capacity` are counted, not kept.
__global__ void dataset_kernel(const MapDev m, const float *__restrict__ x, const float *__restrict__ y,
                               const float *__restrict__ z, long long n, int max_dist, rbsm_sample *out,
                               long long capacity, unsigned long long *counter)
{
    const unsigned lane = lane_id();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
        const long long k = base + threadIdx.x;
        bool edge = false;
        FragResult r{0.0f, 0.0f, 0};
        uint32_t bits = 0;
        float xv = 0.0f, yv = 0.0f, zv = 0.0f;
        if (k < n) {
            xv = x[k];
            yv = y[k];
            zv = z[k];
            edge = classify<2, false>(m, xv, yv, zv, r, bits);
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
        rbsm_sample smp;
        fragment_features(m, xv, yv, zv, smp.bits, smp.fx, smp.fy, smp.gap);
        smp.label = r.fil;
        out[slot] = smp;
    }
}

// ----------------------------------------------------------- training --

constexpr int kTrainWarps = 4;
constexpr int kChunk = 16 * kTrainWarps;     // 64 samples per CTA iteration

struct TrainSmem {
    uint16_t w1t[kW1tElems];
    uint16_t w2t[kW2tElems];
    uint16_t w2[kW2Elems];
    uint16_t w3t[kW3tElems];
    uint16_t w3[kW3Elems];
    float b1[kHid], b2[kHid], b3[kOutPad];
    uint16_t x[kChunk * kIn];
    uint16_t h1[kChunk * kHid];
    uint16_t h2[kChunk * kHid];
    uint16_t dy[kChunk * 16];
    uint16_t da2[kChunk * kHid];
    uint16_t da1[kChunk * kHid];
    float label[kChunk];
    float db1[kHid], db2[kHid], db3[kOutPad];
    float loss;
};

// Sum over the 8 lanes that share t = lane % 4 (the rows g of a C tile).
__device__ __forceinline__ float sum_over_g(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// Gradient of the loss over one minibatch (rows order[0..batch) of the
// sample set), accumulated into state.grad, and the loss sum into
// state.loss.  Each CTA takes 64-sample chunks; its four warps run forward
// and the backward-data products on 16 samples each in registers, then all
// four share the chunk's activations (shared memory) for the weight-gradient
// products, whose 52 output tiles they split 13 each.
__global__ void __launch_bounds__(32 * kTrainWarps)
train_grad_kernel(void *base, const rbsm_sample *__restrict__ data, const int *__restrict__ order, int batch,
                  float inv_batch)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smem_raw);
    const State st = state_of(base);
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;

    for (int k = threadIdx.x; k < kW1tElems; k += blockDim.x) sm.w1t[k] = st.w1t[k];
    for (int k = threadIdx.x; k < kW2tElems; k += blockDim.x) { sm.w2t[k] = st.w2t[k]; sm.w2[k] = st.w2[k]; }
    for (int k = threadIdx.x; k < kW3tElems; k += blockDim.x) sm.w3t[k] = st.w3t[k];
    for (int k = threadIdx.x; k < kW3Elems; k += blockDim.x) sm.w3[k] = st.w3[k];
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        sm.b1[k] = st.master[kOffB1 + k];
        sm.b2[k] = st.master[kOffB2 + k];
        sm.db1[k] = 0.0f;
        sm.db2[k] = 0.0f;
    }
    for (int k = threadIdx.x; k < kOutPad; k += blockDim.x) {
        sm.b3[k] = k < kOut ? st.master[kOffB3 + k] : 0.0f;
        sm.db3[k] = 0.0f;
    }
    for (int k = threadIdx.x; k < kChunk * 16; k += blockDim.x)
        sm.dy[k] = 0;
    if (threadIdx.x == 0)
        sm.loss = 0.0f;
    __syncthreads();

    // weight-gradient tiles of this warp: tile q in 0..51 -> (matrix, m-tile, n-tile)
    float acc[13][4];
#pragma unroll
    for (int q = 0; q < 13; ++q)
        acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0f;

    const int chunks = (batch + kChunk - 1) / kChunk;
    for (int ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const int r0 = warp * 16;                      // this warp's rows in the chunk
        // inputs of rows r0..r0+15 (lanes 0..15 write one row each)
        if (lane < 16) {
            const int row = r0 + lane;
            const int b = ch * kChunk + row;
            uint16_t *xr = sm.x + row * kIn;
            if (b < batch) {
                const rbsm_sample s = data[order[b]];
                write_input_row(xr, s.bits, s.fx, s.fy, s.gap);
                sm.label[row] = s.label;
            } else {
                for (int k = 0; k < kIn; ++k) xr[k] = 0;
                sm.label[row] = 0.0f;
            }
        }
        __syncwarp();
        uint32_t xa[2][4];
        load_a(sm.x, kIn, r0, 0, lane, xa[0]);
        load_a(sm.x, kIn, r0, 1, lane, xa[1]);
        HiddenFrags h1, h2;
        uint32_t mask1, mask2;
        layer(xa, 2, sm.w1t, kIn, sm.b1, lane, h1, mask1);
        layer(h1.a, 4, sm.w2t, kHid, sm.b2, lane, h2, mask2);
        float y[4];
        {
            const float bl = sm.b3[2 * t], bh = sm.b3[2 * t + 1];
            y[0] = bl; y[1] = bh; y[2] = bl; y[3] = bh;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t b0, b1;
                load_b(sm.w3t, kHid, kt, 0, lane, b0, b1);
                mma_bf16(y, h2.a[kt], b0, b1);
            }
        }
        // store h1, h2 rows (BF16) for the weight-gradient products
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const int c0 = kt * 16 + 2 * t;
            *reinterpret_cast<uint32_t *>(sm.h1 + (r0 + g) * kHid + c0) = h1.a[kt][0];
            *reinterpret_cast<uint32_t *>(sm.h1 + (r0 + g + 8) * kHid + c0) = h1.a[kt][1];
            *reinterpret_cast<uint32_t *>(sm.h1 + (r0 + g) * kHid + c0 + 8) = h1.a[kt][2];
            *reinterpret_cast<uint32_t *>(sm.h1 + (r0 + g + 8) * kHid + c0 + 8) = h1.a[kt][3];
            *reinterpret_cast<uint32_t *>(sm.h2 + (r0 + g) * kHid + c0) = h2.a[kt][0];
            *reinterpret_cast<uint32_t *>(sm.h2 + (r0 + g + 8) * kHid + c0) = h2.a[kt][1];
            *reinterpret_cast<uint32_t *>(sm.h2 + (r0 + g) * kHid + c0 + 8) = h2.a[kt][2];
            *reinterpret_cast<uint32_t *>(sm.h2 + (r0 + g + 8) * kHid + c0 + 8) = h2.a[kt][3];
        }
        // loss and output gradient (lanes with t == 0 hold columns 0 and 1)
        float dyv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        float lsum = 0.0f;
        if (t == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = r0 + g + 8 * h;
                const bool ok = ch * kChunk + row < batch;
                const float v = y[2 * h], e = y[2 * h + 1], tl = sm.label[row];
                const float vc = fminf(fmaxf(v, 0.0f), 1.0f);
                const float et = fabsf(vc - tl);
                const float rv = v - tl, re = e - et;
                if (ok) {
                    dyv[2 * h] = 2.0f * rv * inv_batch;
                    dyv[2 * h + 1] = 2.0f * re * inv_batch;
                    lsum += rv * rv + re * re;
                }
                *reinterpret_cast<uint32_t *>(sm.dy + row * 16) = pack_bf16(dyv[2 * h], dyv[2 * h + 1]);
            }
        }
        // bias gradient of layer 3 (FP32)
        {
            const float s0 = sum_over_g(dyv[0] + dyv[2]), s1 = sum_over_g(dyv[1] + dyv[3]);
            if (lane == 0) {
                atomicAdd(&sm.db3[0], s0);
                atomicAdd(&sm.db3[1], s1);
            }
        }
        lsum = sum_over_g(lsum);
        if (lane == 0)
            atomicAdd(&sm.loss, lsum);
        // dh2 = dy W3^T (A: dy as one k-tile whose columns 2..15 are zero)
        uint32_t dya[4];
        dya[0] = (t == 0) ? pack_bf16(dyv[0], dyv[1]) : 0u;
        dya[1] = (t == 0) ? pack_bf16(dyv[2], dyv[3]) : 0u;
        dya[2] = 0u;
        dya[3] = 0u;
        HiddenFrags da2f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            uint32_t b0, b1;
            load_b(sm.w3, 16, 0, nt, lane, b0, b1);
            mma_bf16(c, dya, b0, b1);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (!((mask2 >> (4 * nt + q)) & 1u)) c[q] = 0.0f;
            const float s0 = sum_over_g(c[0] + c[2]), s1 = sum_over_g(c[1] + c[3]);
            if (g == 0) {
                atomicAdd(&sm.db2[nt * 8 + 2 * t], s0);
                atomicAdd(&sm.db2[nt * 8 + 2 * t + 1], s1);
            }
            const int kt = nt >> 1, hi = nt & 1;
            da2f.a[kt][hi ? 2 : 0] = pack_bf16(c[0], c[1]);
            da2f.a[kt][hi ? 3 : 1] = pack_bf16(c[2], c[3]);
        }
        // dh1 = da2 W2^T (B^T = W2 as (in, out))
        HiddenFrags da1f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t b0, b1;
                load_b(sm.w2, kHid, kt, nt, lane, b0, b1);
                mma_bf16(c, da2f.a[kt], b0, b1);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (!((mask1 >> (4 * nt + q)) & 1u)) c[q] = 0.0f;
            const float s0 = sum_over_g(c[0] + c[2]), s1 = sum_over_g(c[1] + c[3]);
            if (g == 0) {
                atomicAdd(&sm.db1[nt * 8 + 2 * t], s0);
                atomicAdd(&sm.db1[nt * 8 + 2 * t + 1], s1);
            }
            const int kt = nt >> 1, hi = nt & 1;
            da1f.a[kt][hi ? 2 : 0] = pack_bf16(c[0], c[1]);
            da1f.a[kt][hi ? 3 : 1] = pack_bf16(c[2], c[3]);
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const int c0 = kt * 16 + 2 * t;
            *reinterpret_cast<uint32_t *>(sm.da2 + (r0 + g) * kHid + c0) = da2f.a[kt][0];
            *reinterpret_cast<uint32_t *>(sm.da2 + (r0 + g + 8) * kHid + c0) = da2f.a[kt][1];
            *reinterpret_cast<uint32_t *>(sm.da2 + (r0 + g) * kHid + c0 + 8) = da2f.a[kt][2];
            *reinterpret_cast<uint32_t *>(sm.da2 + (r0 + g + 8) * kHid + c0 + 8) = da2f.a[kt][3];
            *reinterpret_cast<uint32_t *>(sm.da1 + (r0 + g) * kHid + c0) = da1f.a[kt][0];
            *reinterpret_cast<uint32_t *>(sm.da1 + (r0 + g + 8) * kHid + c0) = da1f.a[kt][1];
            *reinterpret_cast<uint32_t *>(sm.da1 + (r0 + g) * kHid + c0 + 8) = da1f.a[kt][2];
            *reinterpret_cast<uint32_t *>(sm.da1 + (r0 + g + 8) * kHid + c0 + 8) = da1f.a[kt][3];
        }
        __syncthreads();
        // weight gradients over the chunk's 64 samples (k = sample):
        //   tiles  0..15: dW1 = X^T da1   (m: 2 tiles of in, n: 8 tiles of out)
        //   tiles 16..47: dW2 = h1^T da2  (4 x 8)
        //   tiles 48..51: dW3 = h2^T dy   (4 x 1)
#pragma unroll
        for (int q = 0; q < 13; ++q) {
            const int tile = warp + 4 * q;
            const uint16_t *am, *bm;
            int lda, ldb, mt, nt;
            if (tile < 16) {
                am = sm.x; lda = kIn; bm = sm.da1; ldb = kHid; mt = tile / 8; nt = tile % 8;
            } else if (tile < 48) {
                am = sm.h1; lda = kHid; bm = sm.da2; ldb = kHid; mt = (tile - 16) / 8; nt = (tile - 16) % 8;
            } else {
                am = sm.h2; lda = kHid; bm = sm.dy; ldb = 16; mt = tile - 48; nt = 0;
            }
#pragma unroll
            for (int ks = 0; ks < kChunk / 16; ++ks) {
                uint32_t a[4], b0, b1;
                load_a_trans(am, lda, mt * 16, ks * 16, lane, a);
                load_b_rows(bm, ldb, ks * 16, nt * 8, lane, b0, b1);
                mma_bf16(acc[q], a, b0, b1);
            }
        }
        __syncthreads();
    }

    // flush: weight tiles, bias sums and loss into the state (FP32 atomics)
#pragma unroll
    for (int q = 0; q < 13; ++q) {
        const int tile = warp + 4 * q;
        int off, ldo, mt, nt, ncols;
        if (tile < 16) {
            off = kOffW1; ldo = kHid; mt = tile / 8; nt = tile % 8; ncols = kHid;
        } else if (tile < 48) {
            off = kOffW2; ldo = kHid; mt = (tile - 16) / 8; nt = (tile - 16) % 8; ncols = kHid;
        } else {
            off = kOffW3; ldo = kOut; mt = tile - 48; nt = 0; ncols = kOut;
        }
        const int m = mt * 16 + g, n = nt * 8 + 2 * t;
        if (n < ncols) {
            atomicAdd(&st.grad[off + m * ldo + n], acc[q][0]);
            atomicAdd(&st.grad[off + (m + 8) * ldo + n], acc[q][2]);
        }
        if (n + 1 < ncols) {
            atomicAdd(&st.grad[off + m * ldo + n + 1], acc[q][1]);
            atomicAdd(&st.grad[off + (m + 8) * ldo + n + 1], acc[q][3]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        atomicAdd(&st.grad[kOffB1 + k], sm.db1[k]);
        atomicAdd(&st.grad[kOffB2 + k], sm.db2[k]);
    }
    if (threadIdx.x < kOut)
        atomicAdd(&st.grad[kOffB3 + threadIdx.x], sm.db3[threadIdx.x]);
    if (threadIdx.x == 0) {
        atomicAdd(&st.loss[0], sm.loss);
    }
}

// Forward pass of n samples (outputs n x 2, FP32): each warp takes 16
// samples at a time.  Used to check the tensor-core forward against the
// reference and to score held-out data.
__global__ void __launch_bounds__(128) forward_kernel(const void *base, const rbsm_sample *__restrict__ data,
                                                      long long n, float *__restrict__ out)
{
    __shared__ SmemWeights w;
    __shared__ __align__(16) uint16_t xs[4][16 * kIn];
    const State st = state_of(const_cast<void *>(base));
    for (int k = threadIdx.x; k < kW1tElems; k += blockDim.x) w.w1t[k] = st.w1t[k];
    for (int k = threadIdx.x; k < kW2tElems; k += blockDim.x) w.w2t[k] = st.w2t[k];
    for (int k = threadIdx.x; k < kW3tElems; k += blockDim.x) w.w3t[k] = st.w3t[k];
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        w.b1[k] = st.master[kOffB1 + k];
        w.b2[k] = st.master[kOffB2 + k];
    }
    for (int k = threadIdx.x; k < kOutPad; k += blockDim.x)
        w.b3[k] = k < kOut ? st.master[kOffB3 + k] : 0.0f;
    __syncthreads();
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const long long tiles = (n + 15) / 16;
    for (long long tl = (long long)blockIdx.x * 4 + warp; tl < tiles; tl += (long long)gridDim.x * 4) {
        if (lane < 16) {
            const long long b = tl * 16 + lane;
            uint16_t *xr = xs[warp] + lane * kIn;
            if (b < n) {
                const rbsm_sample s = data[b];
                write_input_row(xr, s.bits, s.fx, s.fy, s.gap);
            } else {
                for (int k = 0; k < kIn; ++k) xr[k] = 0;
            }
        }
        __syncwarp();
        uint32_t xa[2][4];
        load_a(xs[warp], kIn, 0, 0, lane, xa[0]);
        load_a(xs[warp], kIn, 0, 1, lane, xa[1]);
        HiddenFrags h1, h2;
        uint32_t m1, m2;
        layer(xa, 2, w.w1t, kIn, w.b1, lane, h1, m1);
        layer(h1.a, 4, w.w2t, kHid, w.b2, lane, h2, m2);
        float y[4];
        output_layer(h2, w, lane, y);
        if (t == 0) {
            const long long b0 = tl * 16 + g, b1 = tl * 16 + g + 8;
            if (b0 < n) { out[2 * b0] = y[0]; out[2 * b0 + 1] = y[1]; }
            if (b1 < n) { out[2 * b1] = y[2]; out[2 * b1 + 1] = y[3]; }
        }
        __syncwarp();
    }
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
    if ((rc = check_params(params, &max_dist)) != RBSM_OK) return rc;
    if (!counter || capacity < 0 || (capacity > 0 && !samples))
        return RBSM_ERR_ARG;
    if (frags->n == 0)
        return RBSM_OK;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    long long blocks = (frags->n + 255) / 256;
    if (blocks > (long long)sms * 8)
        blocks = (long long)sms * 8;
    mlp::dataset_kernel<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        to_dev(*map), frags->x, frags->y, frags->z, frags->n, max_dist, samples, capacity, counter);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

int rbsm_mlp_grad(void *state, const rbsm_sample *samples, const int32_t *order, int32_t batch, void *stream)
{
    if (!state || !samples || !order || batch < 1)
        return RBSM_ERR_ARG;
    static KernelSetup setup;
    const size_t smem = sizeof(mlp::TrainSmem);
    int occ = 0;
    int rc = setup.get(mlp::train_grad_kernel, 32 * mlp::kTrainWarps, smem, &occ);
    if (rc != RBSM_OK)
        return rc;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    long long chunks = (batch + mlp::kChunk - 1) / mlp::kChunk;
    long long grid = (long long)sms * occ;
    if (grid > chunks)
        grid = chunks;
    mlp::train_grad_kernel<<<(unsigned)grid, 32 * mlp::kTrainWarps, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
        state, samples, order, batch, 1.0f / (float)batch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
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
    cudaError_t e = cudaSuccess;
    if (grad)
        e = cudaMemcpyAsync(grad, st.grad, mlp::kParams * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && loss)
        e = cudaMemcpyAsync(loss, st.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
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
    if (!state || n < 0 || (n > 0 && (!samples || !out)))
        return RBSM_ERR_ARG;
    if (n == 0)
        return RBSM_OK;
    const int sms = device_sm_count();
    if (sms <= 0)
        return cuda_fail(cudaErrorNoDevice);
    long long blocks = (n + 63) / 64;
    if (blocks > (long long)sms * 8)
        blocks = (long long)sms * 8;
    mlp::forward_kernel<<<(unsigned)blocks, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(state, samples, n,
                                                                                                out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}

}  // extern "C"
