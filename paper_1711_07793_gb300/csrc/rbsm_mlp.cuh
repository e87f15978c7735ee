// Tensor-core building blocks of the learned penumbra surrogate (sm_103a).
//
// The surrogate is this project's addition (the paper has no network): a
// 32-64-64-2 perceptron on the 5x5 shadow-test pattern of an edge fragment,
// its in-texel offsets and its blocker-receiver depth gap.  BF16 operands,
// FP32 accumulation; everything around the products (bias, ReLU, loss,
// guard) is FP32 on the CUDA cores.  Training and the stand-alone forward
// pass run on tcgen05 (rbsm_learned.cu, 128-sample tiles); the guarded
// inference inside the batched visibility kernel takes the edge fragments
// of one warp, 32 at a time, with the warp-level mma.sync m16n8k16 tiles
// below.
//
// Fragment layouts of mma.m16n8k16 (g = lane / 4, t = lane % 4):
//   A (16 x 16, row-major): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..2t+1],
//                           a2 = A[g][2t+8..2t+9], a3 = A[g+8][2t+8..2t+9]
//   B (16 x 8), given as its transpose Bt[n][k]: b0 = Bt[g][2t..2t+1],
//                           b1 = Bt[g][2t+8..2t+9]
//   C (16 x 8, FP32):       c0, c1 = C[g][2t..2t+1], c2, c3 = C[g+8][2t..2t+1]
// Two adjacent C tiles of one layer are, after rounding to BF16, exactly
// the A fragment of the next layer's k-tile, so a warp chains the three
// layers of 16 samples in registers.
#pragma once

#include <cuda_bf16.h>
#include <cstddef>
#include <cstdint>

namespace rbsm {
namespace mlp {

constexpr int kIn = 32;        // 25 pattern bits, fx, fy, gap, 4 zeros
constexpr int kHid = 64;
constexpr int kOut = 2;        // visibility estimate, estimate of its error
constexpr int kOutPad = 8;     // one n-tile
constexpr int kPatternBits = 25;

// FP32 parameter vector, canonical order (weights as (in, out), row-major).
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kIn * kHid;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kOut;
constexpr int kParams = kOffB3 + kOut;           // 6402

// BF16 copies the kernels read (elements).
constexpr int kW1tElems = kHid * kIn;            // [out 64][in 32]   forward layer 1
constexpr int kW2tElems = kHid * kHid;           // [out 64][in 64]   forward layer 2
constexpr int kW3tElems = kOutPad * kHid;        // [out 8][in 64]    forward layer 3 (rows 2..7 zero)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // round to nearest even
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint16_t float_to_bf16(float f)
{
    __nv_bfloat16 v = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t *>(&v);
}

// D = A * B + C on one m16n8k16 tile.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragment of k-tile kt, n-tile nt from a transposed matrix Bt[n][k]
// (row pitch ld elements, BF16) in the network state in global memory,
// read through the read-only path.
__device__ __forceinline__ void load_b(const uint16_t *__restrict__ bt, int ld, int kt, int nt, unsigned lane,
                                       uint32_t &b0, uint32_t &b1)
{
    const int g = lane >> 2, t = lane & 3;
    const uint16_t *p = bt + (nt * 8 + g) * ld + kt * 16 + 2 * t;
    b0 = __ldg(reinterpret_cast<const unsigned int *>(p));
    b1 = __ldg(reinterpret_cast<const unsigned int *>(p + 8));
}

// A fragment of m-tile rows [r0, r0+16), k-tile kt, from a row-major BF16
// matrix A[row][k] (pitch ld) in shared memory.
__device__ __forceinline__ void load_a(const uint16_t *a, int ld, int r0, int kt, unsigned lane, uint32_t (&f)[4])
{
    const int g = lane >> 2, t = lane & 3;
    const uint16_t *p = a + (r0 + g) * ld + kt * 16 + 2 * t;
    f[0] = *reinterpret_cast<const uint32_t *>(p);
    f[1] = *reinterpret_cast<const uint32_t *>(p + 8 * ld);
    f[2] = *reinterpret_cast<const uint32_t *>(p + 8);
    f[3] = *reinterpret_cast<const uint32_t *>(p + 8 * ld + 8);
}

// Layout of the network state block (bytes; sections 256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kByteMaster = 0;
constexpr size_t kByteGrad = kByteMaster + align256(kParams * 4);
constexpr size_t kByteM = kByteGrad + align256(kParams * 4);
constexpr size_t kByteV = kByteM + align256(kParams * 4);
constexpr size_t kByteW1t = kByteV + align256(kParams * 4);
constexpr size_t kByteW2t = kByteW1t + align256(kW1tElems * 2);
constexpr size_t kByteW3t = kByteW2t + align256(kW2tElems * 2);
constexpr size_t kByteLoss = kByteW3t + align256(kW3tElems * 2);
// Training partials: one row per CTA of the gradient kernel, the CTA's sums
// over its samples of every parameter's gradient (canonical order) and, at
// index kParams, of the loss.  Reduced in a fixed order afterwards, so a
// gradient does not depend on which CTA finishes first.
constexpr int kPartStride = 6464;                // floats per CTA row (>= kParams + 1)
constexpr int kMaxGradCtas = 256;
constexpr size_t kBytePart = kByteLoss + 256;
// Trusted 5x5 shadow-test patterns: one bit per 25-bit pattern (bit p & 31
// of word p >> 5), set by calibration; consulted when the trust word of the
// loss section is nonzero.
constexpr int kTrustWords = 1 << 20;
constexpr size_t kByteTrust = kBytePart + align256((size_t)kMaxGradCtas * kPartStride * 4);
constexpr size_t kStateBytes = kByteTrust + (size_t)kTrustWords * 4;
constexpr size_t kByteBf16 = kByteW1t;
constexpr size_t kBf16Bytes = kByteLoss - kByteW1t;
static_assert(kPartStride >= kParams + 1, "partial row holds every parameter and the loss");

struct State {
    float *master, *grad, *m, *v;
    uint16_t *w1t, *w2t, *w3t;
    float *loss;              // [0] sum of per-sample losses, [1] samples
    unsigned *status;         // RBSM_ERR_* recorded by a kernel (0 = none)
    float *part;              // kMaxGradCtas x kPartStride training partials
    unsigned *trust_on;       // nonzero: the trust bitmap is in force
    uint32_t *trust;          // kTrustWords words
};

__host__ __device__ inline State state_of(void *base)
{
    char *b = reinterpret_cast<char *>(base);
    return State{reinterpret_cast<float *>(b + kByteMaster), reinterpret_cast<float *>(b + kByteGrad),
                 reinterpret_cast<float *>(b + kByteM), reinterpret_cast<float *>(b + kByteV),
                 reinterpret_cast<uint16_t *>(b + kByteW1t), reinterpret_cast<uint16_t *>(b + kByteW2t),
                 reinterpret_cast<uint16_t *>(b + kByteW3t), reinterpret_cast<float *>(b + kByteLoss),
                 reinterpret_cast<unsigned *>(b + kByteLoss + 16), reinterpret_cast<float *>(b + kBytePart),
                 reinterpret_cast<unsigned *>(b + kByteLoss + 20), reinterpret_cast<uint32_t *>(b + kByteTrust)};
}

// Whether a 5x5 pattern is trusted (always, when no bitmap is in force).
__device__ __forceinline__ bool pattern_trusted(const uint32_t *trust, uint32_t pattern)
{
    return trust == nullptr || ((__ldg(trust + (pattern >> 5)) >> (pattern & 31u)) & 1u) != 0;
}

// One network as the inference kernels read it: the biases in shared
// memory, the three weight matrices where the state holds them (13 KB of
// global memory that every warp of an SM reads through the same L1 lines).
// Keeping the matrices out of shared memory lets the guarded batch kernel
// run four CTAs of 256 per SM instead of three (measured on 8 C5 frames:
// 0.575 against 0.623 ms per step, the same answers).
struct InferWeights {
    float b1[kHid];
    float b2[kHid];
    float b3[kOutPad];
    const uint16_t *w1t, *w2t, *w3t;
};

// Forward pass of one m-tile of 16 samples whose inputs are the A
// fragments x[2][4] (k-tiles 0 and 1).  Returns the output C tile (only
// columns 0 and 1 are meaningful) and, when wanted, the ReLU masks (bit
// 4*nt + q of mask1/mask2 for element q of n-tile nt) and the BF16 hidden
// activations h1/h2 as A fragments of the next layer.
struct HiddenFrags {
    uint32_t a[4][4];          // 4 k-tiles of 16 hidden units
};

__device__ __forceinline__ void layer(const uint32_t (*ain)[4], int ktiles, const uint16_t *wt, int ldw,
                                      const float *bias, unsigned lane, HiddenFrags &out, uint32_t &mask)
{
    const int t = lane & 3;
    mask = 0;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float bl = bias[nt * 8 + 2 * t], bh = bias[nt * 8 + 2 * t + 1];
        float c[4] = {bl, bh, bl, bh};
        for (int kt = 0; kt < ktiles; ++kt) {
            uint32_t b0, b1;
            load_b(wt, ldw, kt, nt, lane, b0, b1);
            mma_bf16(c, ain[kt], b0, b1);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (c[q] > 0.0f)
                mask |= 1u << (4 * nt + q);
            c[q] = fmaxf(c[q], 0.0f);
        }
        // C tile nt -> half of the A fragment of k-tile nt / 2
        const int kt = nt >> 1, hi = nt & 1;
        out.a[kt][hi ? 2 : 0] = pack_bf16(c[0], c[1]);
        out.a[kt][hi ? 3 : 1] = pack_bf16(c[2], c[3]);
    }
}

__device__ __forceinline__ void output_layer(const HiddenFrags &h2, const uint16_t *w3t, const float *b3, unsigned lane,
                                             float (&y)[4])
{
    const int t = lane & 3;
    const float bl = b3[2 * t], bh = b3[2 * t + 1];
    y[0] = bl; y[1] = bh; y[2] = bl; y[3] = bh;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        uint32_t b0, b1;
        load_b(w3t, kHid, kt, 0, lane, b0, b1);
        mma_bf16(y, h2.a[kt], b0, b1);
    }
}

// Input row of one sample: 25 pattern bits, fx, fy, gap, zeros; written as
// 32 BF16 values (the bits and zeros are exact in BF16).
__device__ __forceinline__ void write_input_row(uint16_t *row, uint32_t bits, float fx, float fy, float gap)
{
    uint32_t *r32 = reinterpret_cast<uint32_t *>(row);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const uint32_t lo = (bits >> (2 * k)) & 1u, hi = (bits >> (2 * k + 1)) & 1u;
        r32[k] = (lo ? 0x3F80u : 0u) | ((hi ? 0x3F80u : 0u) << 16);     // 1.0 in BF16 is 0x3F80
    }
    r32[12] = (((bits >> 24) & 1u) ? 0x3F80u : 0u) | ((uint32_t)float_to_bf16(fx) << 16);
    r32[13] = (uint32_t)float_to_bf16(fy) | ((uint32_t)float_to_bf16(gap) << 16);
    r32[14] = 0u;
    r32[15] = 0u;
}

}  // namespace mlp
}  // namespace rbsm
