// The learned hit proposal: a 12 -> 64 -> 64 -> 1 perceptron with ReLU that
// scores (candidate, hit) pairs.  The paper has no learned component; this is
// the proposal the build step can use to rank a candidate's in-window hits so
// that only the best k get the full Kalman chi2.
//
// The network's weights are BF16 (W1, W2 and W3, rounded from the FP32 master
// weights when they are loaded), its biases FP32.  Inference runs on the
// tensor cores with FP32 accumulation.  Activations (the inputs and the first
// hidden layer) are carried as a pair of BF16 numbers, hi = bf16(a) and lo =
// bf16(a - hi), and each product is issued twice, once per part: the result
// is the FP32 evaluation of the BF16-weight network to about 2^-16 of each
// activation, so the ranking a build takes from the logits is that of the
// network itself, not of a rounding of its inputs.
//
// One warp scores 32 rows at a time with mma.sync.m16n8k16 (inline PTX).  The
// layer-1 accumulators are turned into the layer-2 A fragments in registers
// (the m16n8 accumulator layout of two adjacent n-tiles is the m16k16 A
// layout), and the last layer (64 -> 1) is a dot product in FP32 reduced over
// the four lanes of a group, so a call touches memory only for its FP32 input
// rows and the weights.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace kf {

constexpr int kMlpIn = 12, kMlpHid = 64;
// flat parameter layout: W1 [12][64], b1 [64], W2 [64][64], b2 [64], W3 [64], b3
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpIn * kMlpHid, kOffW2 = kOffB1 + kMlpHid;
constexpr int kOffB2 = kOffW2 + kMlpHid * kMlpHid, kOffW3 = kOffB2 + kMlpHid, kOffB3 = kOffW3 + kMlpHid;
constexpr int kMlpParams = kOffB3 + 1;  // 5057

// Row strides (in bf16) of the shared-memory copies: W1 and W2 are held
// transposed ([n][k], k contiguous, as the col-major B fragment reads them)
// with rows padded so that the eight rows a fragment load touches fall in
// distinct banks.
constexpr int kW1Ld = 24, kW2Ld = 72;
constexpr int kW1Elems = kMlpHid * kW1Ld, kW2Elems = kMlpHid * kW2Ld;

// Weights as the tensor cores read them (shared memory, per block).
struct __align__(16) MlpSmemWeights {
    __nv_bfloat16 W1t[kW1Elems];  // [64][24]: W1t[n][k] = W1[k][n], k >= 12 zero
    __nv_bfloat16 W2t[kW2Elems];  // [64][72]: W2t[n][k] = W2[k][n], k >= 64 zero
    float b1[kMlpHid], b2[kMlpHid], W3[kMlpHid], b3;
};

// Load the BF16 device copies (prepared by kf_proposal_load in the layout
// above) into shared memory; all threads of the block call it, followed by
// __syncthreads().
__device__ __forceinline__ void mlp_load_weights(MlpSmemWeights *w, const __nv_bfloat16 *W1p, const __nv_bfloat16 *W2p,
                                                 const float *f32)
{
    const uint4 *s1 = reinterpret_cast<const uint4 *>(W1p), *s2 = reinterpret_cast<const uint4 *>(W2p);
    uint4 *d1 = reinterpret_cast<uint4 *>(w->W1t), *d2 = reinterpret_cast<uint4 *>(w->W2t);
    for (int i = threadIdx.x; i < kW1Elems / 8; i += blockDim.x) d1[i] = s1[i];
    for (int i = threadIdx.x; i < kW2Elems / 8; i += blockDim.x) d2[i] = s2[i];
    for (int i = threadIdx.x; i < kMlpHid; i += blockDim.x) {
        w->b1[i] = f32[kOffB1 + i];
        w->b2[i] = f32[kOffB2 + i];
        w->W3[i] = f32[kOffW3 + i];
    }
    if (threadIdx.x == 0) w->b3 = f32[kOffB3];
}

__device__ __forceinline__ void mma_bf16_m16n8k16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                                  uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// A float pair as a BF16 pair (hi) and the BF16 rounding of what hi leaves
// over (lo): hi + lo carries 16 significant bits of each value.
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// Where the scorer reads the network: W1t and W2t in the padded transposed
// BF16 layouts of MlpSmemWeights (as 32-bit pairs), the FP32 biases, the
// BF16-valued W3 (as floats) and b3.  Shared or global memory.
struct MlpWeightsRef {
    const uint32_t *W1, *W2;
    const float *b1, *b2, *W3;
    float b3;
};

// Score 32 input rows X [32][ldx] (FP32, row r belongs to lane r; columns
// 0..11 used) with split activations.  Warp-collective: every lane calls it
// converged.  Returns the logit of the calling lane's row.
//
// Fragment layouts (PTX ISA, mma.m16n8k16 with .bf16): g = lane / 4,
// t = lane % 4; A (16x16, row-major) registers hold rows {g, g+8} x columns
// {2t, 2t+1} and {2t+8, 2t+9}; B (16x8, col-major) rows {2t, 2t+1} and
// {2t+8, 2t+9} of column g; the accumulator rows {g, g+8} x columns {2t, 2t+1}.
__device__ __forceinline__ float mlp_score_warp_split(const MlpWeightsRef &w, const float *X, int ldx)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __syncwarp();
    float zr[2][2];  // [m-tile][row g, row g+8]
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const float *x0 = X + (mt * 16 + g) * ldx, *x1 = x0 + 8 * ldx;
        uint32_t ah[4], al[4];  // layer-1 A fragment, hi and lo
        split_bf16x2(x0[2 * t], x0[2 * t + 1], ah[0], al[0]);
        split_bf16x2(x1[2 * t], x1[2 * t + 1], ah[1], al[1]);
        if (2 * t + 8 < kMlpIn) {
            split_bf16x2(x0[2 * t + 8], x0[2 * t + 9], ah[2], al[2]);
            split_bf16x2(x1[2 * t + 8], x1[2 * t + 9], ah[3], al[3]);
        } else {
            ah[2] = al[2] = ah[3] = al[3] = 0u;
        }
        // layer 1 -> A fragments of layer 2 (k-step ks = n-tiles 2ks, 2ks+1)
        uint32_t a[4][4], b[4][4];  // hi, lo
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n = nt * 8 + g, j = nt * 8 + 2 * t;
            const uint32_t w0 = w.W1[n * (kW1Ld / 2) + t], w1 = w.W1[n * (kW1Ld / 2) + t + 4];
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            mma_bf16_m16n8k16(c, ah[0], ah[1], ah[2], ah[3], w0, w1);
            mma_bf16_m16n8k16(c, al[0], al[1], al[2], al[3], w0, w1);
            const float2 bb = *reinterpret_cast<const float2 *>(w.b1 + j);
            split_bf16x2(fmaxf(c[0] + bb.x, 0.0f), fmaxf(c[1] + bb.y, 0.0f), a[nt >> 1][(nt & 1) * 2 + 0],
                         b[nt >> 1][(nt & 1) * 2 + 0]);
            split_bf16x2(fmaxf(c[2] + bb.x, 0.0f), fmaxf(c[3] + bb.y, 0.0f), a[nt >> 1][(nt & 1) * 2 + 1],
                         b[nt >> 1][(nt & 1) * 2 + 1]);
        }
        // layer 2, one n-tile at a time, folded into the 64 -> 1 dot product
        float z0 = 0.0f, z1 = 0.0f;
#pragma unroll 1
        for (int nt = 0; nt < 8; ++nt) {
            const int n = nt * 8 + g, j = nt * 8 + 2 * t;
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t w0 = w.W2[n * (kW2Ld / 2) + ks * 8 + t], w1 = w.W2[n * (kW2Ld / 2) + ks * 8 + t + 4];
                mma_bf16_m16n8k16(c, a[ks][0], a[ks][1], a[ks][2], a[ks][3], w0, w1);
                mma_bf16_m16n8k16(c, b[ks][0], b[ks][1], b[ks][2], b[ks][3], w0, w1);
            }
            const float2 bb = *reinterpret_cast<const float2 *>(w.b2 + j);
            const float2 ww = *reinterpret_cast<const float2 *>(w.W3 + j);
            z0 = fmaf(ww.x, fmaxf(c[0] + bb.x, 0.0f), fmaf(ww.y, fmaxf(c[1] + bb.y, 0.0f), z0));
            z1 = fmaf(ww.x, fmaxf(c[2] + bb.x, 0.0f), fmaf(ww.y, fmaxf(c[3] + bb.y, 0.0f), z1));
        }
        z0 += __shfl_xor_sync(0xffffffffu, z0, 1);
        z0 += __shfl_xor_sync(0xffffffffu, z0, 2);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 1);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 2);
        zr[mt][0] = z0;
        zr[mt][1] = z1;
    }
    // row `lane` lives in group lane % 8 as (m-tile lane / 16, half (lane / 8) % 2)
    const int src = (lane & 7) * 4;
    const float v00 = __shfl_sync(0xffffffffu, zr[0][0], src), v01 = __shfl_sync(0xffffffffu, zr[0][1], src);
    const float v10 = __shfl_sync(0xffffffffu, zr[1][0], src), v11 = __shfl_sync(0xffffffffu, zr[1][1], src);
    const int mt = lane >> 4, half = (lane >> 3) & 1;
    const float z = mt ? (half ? v11 : v10) : (half ? v01 : v00);
    __syncwarp();
    return z + w.b3;
}

}  // namespace kf
