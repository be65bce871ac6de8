// The learned hit proposal: a 12 -> 64 -> 64 -> 1 perceptron with ReLU that
// scores (candidate, hit) pairs.  The paper has no learned component; this is
// the proposal the build step can use to rank a candidate's in-window hits so
// that only the best k get the full Kalman chi2.
//
// Inference runs on the tensor cores in BF16 with FP32 accumulation, one warp
// scoring 32 rows at a time (warp-level mma.sync through nvcuda::wmma,
// m16n16k16): the build kernel scores at most a few dozen hits per warp per
// layer, inside a per-warp loop, where CTA-wide tcgen05 tiles do not fit.
#pragma once

#include <cuda_bf16.h>
#include <mma.h>
#include <stdint.h>

namespace kf {

constexpr int kMlpIn = 12, kMlpInPad = 16, kMlpHid = 64;
// flat parameter layout: W1 [12][64], b1 [64], W2 [64][64], b2 [64], W3 [64], b3
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpIn * kMlpHid, kOffW2 = kOffB1 + kMlpHid;
constexpr int kOffB2 = kOffW2 + kMlpHid * kMlpHid, kOffW3 = kOffB2 + kMlpHid, kOffB3 = kOffW3 + kMlpHid;
constexpr int kMlpParams = kOffB3 + 1;  // 5057

// Weights as the tensor cores read them (shared memory, per block).
struct __align__(128) MlpSmemWeights {
    __nv_bfloat16 W1[kMlpInPad * kMlpHid];  // [16][64], rows 12..15 zero
    __nv_bfloat16 W2[kMlpHid * kMlpHid];    // [64][64]
    float b1[kMlpHid], b2[kMlpHid], W3[kMlpHid], b3;
};

// Per-warp staging for 32 rows.
struct __align__(128) MlpWarpStage {
    __nv_bfloat16 X[32 * kMlpInPad];  // inputs, [32][16]
    __nv_bfloat16 H1[32 * kMlpHid];   // first hidden layer after ReLU
    float acc[32 * kMlpHid];          // accumulator staging
};

// Load the BF16 device copies (prepared by kf_proposal_load) into shared
// memory; all threads of the block call it, followed by __syncthreads().
__device__ __forceinline__ void mlp_load_weights(MlpSmemWeights *w, const __nv_bfloat16 *W1p, const __nv_bfloat16 *W2p,
                                                 const float *f32)
{
    for (int i = threadIdx.x; i < kMlpInPad * kMlpHid; i += blockDim.x) w->W1[i] = W1p[i];
    for (int i = threadIdx.x; i < kMlpHid * kMlpHid; i += blockDim.x) w->W2[i] = W2p[i];
    for (int i = threadIdx.x; i < kMlpHid; i += blockDim.x) {
        w->b1[i] = f32[kOffB1 + i];
        w->b2[i] = f32[kOffB2 + i];
        w->W3[i] = f32[kOffW3 + i];
    }
    if (threadIdx.x == 0) w->b3 = f32[kOffB3];
}

// Score the 32 rows of st->X (row r belongs to lane r; rows a lane does not
// use may hold anything).  Warp-collective: every lane of the warp calls it
// converged.  Returns the logit of the calling lane's row.
__device__ __forceinline__ float mlp_score_warp(const MlpSmemWeights *w, MlpWarpStage *st)
{
    using namespace nvcuda;
    const int lane = threadIdx.x & 31;
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> a;
        wmma::load_matrix_sync(a, st->X + m * 16 * kMlpInPad, kMlpInPad);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
            wmma::fragment<wmma::accumulator, 16, 16, 16, float> c;
            wmma::fill_fragment(c, 0.0f);
            wmma::load_matrix_sync(b, w->W1 + n * 16, kMlpHid);
            wmma::mma_sync(c, a, b, c);
            wmma::store_matrix_sync(st->acc + m * 16 * kMlpHid + n * 16, c, kMlpHid, wmma::mem_row_major);
        }
    }
    __syncwarp();
#pragma unroll 8
    for (int j = 0; j < kMlpHid; ++j)
        st->H1[lane * kMlpHid + j] = __float2bfloat16(fmaxf(st->acc[lane * kMlpHid + j] + w->b1[j], 0.0f));
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 2; ++m) {
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            wmma::fragment<wmma::accumulator, 16, 16, 16, float> c;
            wmma::fill_fragment(c, 0.0f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> a;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
                wmma::load_matrix_sync(a, st->H1 + m * 16 * kMlpHid + k * 16, kMlpHid);
                wmma::load_matrix_sync(b, w->W2 + k * 16 * kMlpHid + n * 16, kMlpHid);
                wmma::mma_sync(c, a, b, c);
            }
            wmma::store_matrix_sync(st->acc + m * 16 * kMlpHid + n * 16, c, kMlpHid, wmma::mem_row_major);
        }
    }
    __syncwarp();
    float z = w->b3;
#pragma unroll 8
    for (int j = 0; j < kMlpHid; ++j) z = fmaf(w->W3[j], fmaxf(st->acc[lane * kMlpHid + j] + w->b2[j], 0.0f), z);
    __syncwarp();
    return z;
}

}  // namespace kf
