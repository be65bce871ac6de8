// Training and batched inference of the learned hit proposal (kf_mlp.cuh).
//
// Training runs in FP32 (master weights, gradients and Adam moments): each
// block takes a tile of 64 samples, computes the forward pass, the binary
// cross-entropy on the logits and the backward pass in shared memory, and adds
// its part of the weight gradients to a global buffer; an Adam kernel then
// updates the weights.  Inference copies the weights to BF16 and scores on the
// tensor cores (mlp_score_warp).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kf.h"
#include "kf_api_internal.h"
#include "kf_mlp.cuh"

namespace kf {

struct MlpState {
    float *grad = nullptr, *m = nullptr, *v = nullptr;  // [kMlpParams] each
    float *loss = nullptr;                              // one accumulator
    float *w32 = nullptr;                               // loaded weights, FP32
    __nv_bfloat16 *W1 = nullptr, *W2 = nullptr;         // loaded weights, BF16, transposed and padded
    unsigned *status = nullptr;                         // set by a tcgen05 scoring wait that expired
    bool loaded = false;
};

void destroy_mlp_state(MlpState *s)
{
    if (!s) return;
    cudaFree(s->grad);
    cudaFree(s->m);
    cudaFree(s->v);
    cudaFree(s->loss);
    cudaFree(s->w32);
    cudaFree(s->W1);
    cudaFree(s->W2);
    cudaFree(s->status);
    delete s;
}

bool proposal_loaded(kf_context *ctx)
{
    MlpState *s = context_mlp_state(ctx);
    return s && s->loaded;
}

void proposal_weights(kf_context *ctx, const __nv_bfloat16 **W1, const __nv_bfloat16 **W2, const float **w32)
{
    MlpState *s = context_mlp_state(ctx);
    *W1 = s->W1;
    *W2 = s->W2;
    *w32 = s->w32;
}

namespace {

constexpr int kTile = 64, kTrainThreads = 256;

struct TrainSmem {
    float X[kTile][kMlpIn];
    float H1[kTile][kMlpHid];
    float H2[kTile][kMlpHid];
    float dH2[kTile][kMlpHid];
    float dH1[kTile][kMlpHid];
    float dz[kTile];
    float W1[kMlpIn][kMlpHid];
    float W2[kMlpHid][kMlpHid];
    float b1[kMlpHid], b2[kMlpHid], W3[kMlpHid], b3;
};

// Samples [start, start + count) of the epoch's order, sample = (j P + off) mod n.
__global__ void __launch_bounds__(kTrainThreads) mlp_grad_kernel(const float *w, const float *X, const float *y, int64_t n,
                                                                 int64_t start, int64_t count, int64_t P, int64_t off,
                                                                 float inv_batch, float *grad, float *loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &s = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t j0 = start + (int64_t)blockIdx.x * kTile;
    for (int i = tid; i < kMlpIn * kMlpHid; i += kTrainThreads) s.W1[i / kMlpHid][i % kMlpHid] = w[kOffW1 + i];
    for (int i = tid; i < kMlpHid * kMlpHid; i += kTrainThreads) s.W2[i / kMlpHid][i % kMlpHid] = w[kOffW2 + i];
    for (int i = tid; i < kMlpHid; i += kTrainThreads) {
        s.b1[i] = w[kOffB1 + i];
        s.b2[i] = w[kOffB2 + i];
        s.W3[i] = w[kOffW3 + i];
    }
    if (tid == 0) s.b3 = w[kOffB3];
    for (int i = tid; i < kTile * kMlpIn; i += kTrainThreads) {
        const int r = i / kMlpIn, f = i % kMlpIn;
        const int64_t j = j0 + r;
        float val = 0.0f;
        if (j < start + count) val = X[((j * P + off) % n) * kMlpIn + f];
        s.X[r][f] = val;
    }
    __syncthreads();
    for (int i = tid; i < kTile * kMlpHid; i += kTrainThreads) {  // H1 = relu(X W1 + b1)
        const int r = i / kMlpHid, u = i % kMlpHid;
        float a = s.b1[u];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) a = fmaf(s.X[r][k], s.W1[k][u], a);
        s.H1[r][u] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (int i = tid; i < kTile * kMlpHid; i += kTrainThreads) {  // H2 = relu(H1 W2 + b2)
        const int r = i / kMlpHid, u = i % kMlpHid;
        float a = s.b2[u];
#pragma unroll 16
        for (int k = 0; k < kMlpHid; ++k) a = fmaf(s.H1[r][k], s.W2[k][u], a);
        s.H2[r][u] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    if (tid < kTile) {  // logit, loss, dL/dz
        const int64_t j = j0 + tid;
        float z = s.b3;
#pragma unroll 16
        for (int k = 0; k < kMlpHid; ++k) z = fmaf(s.H2[tid][k], s.W3[k], z);
        float d = 0.0f, l = 0.0f;
        if (j < start + count) {
            const float t = y[(j * P + off) % n];
            l = fmaxf(z, 0.0f) - z * t + log1pf(expf(-fabsf(z)));
            d = (1.0f / (1.0f + expf(-z)) - t) * inv_batch;
        }
        s.dz[tid] = d;
        // warp sum of the loss, one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((tid & 31) == 0) atomicAdd(loss, l);
    }
    __syncthreads();
    for (int i = tid; i < kTile * kMlpHid; i += kTrainThreads) {  // dH2 = dz W3^T on active units
        const int r = i / kMlpHid, u = i % kMlpHid;
        s.dH2[r][u] = s.H2[r][u] > 0.0f ? s.dz[r] * s.W3[u] : 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < kTile * kMlpHid; i += kTrainThreads) {  // dH1 = dH2 W2^T on active units
        const int r = i / kMlpHid, k = i % kMlpHid;
        float a = 0.0f;
        if (s.H1[r][k] > 0.0f) {
#pragma unroll 16
            for (int u = 0; u < kMlpHid; ++u) a = fmaf(s.dH2[r][u], s.W2[k][u], a);
        }
        s.dH1[r][k] = a;
    }
    __syncthreads();
    // this tile's share of the gradient
    for (int i = tid; i < kMlpHid * kMlpHid; i += kTrainThreads) {
        const int k = i / kMlpHid, u = i % kMlpHid;
        float a = 0.0f;
        for (int r = 0; r < kTile; ++r) a = fmaf(s.H1[r][k], s.dH2[r][u], a);
        atomicAdd(&grad[kOffW2 + i], a);
    }
    for (int i = tid; i < kMlpIn * kMlpHid; i += kTrainThreads) {
        const int f = i / kMlpHid, u = i % kMlpHid;
        float a = 0.0f;
        for (int r = 0; r < kTile; ++r) a = fmaf(s.X[r][f], s.dH1[r][u], a);
        atomicAdd(&grad[kOffW1 + i], a);
    }
    for (int u = tid; u < kMlpHid; u += kTrainThreads) {
        float g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
        for (int r = 0; r < kTile; ++r) {
            g1 += s.dH1[r][u];
            g2 += s.dH2[r][u];
            g3 = fmaf(s.H2[r][u], s.dz[r], g3);
        }
        atomicAdd(&grad[kOffB1 + u], g1);
        atomicAdd(&grad[kOffB2 + u], g2);
        atomicAdd(&grad[kOffW3 + u], g3);
    }
    if (tid == 0) {
        float g = 0.0f;
        for (int r = 0; r < kTile; ++r) g += s.dz[r];
        atomicAdd(&grad[kOffB3], g);
    }
}

// Adam (Kingma and Ba) on every parameter, then clear the gradient.
__global__ void adam_kernel(float *w, float *grad, float *m, float *v, int t, float lr, float b1, float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(b1, (float)t)), vh = vi / (1.0f - powf(b2, (float)t));
    w[i] -= lr * mh / (sqrtf(vh) + eps);
    grad[i] = 0.0f;
}

// FP32 master weights -> the network inference uses: W1 and W2 as the
// transposed, padded BF16 copies the tensor cores read, W3 rounded to BF16 in
// place in the FP32 copy (w32), the biases left in FP32.
__global__ void to_bf16_kernel(float *w32, __nv_bfloat16 *W1t, __nv_bfloat16 *W2t)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kW1Elems; i += gridDim.x * blockDim.x) {
        const int n = i / kW1Ld, k = i % kW1Ld;
        W1t[i] = __float2bfloat16(k < kMlpIn ? w32[kOffW1 + k * kMlpHid + n] : 0.0f);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kW2Elems; i += gridDim.x * blockDim.x) {
        const int n = i / kW2Ld, k = i % kW2Ld;
        W2t[i] = __float2bfloat16(k < kMlpHid ? w32[kOffW2 + k * kMlpHid + n] : 0.0f);
    }
    __syncthreads();  // every W1/W2 read above precedes this block's W3 writes (disjoint ranges anyway)
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < kMlpHid; i += blockDim.x)
            w32[kOffW3 + i] = __bfloat162float(__float2bfloat16(w32[kOffW3 + i]));
}

constexpr int kScoreWarps = 4, kScoreLd = 12;
// kf_proposal_score's engine (KF_SCORE_AUTO), chosen by measurement on one
// GB300: mma.sync below this many rows (at 65,536 rows 0.015 against 0.025
// ms), tcgen05 from it on (1.24x faster at 2^20 rows, 1.68x at 2^24)
constexpr int64_t kScoreTcMinRows = 262144;

struct ScoreSmem {
    MlpSmemWeights w;
    float X[kScoreWarps][32 * kScoreLd];
};

// Each warp scores 32 rows at a time on the tensor cores (mma.sync, split
// activations).
__global__ void __launch_bounds__(32 * kScoreWarps) mlp_score_kernel(const __nv_bfloat16 *W1, const __nv_bfloat16 *W2,
                                                                     const float *w32, const float *X, int64_t n,
                                                                     float *logits)
{
    extern __shared__ __align__(128) unsigned char score_smem_raw[];
    ScoreSmem &s = *reinterpret_cast<ScoreSmem *>(score_smem_raw);
    mlp_load_weights(&s.w, W1, W2, w32);
    __syncthreads();
    const MlpWeightsRef mw{reinterpret_cast<const uint32_t *>(s.w.W1t), reinterpret_cast<const uint32_t *>(s.w.W2t),
                           s.w.b1, s.w.b2, s.w.W3, s.w.b3};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *xs = s.X[warp];
    const int64_t n_chunks = (n + 31) / 32;
    for (int64_t ch = (int64_t)blockIdx.x * kScoreWarps + warp; ch < n_chunks; ch += (int64_t)gridDim.x * kScoreWarps) {
        const int64_t row = ch * 32 + lane;
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) xs[lane * kScoreLd + i] = row < n ? X[row * kMlpIn + i] : 0.0f;
        const float z = mlp_score_warp_split(mw, xs, kScoreLd);
        if (row < n) logits[row] = z;
    }
}

// ---------------------------------------------------------------------------
// The same scoring on the fifth-generation tensor cores (tcgen05): one CTA of
// 128 threads scores 128-row tiles.  The weights are staged once per CTA in
// shared memory; per tile the rows' split inputs go to shared memory, one
// thread issues the layer-1 products (hi and lo parts into one TMEM
// accumulator, M = 128, N = 64, K = 16), the four warps read the accumulator
// back from TMEM (warp w owns TMEM lanes 32w..32w+31, thread t row t), add the
// bias, apply the ReLU, split the result and write it as the layer-2 A operand;
// the layer-2 products (4 K-steps x hi/lo) accumulate into a second TMEM
// region, which the warps read back for the 64 -> 1 dot product.
//
// Operands are K-major without swizzle, in core matrices of 8 rows x 16 bytes
// (8 BF16 values): element (r, k) of a tile with K columns is at byte
// ((r / 8) (K / 8) + k / 8) 128 + (r % 8) 16 + (k % 8) 2.  In the shared
// memory descriptor the leading-dimension offset is the distance between core
// matrices adjacent in K (128 B) and the stride-dimension offset the distance
// between 8-row groups ((K / 8) 128 B).

constexpr int kTcRows = 128, kTcCols = 128;  // rows per tile; TMEM columns (two 64-column accumulators)
constexpr int kTcCtasPerSm = 4;               // 4 x 128 = the SM's 512 TMEM columns (and ~52 KB of
                                              // shared memory each: a fifth cannot be resident)
constexpr uint32_t kTcWaitLimit = 1u << 24;   // mbarrier polls before a wait gives up

struct __align__(128) TcSmem {
    uint8_t A1h[kTcRows * 32], A1l[kTcRows * 32];    // inputs, K = 16 (12 used, 3 bias columns)
    uint8_t A2h[kTcRows * 128], A2l[kTcRows * 128];  // first hidden layer, K = 64
    uint8_t B1[kMlpHid * 32];                         // W1^T and b1's parts: N = 64 x K = 16
    uint8_t B2[kMlpHid * 128];                        // W2^T: N = 64 x K = 64
    uint8_t B2b[kMlpHid * 32];                        // b2's parts: N = 64 x K = 16 (3 used)
    float W3[kMlpHid], b3;
    unsigned long long mbar;
    uint32_t taddr;
};

// A bias b as three BF16 parts whose sum is b exactly (8 significant bits
// each: FP32's 24), so that a product with 1.0 on the tensor cores adds b.
__device__ __forceinline__ void bf16_parts3(float b, __nv_bfloat16 p[3])
{
    p[0] = __float2bfloat16(b);
    const float r1 = b - __bfloat162float(p[0]);
    p[1] = __float2bfloat16(r1);
    p[2] = __float2bfloat16(r1 - __bfloat162float(p[1]));
}

__device__ __forceinline__ uint32_t core_offset(int r, int k, int K)
{
    return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared memory matrix descriptor (tcgen05): start address, leading- and
// stride-dimension byte offsets (all >> 4), the fixed version bits 46..48 =
// 0b001, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A
// and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kMlpHid >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(unsigned long long *mbar)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(mbar);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(a) : "memory");
}

// Wait for the mbarrier's phase `parity` to complete, polling at most
// kTcWaitLimit times; false if it did not.
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, uint32_t parity)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(mbar);
    for (uint32_t i = 0; i < kTcWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 columns of this thread's TMEM lane, without the wait
// (tmem_wait() before the values are used).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void st_shared_v4(uint8_t *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    *reinterpret_cast<uint4 *>(p) = make_uint4(a, b, c, d);
}

__global__ void __launch_bounds__(kTcRows, kTcCtasPerSm) mlp_score_tc_kernel(const float *w32, const float *X,
                                                                              int64_t n, float *logits,
                                                                              unsigned *status)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    TcSmem &s = *reinterpret_cast<TcSmem *>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights: W1^T with b1's parts as its K rows 12..14, W2^T, and b2's parts
    // (K rows 0..2 of B2b), in BF16, K-major core matrices
    for (int nn = tid; nn < kMlpHid; nn += kTcRows) {
        __nv_bfloat16 p1[3], p2[3];
        bf16_parts3(w32[kOffB1 + nn], p1);
        bf16_parts3(w32[kOffB2 + nn], p2);
        for (int k = 0; k < 16; ++k) {
            const __nv_bfloat16 v = k < kMlpIn ? __float2bfloat16(w32[kOffW1 + k * kMlpHid + nn])
                                    : k < kMlpIn + 3 ? p1[k - kMlpIn]
                                                     : __float2bfloat16(0.0f);
            *reinterpret_cast<__nv_bfloat16 *>(s.B1 + core_offset(nn, k, 16)) = v;
            *reinterpret_cast<__nv_bfloat16 *>(s.B2b + core_offset(nn, k, 16)) = k < 3 ? p2[k] : __float2bfloat16(0.0f);
        }
        s.W3[nn] = w32[kOffW3 + nn];
    }
    for (int i = tid; i < kMlpHid * kMlpHid; i += kTcRows) {
        const int nn = i >> 6, k = i & 63;
        *reinterpret_cast<__nv_bfloat16 *>(s.B2 + core_offset(nn, k, 64)) =
            __float2bfloat16(w32[kOffW2 + k * kMlpHid + nn]);
    }
    if (tid == 0) {
        s.b3 = w32[kOffB3];
        const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&s.mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(&s.taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(a), "n"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the staged weights, for the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s.taddr;
    const uint32_t d1 = tmem, d2 = tmem + kMlpHid;      // accumulators: columns 0..63 and 64..127
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lanes
    const float b3 = s.b3;
    uint32_t parity = 0;
    bool failed = false;
    const int64_t tiles = (n + kTcRows - 1) / kTcRows;
    // row `tid` of a tile's inputs; the next tile's are loaded while the
    // current tile's products run
    auto load_row = [&](int64_t tile, float f[kMlpIn]) {
        const int64_t row = tile * kTcRows + tid;
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) f[i] = (tile < tiles && row < n) ? __ldcs(X + row * kMlpIn + i) : 0.0f;
    };
    float fin[kMlpIn];
    load_row(blockIdx.x, fin);
    for (int64_t tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
        const int64_t row = tile * kTcRows + tid;
        // inputs of row `tid` and three 1s (the bias columns), split into BF16
        // hi and lo (1 is exact: its lo part is 0)
        float f[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) f[i] = i < kMlpIn ? fin[i] : i < kMlpIn + 3 ? 1.0f : 0.0f;
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split_bf16x2(f[2 * i], f[2 * i + 1], h[i], l[i]);
#pragma unroll
        for (int kg = 0; kg < 2; ++kg) {
            st_shared_v4(s.A1h + core_offset(tid, kg * 8, 16), h[4 * kg], h[4 * kg + 1], h[4 * kg + 2], h[4 * kg + 3]);
            st_shared_v4(s.A1l + core_offset(tid, kg * 8, 16), l[4 * kg], l[4 * kg + 1], l[4 * kg + 2], l[4 * kg + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_mma(d1, smem_desc(s.A1h, 128, 256), smem_desc(s.B1, 128, 256), 0u);
            tc_mma(d1, smem_desc(s.A1l, 128, 256), smem_desc(s.B1, 128, 256), 1u);
            tc_commit(&s.mbar);
        }
        load_row(tile + gridDim.x, fin);
        bool ok = mbar_wait(&s.mbar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // layer 1 epilogue (the bias is in the accumulator): ReLU, split ->
        // layer-2 A operand (row tid)
#pragma unroll
        for (int c0 = 0; c0 < kMlpHid; c0 += 32) {
            uint32_t a[32];
            tmem_ld32(d1 + lane_base + c0, a);
            tmem_wait();
            uint32_t hh[16], ll[16];
#pragma unroll
            for (int i = 0; i < 16; ++i)
                split_bf16x2(fmaxf(__uint_as_float(a[2 * i]), 0.0f), fmaxf(__uint_as_float(a[2 * i + 1]), 0.0f), hh[i],
                             ll[i]);
#pragma unroll
            for (int kg = 0; kg < 4; ++kg) {
                st_shared_v4(s.A2h + core_offset(tid, c0 + kg * 8, 64), hh[4 * kg], hh[4 * kg + 1], hh[4 * kg + 2],
                             hh[4 * kg + 3]);
                st_shared_v4(s.A2l + core_offset(tid, c0 + kg * 8, 64), ll[4 * kg], ll[4 * kg + 1], ll[4 * kg + 2],
                             ll[4 * kg + 3]);
            }
        }
        // layer 1's inputs are consumed: A1h row tid becomes (1, 1, 1, 0, ...),
        // the A operand of layer 2's bias product
        st_shared_v4(s.A1h + core_offset(tid, 0, 16), 0x3F803F80u, 0x00003F80u, 0u, 0u);
        st_shared_v4(s.A1h + core_offset(tid, 8, 16), 0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {  // K-step ks: core matrices 2ks, 2ks + 1 along K
                const uint64_t b = smem_desc(s.B2 + ks * 256, 128, 1024);
                tc_mma(d2, smem_desc(s.A2h + ks * 256, 128, 1024), b, ks > 0 ? 1u : 0u);
                tc_mma(d2, smem_desc(s.A2l + ks * 256, 128, 1024), b, 1u);
            }
            tc_mma(d2, smem_desc(s.A1h, 128, 256), smem_desc(s.B2b, 128, 256), 1u);  // + b2
            tc_commit(&s.mbar);
        }
        ok = mbar_wait(&s.mbar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // layer 2 epilogue (the bias is in the accumulator): ReLU, the 64 -> 1
        // dot product
        uint32_t a[64];
        tmem_ld32(d2 + lane_base, a);
        tmem_ld32(d2 + lane_base + 32, a + 32);
        tmem_wait();
        float z = b3;
#pragma unroll
        for (int c = 0; c < kMlpHid; c += 4) {
            const float4 w = *reinterpret_cast<const float4 *>(s.W3 + c);
            z = fmaf(w.x, fmaxf(__uint_as_float(a[c]), 0.0f), z);
            z = fmaf(w.y, fmaxf(__uint_as_float(a[c + 1]), 0.0f), z);
            z = fmaf(w.z, fmaxf(__uint_as_float(a[c + 2]), 0.0f), z);
            z = fmaf(w.w, fmaxf(__uint_as_float(a[c + 3]), 0.0f), z);
        }
        if (row < n) logits[row] = z;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // TMEM read and shared operands consumed before the next tile reuses them
    }
    if (failed) {
        // a product did not complete in time: report it, give whatever is
        // still in flight a bounded while to land, then release TMEM
        if (tid == 0) atomicOr(status, 1u);
        mbar_wait(&s.mbar, parity);
        __syncthreads();
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcCols));
}

int ensure_state(kf_context *ctx, MlpState **out)
{
    MlpState *&s = context_mlp_state(ctx);
    if (!s) {
        s = new MlpState;
        bool ok = cudaMalloc(&s->grad, kMlpParams * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&s->m, kMlpParams * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&s->v, kMlpParams * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&s->loss, sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&s->w32, kMlpParams * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&s->W1, kW1Elems * sizeof(__nv_bfloat16)) == cudaSuccess &&
                  cudaMalloc(&s->W2, kW2Elems * sizeof(__nv_bfloat16)) == cudaSuccess &&
                  cudaMalloc(&s->status, sizeof(unsigned)) == cudaSuccess &&
                  cudaMemset(s->status, 0, sizeof(unsigned)) == cudaSuccess;
        if (!ok) {
            destroy_mlp_state(s);
            s = nullptr;
            return set_error(ctx, KF_ERR_NOMEM, "could not allocate the proposal's scratch");
        }
    }
    *out = s;
    return KF_OK;
}

int launch_grad(kf_context *ctx, MlpState *s, const float *w, const float *X, const float *y, int64_t n, int64_t start,
                int64_t count, int64_t P, int64_t off, float inv_batch, cudaStream_t stream)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
        attr = true;
    }
    const unsigned blocks = (unsigned)((count + kTile - 1) / kTile);
    mlp_grad_kernel<<<blocks, kTrainThreads, sizeof(TrainSmem), stream>>>(w, X, y, n, start, count, P, off, inv_batch,
                                                                          s->grad, s->loss);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : cuda_error(ctx, e, "proposal gradient launch");
}

int64_t gcd64(int64_t a, int64_t b) { return b ? gcd64(b, a % b) : a; }

}  // namespace
}  // namespace kf

using namespace kf;

extern "C" {

int kf_proposal_gradient(kf_context *ctx, const float *weights, const float *features, const float *labels, int64_t n,
                         float *grad, float *loss, kf_stream stream_)
{
    if (!ctx) return KF_ERR_ARG;
    if (n < 1) return set_error(ctx, KF_ERR_ARG, "n must be >= 1");
    int rc;
    if ((rc = check_ptr(ctx, weights, 4, "weights")) || (rc = check_ptr(ctx, features, 4, "features")) ||
        (rc = check_ptr(ctx, labels, 4, "labels")) || (rc = check_ptr(ctx, grad, 4, "grad")))
        return rc;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    MlpState *s;
    if ((rc = ensure_state(ctx, &s))) return rc;
    cudaMemsetAsync(s->grad, 0, kMlpParams * sizeof(float), stream);
    cudaMemsetAsync(s->loss, 0, sizeof(float), stream);
    if ((rc = launch_grad(ctx, s, weights, features, labels, n, 0, n, 1, 0, 1.0f / (float)n, stream))) return rc;
    cudaMemcpyAsync(grad, s->grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, stream);
    if (loss) {
        float l = 0.0f;
        cudaMemcpyAsync(&l, s->loss, sizeof(float), cudaMemcpyDeviceToHost, stream);
        const cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_error(ctx, e, "proposal gradient");
        *loss = l / (float)n;
    }
    return KF_OK;
}

int kf_proposal_train(kf_context *ctx, float *weights, const float *features, const float *labels, int64_t n, int epochs,
                      int batch, float learning_rate, float *epoch_loss, kf_stream stream_)
{
    if (!ctx) return KF_ERR_ARG;
    if (n < 1 || epochs < 0 || batch < 1 || !(learning_rate > 0.0f))
        return set_error(ctx, KF_ERR_ARG, "n >= 1, epochs >= 0, batch >= 1 and learning_rate > 0 required");
    int rc;
    if ((rc = check_ptr(ctx, weights, 4, "weights")) || (rc = check_ptr(ctx, features, 4, "features")) ||
        (rc = check_ptr(ctx, labels, 4, "labels")))
        return rc;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    MlpState *s;
    if ((rc = ensure_state(ctx, &s))) return rc;
    cudaMemsetAsync(s->grad, 0, kMlpParams * sizeof(float), stream);
    cudaMemsetAsync(s->m, 0, kMlpParams * sizeof(float), stream);
    cudaMemsetAsync(s->v, 0, kMlpParams * sizeof(float), stream);
    // epoch order: sample = (j P + off) mod n with P coprime to n
    int64_t P = 1000003;
    while (gcd64(P, n) != 1) P += 2;
    int t = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        cudaMemsetAsync(s->loss, 0, sizeof(float), stream);
        const int64_t off = (int64_t)ep * 7919 % n;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t cnt = std::min<int64_t>(batch, n - b0);
            if ((rc = launch_grad(ctx, s, weights, features, labels, n, b0, cnt, P, off, 1.0f / (float)cnt, stream)))
                return rc;
            adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(weights, s->grad, s->m, s->v, ++t, learning_rate,
                                                                     0.9f, 0.999f, 1e-8f);
        }
        if (epoch_loss) {
            float l = 0.0f;
            cudaMemcpyAsync(&l, s->loss, sizeof(float), cudaMemcpyDeviceToHost, stream);
            const cudaError_t e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return cuda_error(ctx, e, "proposal training");
            epoch_loss[ep] = l / (float)n;
        }
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : cuda_error(ctx, e, "proposal training");
}

int kf_proposal_load(kf_context *ctx, const float *weights, kf_stream stream_)
{
    if (!ctx) return KF_ERR_ARG;
    int rc;
    if ((rc = check_ptr(ctx, weights, 4, "weights"))) return rc;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    MlpState *s;
    if ((rc = ensure_state(ctx, &s))) return rc;
    cudaMemcpyAsync(s->w32, weights, kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, stream);
    to_bf16_kernel<<<8, 256, 0, stream>>>(s->w32, s->W1, s->W2);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "proposal load");
    s->loaded = true;
    return KF_OK;
}

int kf_load_proposal(kf_context *ctx, const void *weights, size_t bytes)
{
    if (!ctx) return KF_ERR_ARG;
    if (bytes != kMlpParams * sizeof(float))
        return set_error(ctx, KF_ERR_ARG, "weights must be %zu bytes (%d FP32 parameters), got %zu",
                         (size_t)kMlpParams * sizeof(float), kMlpParams, bytes);
    return kf_proposal_load(ctx, static_cast<const float *>(weights), nullptr);
}

int kf_proposal_score_with(kf_context *ctx, const float *features, int64_t n, float *logits, int engine,
                           kf_stream stream_)
{
    if (!ctx) return KF_ERR_ARG;
    if (!proposal_loaded(ctx)) return set_error(ctx, KF_ERR_ARG, "no proposal weights loaded (kf_proposal_load)");
    if (n < 0) return set_error(ctx, KF_ERR_ARG, "n must be >= 0");
    if (engine != KF_SCORE_AUTO && engine != KF_SCORE_MMA_SYNC && engine != KF_SCORE_TCGEN05)
        return set_error(ctx, KF_ERR_ARG, "engine must be KF_SCORE_AUTO, KF_SCORE_MMA_SYNC or KF_SCORE_TCGEN05");
    if (n == 0) return KF_OK;
    int rc;
    if ((rc = check_ptr(ctx, features, 4, "features")) || (rc = check_ptr(ctx, logits, 4, "logits"))) return rc;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    MlpState *s = context_mlp_state(ctx);
    DeviceGuard dg(context_device(ctx));
    if (engine == KF_SCORE_AUTO) engine = n >= kScoreTcMinRows ? KF_SCORE_TCGEN05 : KF_SCORE_MMA_SYNC;
    cudaError_t e;
    if (engine == KF_SCORE_TCGEN05) {
        if ((e = cudaFuncSetAttribute(mlp_score_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(TcSmem))) != cudaSuccess)
            return cuda_error(ctx, e, "tcgen05 scoring shared memory");
        const int64_t tiles = (n + kTcRows - 1) / kTcRows;
        const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)context_sm_count(ctx) * kTcCtasPerSm);
        mlp_score_tc_kernel<<<grid, kTcRows, sizeof(TcSmem), stream>>>(s->w32, features, n, logits, s->status);
    } else {
        if ((e = cudaFuncSetAttribute(mlp_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(ScoreSmem))) != cudaSuccess)
            return cuda_error(ctx, e, "scoring shared memory");
        const int64_t chunks = (n + 31) / 32;
        const unsigned grid = (unsigned)std::min<int64_t>((chunks + kScoreWarps - 1) / kScoreWarps,
                                                          (int64_t)context_sm_count(ctx) * 8);
        mlp_score_kernel<<<grid, 32 * kScoreWarps, sizeof(ScoreSmem), stream>>>(s->W1, s->W2, s->w32, features, n,
                                                                                logits);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : cuda_error(ctx, e, "proposal score launch");
}

int kf_proposal_score(kf_context *ctx, const float *features, int64_t n, float *logits, kf_stream stream)
{
    return kf_proposal_score_with(ctx, features, n, logits, KF_SCORE_AUTO, stream);
}

int kf_proposal_status(kf_context *ctx, int *expired)
{
    if (!ctx || !expired) return KF_ERR_ARG;
    *expired = 0;
    MlpState *s = context_mlp_state(ctx);
    if (!s) return KF_OK;
    DeviceGuard dg(context_device(ctx));
    unsigned v = 0;
    const cudaError_t e = cudaMemcpy(&v, s->status, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(ctx, e, "proposal status");
    *expired = v != 0;
    return KF_OK;
}

}  // extern "C"
