// Hits binned in (phi, z) per (event, layer) segment, shared by the build and
// the seeding (Section 3: hits partitioned spatially so that the compatible
// ones are found without scanning the layer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kf {
namespace {

constexpr float kPi = 3.14159265358979f;

struct BinGrid {
    int n_phi, n_z;
    float z_half;
};

__device__ __forceinline__ int phi_bin(float phi, int n_phi)
{
    const int b = (int)floorf((phi + kPi) * (float)n_phi * (1.0f / (2.0f * kPi)));
    return min(max(b, 0), n_phi - 1);
}
__device__ __forceinline__ int z_bin(float z, const BinGrid &bg)
{
    const int b = (int)floorf((z + bg.z_half) * (float)bg.n_z / (2.0f * bg.z_half));
    return min(max(b, 0), bg.n_z - 1);
}

// Binning is three kernels over all segments at once.  bin_count_kernel and
// bin_scatter_kernel give each block a chunk of kBinChunk hits of one segment
// (virtual blocks seg * chunks + c, grid-strided), with their loads issued
// together; blocks run roughly in segment order, so the segments being
// scattered at any time are few and their keys (16 B per hit, scattered at
// random within the segment) merge into full sectors in L2.  Counting adds
// to a global counter per (segment, bin); bin_scan_kernel turns each
// segment's counts into the bin offsets and into the scatter's cursors.
constexpr int kBinThreadsHP = 256;                       // threads of the count and scatter blocks
constexpr int kBinPerThread = 8;                         // hits per thread
constexpr int kBinChunk = kBinThreadsHP * kBinPerThread;  // hits per virtual block

template <bool SCATTER>
__global__ void __launch_bounds__(kBinThreadsHP, 4) bin_chunk_kernel(const int64_t *seg_off, const float *hit_pos,
                                                                   int64_t H, BinGrid bg, int64_t chunks,
                                                                   int64_t n_virtual, int32_t *counts,
                                                                   float4 *bkey)
{
    const int nb = bg.n_phi * bg.n_z;
    for (int64_t vb = blockIdx.x; vb < n_virtual; vb += gridDim.x) {
        const int64_t seg = vb / chunks, c = vb - seg * chunks;
        const int64_t lo = seg_off[seg], hi = seg_off[seg + 1];
        const int64_t h0 = lo + c * kBinChunk + threadIdx.x;
        if (lo + c * kBinChunk >= hi) continue;  // block-uniform
        int32_t *cnt = counts + seg * nb;
        float x[kBinPerThread], y[kBinPerThread], z[kBinPerThread];
#pragma unroll
        for (int k = 0; k < kBinPerThread; ++k) {
            const int64_t h = h0 + k * kBinThreadsHP;
            if (h < hi) {
                x[k] = hit_pos[h];
                y[k] = hit_pos[H + h];
                z[k] = hit_pos[2 * H + h];
            }
        }
        if constexpr (SCATTER) {
            // all of the thread's cursor claims are issued before the first
            // key store, so that their round trips to L2 overlap
            // (x and y are replaced by phi and the radius as they are used)
            int p[kBinPerThread];
#pragma unroll
            for (int k = 0; k < kBinPerThread; ++k) {
                if (h0 + k * kBinThreadsHP < hi) {
                    const float phi = atan2f(y[k], x[k]), r = sqrtf(x[k] * x[k] + y[k] * y[k]);
                    x[k] = phi;
                    y[k] = r;
                    p[k] = atomicAdd(&cnt[z_bin(z[k], bg) * bg.n_phi + phi_bin(phi, bg.n_phi)], 1);
                }
            }
#pragma unroll
            for (int k = 0; k < kBinPerThread; ++k) {
                const int64_t h = h0 + k * kBinThreadsHP;
                if (h < hi) bkey[lo + p[k]] = make_float4(x[k], z[k], __int_as_float((int)(h - lo)), y[k]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < kBinPerThread; ++k) {
                if (h0 + k * kBinThreadsHP < hi) {
                    const float phi = atan2f(y[k], x[k]);
                    atomicAdd(&cnt[z_bin(z[k], bg) * bg.n_phi + phi_bin(phi, bg.n_phi)], 1);
                }
            }
        }
    }
}

// One block per segment: exclusive scan of its bins' counts into bin_off (the
// segment's [nb + 1] offsets) and into counts, which become the scatter's
// cursors.  Warp w owns bins [w * 32 kScanRun, (w + 1) * 32 kScanRun) and
// walks them in kScanRun rounds of 32 consecutive bins, so that every load
// and store of a warp is one contiguous run; a round is scanned with shuffles
// and its total carried into the next.
constexpr int kScanThreads = 1024, kScanRun = 16;
constexpr int kMaxBins = kScanThreads * kScanRun;  // 16,384 bins per segment
template <int THREADS>
__global__ void __launch_bounds__(THREADS) bin_scan_kernel(const int64_t *seg_off, int nb, int32_t *counts,
                                                           int32_t *bin_off)
{
    __shared__ int warp_sums[THREADS / 32];
    const int64_t seg = blockIdx.x;
    int32_t *cnt = counts + seg * nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wb = warp * 32 * kScanRun + lane;  // this lane's bin in round 0
    int v[kScanRun];
#pragma unroll
    for (int i = 0; i < kScanRun; ++i) v[i] = wb + 32 * i < nb ? cnt[wb + 32 * i] : 0;
    int carry = 0;  // the warp's bins before this round
#pragma unroll
    for (int i = 0; i < kScanRun; ++i) {
        int incl = v[i];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        v[i] = carry + incl - v[i];
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) warp_sums[warp] = carry;
    __syncthreads();
    if (warp == 0) {
        int w = lane < THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += o;
        }
        if (lane < THREADS / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    const int base = warp > 0 ? warp_sums[warp - 1] : 0;
    int32_t *bo = bin_off + seg * (nb + 1);
#pragma unroll
    for (int i = 0; i < kScanRun; ++i)
        if (wb + 32 * i < nb) {
            cnt[wb + 32 * i] = base + v[i];
            bo[wb + 32 * i] = base + v[i];
        }
    if (threadIdx.x == 0) bo[nb] = (int)(seg_off[seg + 1] - seg_off[seg]);
}

// Bin the hits of n_seg segments (seg_off on the device, [n_seg + 1], within
// hit_pos [3][H]; max_seg the largest segment's hit count) into bkey and
// bin_off; counts is scratch of n_seg * nb int32.
inline cudaError_t bin_hits(const int64_t *seg_off, int64_t n_seg, int64_t max_seg, const float *hit_pos, int64_t H,
                            const BinGrid &bg, float4 *bkey, int32_t *bin_off, int32_t *counts, int sm_count,
                            cudaStream_t stream)
{
    if (n_seg <= 0) return cudaSuccess;
    const int nb = bg.n_phi * bg.n_z;
    if (nb < 1 || nb > kMaxBins) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)n_seg * nb * sizeof(int32_t), stream);
    if (e != cudaSuccess) return e;
    const int64_t chunks = max_seg > 0 ? (max_seg + kBinChunk - 1) / kBinChunk : 1;
    const int64_t n_virtual = chunks * n_seg;
    const unsigned grid = (unsigned)(n_virtual < (int64_t)sm_count * 64 ? n_virtual : (int64_t)sm_count * 64);
    bin_chunk_kernel<false><<<grid, kBinThreadsHP, 0, stream>>>(seg_off, hit_pos, H, bg, chunks, n_virtual, counts,
                                                              bkey);
    bin_scan_kernel<kScanThreads><<<(unsigned)n_seg, kScanThreads, 0, stream>>>(seg_off, nb, counts, bin_off);
    bin_chunk_kernel<true><<<grid, kBinThreadsHP, 0, stream>>>(seg_off, hit_pos, H, bg, chunks, n_virtual, counts,
                                                             bkey);
    return cudaGetLastError();
}

__device__ __forceinline__ float wrap_pi(float d)
{
    d = d > kPi ? d - 2.0f * kPi : d;
    return d <= -kPi ? d + 2.0f * kPi : d;
}

}  // namespace
}  // namespace kf
