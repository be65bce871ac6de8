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
__global__ void __launch_bounds__(kBinThreadsHP) bin_chunk_kernel(const int64_t *seg_off, const float *hit_pos,
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
#pragma unroll
        for (int k = 0; k < kBinPerThread; ++k) {
            const int64_t h = h0 + k * kBinThreadsHP;
            if (h < hi) {
                const float phi = atan2f(y[k], x[k]);
                int32_t *slot = &cnt[z_bin(z[k], bg) * bg.n_phi + phi_bin(phi, bg.n_phi)];
                if constexpr (SCATTER) {
                    const int p = atomicAdd(slot, 1);
                    bkey[lo + p] =
                        make_float4(phi, z[k], __int_as_float((int)(h - lo)), sqrtf(x[k] * x[k] + y[k] * y[k]));
                } else {
                    atomicAdd(slot, 1);
                }
            }
        }
    }
}

// One block per segment: exclusive scan of its bins' counts (each thread owns
// a contiguous run of bins) into bin_off (the segment's [nb + 1] offsets) and
// into counts, which become the scatter's cursors.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) bin_scan_kernel(const int64_t *seg_off, int nb, int32_t *counts,
                                                           int32_t *bin_off)
{
    __shared__ int warp_sums[THREADS / 32];
    const int64_t seg = blockIdx.x;
    int32_t *cnt = counts + seg * nb;
    const int per = (nb + THREADS - 1) / THREADS;
    const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
    int run = 0;
    for (int b = b0; b < b1; ++b) run += cnt[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) warp_sums[warp] = incl;
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
    int base = incl - run + (warp > 0 ? warp_sums[warp - 1] : 0);
    int32_t *bo = bin_off + seg * (nb + 1);
    for (int b = b0; b < b1; ++b) {
        const int c = cnt[b];
        cnt[b] = base;
        bo[b] = base;
        base += c;
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
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)n_seg * nb * sizeof(int32_t), stream);
    if (e != cudaSuccess) return e;
    const int64_t chunks = max_seg > 0 ? (max_seg + kBinChunk - 1) / kBinChunk : 1;
    const int64_t n_virtual = chunks * n_seg;
    const unsigned grid = (unsigned)(n_virtual < (int64_t)sm_count * 64 ? n_virtual : (int64_t)sm_count * 64);
    bin_chunk_kernel<false><<<grid, kBinThreadsHP, 0, stream>>>(seg_off, hit_pos, H, bg, chunks, n_virtual, counts,
                                                              bkey);
    bin_scan_kernel<1024><<<(unsigned)n_seg, 1024, 0, stream>>>(seg_off, nb, counts, bin_off);
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
