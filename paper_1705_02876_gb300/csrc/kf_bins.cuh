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

// Binning is two kernels.  bin_count_kernel gives each (event, layer)
// segment one block, which counts the segment's hits into a histogram of its
// bins in shared memory (shared-memory atomics; the count a hit finds before
// its own is its rank within the bin, in no fixed order, kept in rank[h]),
// then scans the histogram into the segment's bin offsets.
// bin_scatter_kernel places every hit's key at its bin's offset plus its
// rank: no atomics, each block a chunk of kBinChunk hits of one segment
// (virtual blocks seg * chunks + c, grid-strided) with its loads issued
// together; blocks run roughly in segment order, so the segments being
// scattered at any time are few and their keys (16 B per hit, scattered at
// random within the segment) merge into full sectors in L2.
constexpr int kBinCountThreads = 512;                    // threads of a counting block
constexpr int kBinCountUnroll = 4;                       // hits per thread loaded together when counting
constexpr int kBinThreadsHP = 256;                       // threads of the scatter blocks
constexpr int kBinPerThread = 8;                         // hits per thread
constexpr int kBinChunk = kBinThreadsHP * kBinPerThread;  // hits per virtual block
constexpr int kMaxBins = 16384;                          // bins per segment (64 KB of shared counters)

// The bin of a hit at azimuth phi = atan2f(y, x) and z (the count and the
// scatter both call this, so that they agree on every hit).
__device__ __forceinline__ int hit_bin(float phi, float z, const BinGrid &bg)
{
    return z_bin(z, bg) * bg.n_phi + phi_bin(phi, bg.n_phi);
}

__global__ void __launch_bounds__(kBinCountThreads) bin_count_kernel(const int64_t *seg_off, const float *hit_pos,
                                                                     int64_t H, BinGrid bg, int32_t *rank,
                                                                     int32_t *bin_off)
{
    extern __shared__ int32_t hist[];  // [nb]
    constexpr int W = kBinCountThreads / 32;
    __shared__ int warp_tot[W];
    const int nb = bg.n_phi * bg.n_z;
    const int64_t seg = blockIdx.x;
    const int64_t lo = seg_off[seg], hi = seg_off[seg + 1];
    for (int i = threadIdx.x; i < nb; i += kBinCountThreads) hist[i] = 0;
    __syncthreads();
    for (int64_t h0 = lo + threadIdx.x; h0 < hi; h0 += kBinCountUnroll * kBinCountThreads) {
        float x[kBinCountUnroll], y[kBinCountUnroll], z[kBinCountUnroll];
#pragma unroll
        for (int k = 0; k < kBinCountUnroll; ++k) {
            const int64_t h = h0 + k * kBinCountThreads;
            if (h < hi) {
                x[k] = hit_pos[h];
                y[k] = hit_pos[H + h];
                z[k] = hit_pos[2 * H + h];
            }
        }
#pragma unroll
        for (int k = 0; k < kBinCountUnroll; ++k) {
            const int64_t h = h0 + k * kBinCountThreads;
            if (h < hi) rank[h] = atomicAdd(&hist[hit_bin(atan2f(y[k], x[k]), z[k], bg)], 1);
        }
    }
    __syncthreads();
    // exclusive scan: warp w owns `run` consecutive bins from w * run, read
    // 32 consecutive bins at a time (one bank each)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int run = (nb + W * 32 - 1) / (W * 32) * 32;
    const int b0 = warp * run;
    int tot = 0;
    for (int i = lane; i < run; i += 32) tot += b0 + i < nb ? hist[b0 + i] : 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, d);
    if (lane == 0) warp_tot[warp] = tot;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += warp_tot[w];
    int32_t *bo = bin_off + seg * (nb + 1);
    for (int i = 0; i < run; i += 32) {
        const int b = b0 + i + lane;
        const int v = b < nb ? hist[b] : 0;
        int incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        if (b < nb) bo[b] = base + incl - v;
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (threadIdx.x == 0) bo[nb] = (int)(hi - lo);
}

__global__ void __launch_bounds__(kBinThreadsHP, 3) bin_scatter_kernel(const int64_t *seg_off, const float *hit_pos,
                                                                     int64_t H, BinGrid bg, int64_t chunks,
                                                                     int64_t n_virtual, const int32_t *rank,
                                                                     const int32_t *bin_off, float4 *bkey)
{
    const int nb = bg.n_phi * bg.n_z;
    for (int64_t vb = blockIdx.x; vb < n_virtual; vb += gridDim.x) {
        const int64_t seg = vb / chunks, c = vb - seg * chunks;
        const int64_t lo = seg_off[seg], hi = seg_off[seg + 1];
        const int64_t h0 = lo + c * kBinChunk + threadIdx.x;
        if (lo + c * kBinChunk >= hi) continue;  // block-uniform
        const int32_t *bo = bin_off + seg * (nb + 1);
        float x[kBinPerThread], y[kBinPerThread], z[kBinPerThread];
        int rk[kBinPerThread];
#pragma unroll
        for (int k = 0; k < kBinPerThread; ++k) {
            const int64_t h = h0 + k * kBinThreadsHP;
            if (h < hi) {
                x[k] = hit_pos[h];
                y[k] = hit_pos[H + h];
                z[k] = hit_pos[2 * H + h];
                rk[k] = rank[h];
            }
        }
        // every bin-offset load is issued before the first key store
        int p[kBinPerThread];
#pragma unroll
        for (int k = 0; k < kBinPerThread; ++k) {
            if (h0 + k * kBinThreadsHP < hi) {
                const float phi = atan2f(y[k], x[k]), r = sqrtf(x[k] * x[k] + y[k] * y[k]);
                p[k] = bo[hit_bin(phi, z[k], bg)] + rk[k];
                x[k] = phi;
                y[k] = r;
            }
        }
#pragma unroll
        for (int k = 0; k < kBinPerThread; ++k) {
            const int64_t h = h0 + k * kBinThreadsHP;
            if (h < hi && p[k] < (int)(hi - lo))  // always true: both kernels bin a hit alike
                bkey[lo + p[k]] = make_float4(x[k], z[k], __int_as_float((int)(h - lo)), y[k]);
        }
    }
}

// Bin the hits of n_seg segments (seg_off on the device, [n_seg + 1], within
// hit_pos [3][H]; max_seg the largest segment's hit count) into bkey and
// bin_off [n_seg][nb + 1]; rank is scratch of H int32.
inline cudaError_t bin_hits(const int64_t *seg_off, int64_t n_seg, int64_t max_seg, const float *hit_pos, int64_t H,
                            const BinGrid &bg, float4 *bkey, int32_t *bin_off, int32_t *rank, int sm_count,
                            cudaStream_t stream)
{
    if (n_seg <= 0) return cudaSuccess;
    const int nb = bg.n_phi * bg.n_z;
    if (nb < 1 || nb > kMaxBins) return cudaErrorInvalidValue;
    const int smem = nb * (int)sizeof(int32_t);
    // the dynamic shared memory opt-in is a per-device attribute: set on every call
    cudaError_t e = cudaFuncSetAttribute(bin_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    bin_count_kernel<<<(unsigned)n_seg, kBinCountThreads, smem, stream>>>(seg_off, hit_pos, H, bg, rank, bin_off);
    const int64_t chunks = max_seg > 0 ? (max_seg + kBinChunk - 1) / kBinChunk : 1;
    const int64_t n_virtual = chunks * n_seg;
    const unsigned grid = (unsigned)(n_virtual < (int64_t)sm_count * 64 ? n_virtual : (int64_t)sm_count * 64);
    bin_scatter_kernel<<<grid, kBinThreadsHP, 0, stream>>>(seg_off, hit_pos, H, bg, chunks, n_virtual, rank, bin_off,
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
