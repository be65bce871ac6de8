// Hits binned in (phi, z) per (event, layer) segment, shared by the build and
// the seeding (Section 3: hits partitioned spatially so that the compatible
// ones are found without scanning the layer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kf {
namespace {

constexpr float kPi = 3.14159265358979f;
constexpr int kUnroll = 4;        // hits per thread per step of the binning passes
// One segment per SM at a time: its keys (16 B per hit, about 880 KB for a
// 55,000-hit layer) are scattered at random within the segment and merge into
// full sectors in L2; two segments per SM (512 threads each) overflowed L2
// and were slower.
constexpr int kBinThreads = 1024;

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

// One block per (event, layer) segment: count hits per bin in shared memory,
// scan, scatter each hit's key (phi, z, index within the segment, transverse
// radius) bin by bin (bin = iz * n_phi + iphi).  A key is one 16-byte store here and one 16-byte
// load in the window scan: the destinations are random at a few hits per bin,
// so each key costs one memory sector, not three.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) bin_hits_kernel(const int64_t *seg_off, const float *hit_pos, int64_t H,
                                                           BinGrid bg, float4 *bkey, int32_t *bin_off)
{
    extern __shared__ int cnt[];
    __shared__ int warp_sums[THREADS / 32];
    const int seg = blockIdx.x;
    const int64_t lo = seg_off[seg], hi = seg_off[seg + 1];
    const int nb = bg.n_phi * bg.n_z;
    for (int i = threadIdx.x; i < nb; i += THREADS) cnt[i] = 0;
    __syncthreads();
    // kUnroll hits per thread and step, their loads issued together: the
    // passes over the segment are bound by load latency, not bandwidth
    for (int64_t h0 = lo + threadIdx.x; h0 < hi; h0 += kUnroll * THREADS) {
        float x[kUnroll], y[kUnroll], z[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int64_t h = h0 + k * THREADS;
            if (h < hi) {
                x[k] = hit_pos[h];
                y[k] = hit_pos[H + h];
                z[k] = hit_pos[2 * H + h];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
            if (h0 + k * THREADS < hi)
                atomicAdd(&cnt[z_bin(z[k], bg) * bg.n_phi + phi_bin(atan2f(y[k], x[k]), bg.n_phi)], 1);
    }
    __syncthreads();
    // exclusive scan: each thread owns a contiguous run of bins
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
    int32_t *bo = bin_off + (int64_t)seg * (nb + 1);
    for (int b = b0; b < b1; ++b) {
        const int c = cnt[b];
        cnt[b] = base;
        bo[b] = base;
        base += c;
    }
    if (threadIdx.x == 0) bo[nb] = (int)(hi - lo);
    __syncthreads();
    for (int64_t h0 = lo + threadIdx.x; h0 < hi; h0 += kUnroll * THREADS) {
        float x[kUnroll], y[kUnroll], z[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int64_t h = h0 + k * THREADS;
            if (h < hi) {
                x[k] = hit_pos[h];
                y[k] = hit_pos[H + h];
                z[k] = hit_pos[2 * H + h];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int64_t h = h0 + k * THREADS;
            if (h < hi) {
                const float phi = atan2f(y[k], x[k]);
                const int p = atomicAdd(&cnt[z_bin(z[k], bg) * bg.n_phi + phi_bin(phi, bg.n_phi)], 1);
                bkey[lo + p] =
                    make_float4(phi, z[k], __int_as_float((int)(h - lo)), sqrtf(x[k] * x[k] + y[k] * y[k]));
            }
        }
    }
}

__device__ __forceinline__ float wrap_pi(float d)
{
    d = d > kPi ? d - 2.0f * kPi : d;
    return d <= -kPi ? d + 2.0f * kPi : d;
}

}  // namespace
}  // namespace kf
