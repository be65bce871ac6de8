// Kalman-filter track fit on sm_103a: one thread per track (Section 4.2),
// state and packed covariance in registers, structure-of-arrays inputs read
// coalesced (Section 4.1: element (i, j) of consecutive tracks is contiguous).
#include "kf.h"
#include "kf_fit.cuh"

namespace kf {

namespace {

constexpr uint32_t kStop = KF_FLAG_UNREACHABLE | KF_FLAG_LEFT_BARREL | KF_FLAG_NAN_INPUT;

// 0 * v is 0 for finite v and NaN otherwise
template <int N>
__device__ __forceinline__ bool all_finite(const float *v)
{
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < N; ++i) acc = fmaf(0.0f, v[i], acc);
    return acc == 0.0f;
}

__device__ __forceinline__ void load_hit(const FitIO &io, int l, int64_t t, float m[3], float v[6])
{
    const int64_t T = io.T;
#pragma unroll
    for (int i = 0; i < 3; ++i) m[i] = __ldcs(io.hit_pos + ((int64_t)l * 3 + i) * T + t);
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = __ldcs(io.hit_cov + ((int64_t)l * 6 + i) * T + t);
}

// Fit track t over every layer in order (the steps and stop rules are those of
// kf_fit_tracks in kf.h).  The next present hit is loaded one layer ahead.
__device__ __forceinline__ void fit_track(const FitGeom &g, const Routing &rt, const FitIO &io, int64_t t)
{
    const int64_t T = io.T;
    float x[6], c[21];
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = __ldcs(io.seed_state + i * T + t);
#pragma unroll
    for (int i = 0; i < 21; ++i) c[i] = __ldcs(io.seed_cov + i * T + t);
    const float qkb = (float)io.charge[t] * g.qk;
    const uint32_t mask = __ldcs(io.hit_mask + t);
    uint32_t flags = (all_finite<6>(x) && all_finite<21>(c)) ? 0u : (uint32_t)KF_FLAG_NAN_INPUT;
    float chi2 = 0.0f;
    int nhits = 0;
    float m[3] = {0, 0, 0}, v[6] = {0, 0, 0, 0, 0, 0};
    if (mask & 1u) load_hit(io, 0, t, m, v);
    for (int l = 0; l < g.L && !(flags & kStop); ++l) {
        const bool has = (mask >> l) & 1u;
        const bool has_next = l + 1 < g.L && ((mask >> (l + 1)) & 1u);
        float mn[3], vn[6];
        if (has_next) load_hit(io, l + 1, t, mn, vn);
        float xn[6], s;
        Jac J;
        if (!propagate(x, qkb, g.r[l], xn, s, &J)) {
            flags |= KF_FLAG_UNREACHABLE;
            break;
        }
        if (fabsf(xn[2]) > g.z_half) {
            flags |= KF_FLAG_LEFT_BARREL;
            break;
        }
        transport(J, c);
        add_scattering(xn, g.r[l], g.xx0[l], c);
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = xn[i];
        if (has) {
            if (!all_finite<3>(m) || !all_finite<6>(v)) {
                flags |= KF_FLAG_NAN_INPUT;
                break;
            }
            float d = 0.0f;
            const int st = update(x, c, m, v, rt, &d);
            if (st == 1) {
                flags |= KF_FLAG_INVERSION_FAILED;
            } else {
                chi2 += d;
                ++nhits;
                if (st >= 2) flags |= KF_FLAG_FP64_PATH;
                if (st == 3) flags |= KF_FLAG_PSD_REPAIRED;
            }
        }
        if (has_next) {
#pragma unroll
            for (int i = 0; i < 3; ++i) m[i] = mn[i];
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = vn[i];
        }
    }
    if (flags & KF_FLAG_NAN_INPUT) {  // a track with bad input returns its seed
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = io.seed_state[i * T + t];
#pragma unroll
        for (int i = 0; i < 21; ++i) c[i] = io.seed_cov[i * T + t];
        chi2 = 0.0f;
        nhits = 0;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) __stcs(io.out_state + i * T + t, x[i]);
#pragma unroll
    for (int i = 0; i < 21; ++i) __stcs(io.out_cov + i * T + t, c[i]);
    __stcs(io.out_chi2 + t, chi2);
    io.out_ndof[t] = (int16_t)(3 * nhits - 6);
    io.out_flags[t] = flags;
}

// One thread per track over [t_begin, t_end).
__global__ void __launch_bounds__(256) fit_plain_kernel(const FitGeom g, const Routing rt, const FitIO io,
                                                         int64_t t_begin, int64_t t_end)
{
    const int64_t t = t_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < t_end) fit_track(g, rt, io, t);
}

// Persistent kernel: each warp claims 32-track units from *counter until the
// batch is exhausted (Section 4.2: fill the GPU with the tracks of many events
// in one launch).  Warps schedule themselves, so a warp slowed by an FP64
// update does not hold the rest of its block.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) fit_persistent_kernel(const FitGeom g, const Routing rt, const FitIO io,
                                                                unsigned *counter)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned n_units = (unsigned)((io.T + 31) / 32);
    for (;;) {
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(counter, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        const int64_t t = (int64_t)u * 32 + lane;
        if (t < io.T) fit_track(g, rt, io, t);
    }
}

}  // namespace

cudaError_t launch_fit_plain(const FitGeom &g, const Routing &rt, const FitIO &io, int64_t t_begin,
                             int64_t t_end, int block, cudaStream_t stream)
{
    if (t_end <= t_begin) return cudaSuccess;
    const int64_t n = t_end - t_begin;
    const unsigned grid = (unsigned)((n + block - 1) / block);
    fit_plain_kernel<<<grid, block, 0, stream>>>(g, rt, io, t_begin, t_end);
    return cudaGetLastError();
}

int persistent_blocks_per_sm(int block)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (block) {
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fit_persistent_kernel<32>, 32, 0); break;
    case 64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fit_persistent_kernel<64>, 64, 0); break;
    case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fit_persistent_kernel<128>, 128, 0); break;
    case 256: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fit_persistent_kernel<256>, 256, 0); break;
    default: break;
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_fit_persistent(const FitGeom &g, const Routing &rt, const FitIO &io, int block, int grid,
                                  unsigned *counter, cudaStream_t stream)
{
    switch (block) {
    case 32: fit_persistent_kernel<32><<<grid, 32, 0, stream>>>(g, rt, io, counter); break;
    case 64: fit_persistent_kernel<64><<<grid, 64, 0, stream>>>(g, rt, io, counter); break;
    case 128: fit_persistent_kernel<128><<<grid, 128, 0, stream>>>(g, rt, io, counter); break;
    case 256: fit_persistent_kernel<256><<<grid, 256, 0, stream>>>(g, rt, io, counter); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace kf
