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

// Fit track t over every layer in order (the steps and stop rules are those of
// kf_fit_tracks in kf.h).  The next present hit is loaded one layer ahead,
// through pointers advanced by one layer's stride.  A non-finite value in a
// used hit makes the chi2 increment non-finite, or makes S fail its positive
// definiteness test, so the hit is tested only then.
__device__ __forceinline__ void fit_track(const FitGeom &g, const Routing &rt, const FitIO &io, int64_t t,
                                          float *slot, int stride)
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
    const float *hp = io.hit_pos + t;  // layer l, component i: hp[(3 l + i) T]
    const float *hc = io.hit_cov + t;
    const int64_t T3 = 3 * T, T6 = 6 * T;
    float m[3] = {0, 0, 0}, v[6] = {0, 0, 0, 0, 0, 0};
    auto load_hit = [&](float mm[3], float vv[6]) {
#pragma unroll
        for (int i = 0; i < 3; ++i) mm[i] = __ldcs(hp + i * T);
#pragma unroll
        for (int i = 0; i < 6; ++i) vv[i] = __ldcs(hc + i * T);
    };
    if (mask & 1u) load_hit(m, v);
    for (int l = 0; l < g.L && !(flags & kStop); ++l) {
        const bool has = (mask >> l) & 1u;
        const bool has_next = l + 1 < g.L && ((mask >> (l + 1)) & 1u);
        hp += T3;
        hc += T6;
        float mn[3], vn[6];
        if (has_next) load_hit(mn, vn);
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
        add_scattering(xn, g.inv_r[l], g.xx0[l], c);
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = xn[i];
        if (has) {
            float d = 0.0f;
            const int st = update(x, c, m, v, rt, &d, slot, stride);
            if (st == 1 || !isfinite(d)) {
                if (!all_finite<3>(m) || !all_finite<6>(v)) {
                    flags |= KF_FLAG_NAN_INPUT;
                    break;
                }
            }
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
    extern __shared__ float slots[];
    const int64_t t = t_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < t_end) fit_track(g, rt, io, t, slots + threadIdx.x, blockDim.x);
}

// Persistent kernel: each warp claims 32-track units from *counter until the
// batch is exhausted (Section 4.2: fill the GPU with the tracks of many events
// in one launch).  Warps schedule themselves, so a warp slowed by an
// extended-precision update does not hold the rest of its block.  MINB > 1
// caps the registers per thread at 65536 / (BLOCK * MINB) to raise occupancy.
template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) fit_persistent_kernel(const FitGeom g, const Routing rt,
                                                                      const FitIO io, unsigned *counter)
{
    __shared__ float slots[kSlotSize * BLOCK];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned n_units = (unsigned)((io.T + 31) / 32);
    for (;;) {
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(counter, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        const int64_t t = (int64_t)u * 32 + lane;
        if (t < io.T) fit_track(g, rt, io, t, slots + threadIdx.x, BLOCK);
    }
}

using PersistentFn = void (*)(FitGeom, Routing, FitIO, unsigned *);

// (block, register cap) shapes the autotuner chooses from; cap 0 = none.
// A cap of R registers is __launch_bounds__(BLOCK, 65536 / (R * BLOCK)).
struct Shape {
    int block, cap;
    PersistentFn fn;
};
const Shape kShapes[] = {
    {32, 0, fit_persistent_kernel<32, 1>},     {64, 0, fit_persistent_kernel<64, 1>},
    {128, 0, fit_persistent_kernel<128, 1>},   {256, 0, fit_persistent_kernel<256, 1>},
    {32, 168, fit_persistent_kernel<32, 12>},  {64, 168, fit_persistent_kernel<64, 6>},
    {128, 168, fit_persistent_kernel<128, 3>}, {32, 128, fit_persistent_kernel<32, 16>},
    {64, 128, fit_persistent_kernel<64, 8>},   {128, 128, fit_persistent_kernel<128, 4>},
    {256, 128, fit_persistent_kernel<256, 2>}, {32, 96, fit_persistent_kernel<32, 20>},
    {64, 96, fit_persistent_kernel<64, 10>},   {128, 96, fit_persistent_kernel<128, 5>},
    {32, 80, fit_persistent_kernel<32, 24>},   {64, 80, fit_persistent_kernel<64, 12>},
    {128, 80, fit_persistent_kernel<128, 6>},  {256, 80, fit_persistent_kernel<256, 3>},
};

const Shape *find_shape(int block, int cap)
{
    for (const Shape &sh : kShapes)
        if (sh.block == block && sh.cap == cap) return &sh;
    return nullptr;
}

}  // namespace

cudaError_t launch_fit_plain(const FitGeom &g, const Routing &rt, const FitIO &io, int64_t t_begin,
                             int64_t t_end, int block, cudaStream_t stream)
{
    if (t_end <= t_begin) return cudaSuccess;
    const int64_t n = t_end - t_begin;
    const unsigned grid = (unsigned)((n + block - 1) / block);
    fit_plain_kernel<<<grid, block, kSlotSize * block * sizeof(float), stream>>>(g, rt, io, t_begin, t_end);
    return cudaGetLastError();
}

int persistent_blocks_per_sm(int block, int cap)
{
    const Shape *sh = find_shape(block, cap);
    int n = 0;
    if (!sh || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sh->fn, block, 0) != cudaSuccess) return 0;
    return n;
}

int persistent_shapes(int *blocks, int *caps, int max_n)
{
    int n = 0;
    for (const Shape &sh : kShapes)
        if (n < max_n) {
            blocks[n] = sh.block;
            caps[n] = sh.cap;
            ++n;
        }
    return n;
}

cudaError_t launch_fit_persistent(const FitGeom &g, const Routing &rt, const FitIO &io, int block, int cap, int grid,
                                  unsigned *counter, cudaStream_t stream)
{
    const Shape *sh = find_shape(block, cap);
    if (!sh) return cudaErrorInvalidValue;
    sh->fn<<<grid, block, 0, stream>>>(g, rt, io, counter);
    return cudaGetLastError();
}

}  // namespace kf
