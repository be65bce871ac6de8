// Kalman-filter track fit on sm_103a: one thread per track (Section 4.2),
// state and packed covariance in registers, structure-of-arrays inputs read
// coalesced (Section 4.1: element (i, j) of consecutive tracks is contiguous).
#include <mutex>
#include <set>
#include <utility>

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

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Fit track t over every layer in order (the steps and stop rules are those of
// kf_fit_tracks in kf.h).  Hits are loaded DEPTH layers ahead of their update:
// DEPTH = 1 into registers, through pointers advanced by one layer's stride;
// DEPTH >= 2 by asynchronous copies (cp.async, one commit group per layer,
// empty for a layer without a hit) into this thread's column of a ring of
// DEPTH + 1 shared-memory stages of 9 floats each ([stage * 9 + i][stride]),
// so that the loads in flight hold no registers.  A non-finite value in a
// used hit makes the chi2 increment non-finite, or makes S fail its positive
// definiteness test, so the hit is tested only then.
template <int DEPTH>
__device__ __forceinline__ void fit_track(const FitGeom &g, const Routing &rt, const FitIO &io, int64_t t,
                                          float *slot, int stride, float *ring = nullptr)
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
    // DEPTH >= 2: layer l's hit goes to stage l % (DEPTH + 1); stage_in is the
    // stage of the next layer to issue, stage_out that of the next to use
    int stage_in = 0, stage_out = 0, l_in = 0;
    auto issue = [&]() {
        if (l_in < g.L && ((mask >> l_in) & 1u)) {
            const float *p = io.hit_pos + (int64_t)(3 * l_in) * T + t;
            const float *q = io.hit_cov + (int64_t)(6 * l_in) * T + t;
            float *st = ring + stage_in * 9 * stride;
#pragma unroll
            for (int i = 0; i < 3; ++i) cp_async4(st + i * stride, p + i * T);
#pragma unroll
            for (int i = 0; i < 6; ++i) cp_async4(st + (3 + i) * stride, q + i * T);
        }
        cp_async_commit();
        ++l_in;
        stage_in = stage_in == DEPTH ? 0 : stage_in + 1;
    };
    if constexpr (DEPTH == 1) {
        if (mask & 1u) load_hit(m, v);
    } else {
#pragma unroll
        for (int k = 0; k < DEPTH; ++k) issue();
    }
    for (int l = 0; l < g.L && !(flags & kStop); ++l) {
        const bool has = (mask >> l) & 1u;
        const bool has_next = l + 1 < g.L && ((mask >> (l + 1)) & 1u);
        float mn[3], vn[6];
        if constexpr (DEPTH == 1) {
            hp += T3;
            hc += T6;
            if (has_next) load_hit(mn, vn);
        } else {
            issue();                      // layer l + DEPTH
            cp_async_wait<DEPTH>();       // layer l's group has landed
            if (has) {
                const float *st = ring + stage_out * 9 * stride;
#pragma unroll
                for (int i = 0; i < 3; ++i) m[i] = st[i * stride];
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = st[(3 + i) * stride];
            }
            stage_out = stage_out == DEPTH ? 0 : stage_out + 1;
        }
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
        if constexpr (DEPTH == 1) {
            if (has_next) {
#pragma unroll
                for (int i = 0; i < 3; ++i) m[i] = mn[i];
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = vn[i];
            }
        }
    }
    if constexpr (DEPTH > 1) cp_async_wait<0>();  // no copy of this track may land in the next one's ring
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
    if (t < t_end) fit_track<1>(g, rt, io, t, slots + threadIdx.x, blockDim.x);
}

// Persistent kernel: each warp claims 32-track units from *counter until the
// batch is exhausted (Section 4.2: fill the GPU with the tracks of many events
// in one launch).  Warps schedule themselves, so a warp slowed by an
// extended-precision update does not hold the rest of its block.  MINB > 1
// caps the registers per thread at 65536 / (BLOCK * MINB) to raise occupancy.
// DEPTH >= 2 keeps the hit ring in dynamic shared memory (ring_floats(...)).
template <int BLOCK, int MINB, int DEPTH>
__global__ void __launch_bounds__(BLOCK, MINB) fit_persistent_kernel(const FitGeom g, const Routing rt,
                                                                      const FitIO io, unsigned *counter)
{
    __shared__ float slots[kSlotSize * BLOCK];
    extern __shared__ float ring[];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned n_units = (unsigned)((io.T + 31) / 32);
    for (;;) {
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(counter, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        const int64_t t = (int64_t)u * 32 + lane;
        if (t < io.T) fit_track<DEPTH>(g, rt, io, t, slots + threadIdx.x, BLOCK, ring + threadIdx.x);
    }
}

using PersistentFn = void (*)(FitGeom, Routing, FitIO, unsigned *);

// Dynamic shared memory of a shape: DEPTH + 1 stages of 9 floats per thread.
constexpr size_t ring_bytes(int block, int depth) { return depth > 1 ? (size_t)(depth + 1) * 9 * block * 4 : 0; }

// (block, register cap, hit prefetch depth) shapes the autotuner chooses
// from; cap 0 = none.  A cap of R registers is
// __launch_bounds__(BLOCK, 65536 / (R * BLOCK)).
struct Shape {
    int block, cap, depth;
    PersistentFn fn;
};
const Shape kShapes[] = {
    {32, 0, 1, fit_persistent_kernel<32, 1, 1>},     {64, 0, 1, fit_persistent_kernel<64, 1, 1>},
    {128, 0, 1, fit_persistent_kernel<128, 1, 1>},   {256, 0, 1, fit_persistent_kernel<256, 1, 1>},
    {32, 168, 1, fit_persistent_kernel<32, 12, 1>},  {64, 168, 1, fit_persistent_kernel<64, 6, 1>},
    {128, 168, 1, fit_persistent_kernel<128, 3, 1>}, {32, 128, 1, fit_persistent_kernel<32, 16, 1>},
    {64, 128, 1, fit_persistent_kernel<64, 8, 1>},   {128, 128, 1, fit_persistent_kernel<128, 4, 1>},
    {256, 128, 1, fit_persistent_kernel<256, 2, 1>}, {32, 96, 1, fit_persistent_kernel<32, 20, 1>},
    {64, 96, 1, fit_persistent_kernel<64, 10, 1>},   {128, 96, 1, fit_persistent_kernel<128, 5, 1>},
    {32, 80, 1, fit_persistent_kernel<32, 24, 1>},   {64, 80, 1, fit_persistent_kernel<64, 12, 1>},
    {128, 80, 1, fit_persistent_kernel<128, 6, 1>},  {256, 80, 1, fit_persistent_kernel<256, 3, 1>},
    {32, 128, 2, fit_persistent_kernel<32, 16, 2>},  {64, 128, 2, fit_persistent_kernel<64, 8, 2>},
    {128, 128, 2, fit_persistent_kernel<128, 4, 2>}, {256, 128, 2, fit_persistent_kernel<256, 2, 2>},
    {32, 96, 2, fit_persistent_kernel<32, 20, 2>},   {64, 96, 2, fit_persistent_kernel<64, 10, 2>},
    {128, 96, 2, fit_persistent_kernel<128, 5, 2>},  {32, 128, 4, fit_persistent_kernel<32, 16, 4>},
    {64, 128, 4, fit_persistent_kernel<64, 8, 4>},   {128, 128, 4, fit_persistent_kernel<128, 4, 4>},
    {256, 128, 4, fit_persistent_kernel<256, 2, 4>}, {32, 96, 4, fit_persistent_kernel<32, 20, 4>},
    {64, 96, 4, fit_persistent_kernel<64, 10, 4>},   {128, 96, 4, fit_persistent_kernel<128, 5, 4>},
};

const Shape *find_shape(int block, int cap, int depth)
{
    for (const Shape &sh : kShapes)
        if (sh.block == block && sh.cap == cap && sh.depth == depth) return &sh;
    return nullptr;
}

// Allow a shape's dynamic shared memory on the current device.  The opt-in
// is a per-device function attribute, so it is remembered per (device,
// shape), under a lock: several host threads may launch at once.
cudaError_t prepare_shape(const Shape *sh)
{
    const size_t bytes = ring_bytes(sh->block, sh->depth);
    if (!bytes) return cudaSuccess;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::set<std::pair<int, const Shape *>> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, sh})) return cudaSuccess;
    e = cudaFuncSetAttribute(sh->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.insert({dev, sh});
    return e;
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

int persistent_blocks_per_sm(int block, int cap, int depth)
{
    const Shape *sh = find_shape(block, cap, depth);
    if (!sh) return 0;
    int n = 0;
    if (prepare_shape(sh) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sh->fn, block, ring_bytes(block, depth)) != cudaSuccess)
        return -1;
    return n;
}

int persistent_shapes(int *blocks, int *caps, int *depths, int max_n)
{
    int n = 0;
    for (const Shape &sh : kShapes)
        if (n < max_n) {
            blocks[n] = sh.block;
            caps[n] = sh.cap;
            depths[n] = sh.depth;
            ++n;
        }
    return n;
}

cudaError_t launch_fit_persistent(const FitGeom &g, const Routing &rt, const FitIO &io, int block, int cap, int depth,
                                  int grid, unsigned *counter, cudaStream_t stream)
{
    const Shape *sh = find_shape(block, cap, depth);
    if (!sh) return cudaErrorInvalidValue;
    const cudaError_t e = prepare_shape(sh);
    if (e != cudaSuccess) return e;
    sh->fn<<<grid, block, ring_bytes(block, depth), stream>>>(g, rt, io, counter);
    return cudaGetLastError();
}

}  // namespace kf
