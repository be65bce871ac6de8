// kf_fit_tracks_noalloc: the Kalman-filter fit for callers that cannot
// allocate device memory.
//
// kf_fit_tracks needs a kf_context, and creating one calls cudaMalloc for the
// context's scratch.  Some callers cannot do that: code that runs inside a
// device-memory pool it does not own and may not grow, allocation-free
// real-time or embedded loops that must not touch the allocator after
// start-up, and hosts that forbid allocation while their own work is in
// flight.  This entry point runs the same persistent fit kernel, but the only
// scratch that kernel needs -- the 32-bit counter from which its warps claim
// 32-track units -- lives in a fixed array of this file's device memory.
// Nothing here calls cudaMalloc, cudaFree or any routine that allocates.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "kf.h"
#include "kf_api_internal.h"

// The scratch: one 32-bit work counter, 4 bytes.  Every GPU that loads the
// library holds this array until the process exits.  All calls on a device
// share it and it keeps the last call's contents; each call clears the
// counter on its own stream before its launch.
static __device__ __align__(256) unsigned g_noalloc_scratch[1];

namespace {

constexpr int kMaxDevices = 64;
// resident warps a launch may hold so that the work counter cannot wrap:
// KF_NOALLOC_MAX_TRACKS / 32 units plus this many final claims stay below 2^32
constexpr int64_t kNoallocMaxWarps = 16384;
static_assert(KF_NOALLOC_MAX_TRACKS / 32 + kNoallocMaxWarps < (int64_t(1) << 32), "counter margin");
unsigned *g_scratch_address[kMaxDevices];  // device address of g_noalloc_scratch, per device
std::mutex g_setup_mutex;

// Once per device, with that device current: look up the array's device
// address.  In host code the symbol is only a host-side stand-in; a kernel
// must be given this address instead.
cudaError_t scratch_address(int device, unsigned **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_address[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_address[device] = static_cast<unsigned *>(p);
    }
    *out = g_scratch_address[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int kf_fit_tracks_noalloc(const kf_geometry *geom, int64_t n_tracks, const float *seed_state,
                                     const float *seed_cov, const int8_t *charge, const float *hit_pos,
                                     const float *hit_cov, const uint32_t *hit_mask, float *out_state,
                                     float *out_cov, float *out_chi2, int16_t *out_ndof, uint32_t *out_flags,
                                     const kf_options *opt, kf_stream stream_)
{
    using namespace kf;
    kf_options o;
    if (opt) o = *opt;
    else kf_options_default(&o);
    int rc;
    FitGeom g;
    if ((rc = check_geometry(nullptr, geom, &g))) return rc;
    if ((rc = check_options(nullptr, o))) return rc;
    if (n_tracks < 0) return KF_ERR_ARG;
    if (n_tracks > KF_NOALLOC_MAX_TRACKS) return KF_ERR_TOO_LARGE;
    if (n_tracks == 0) return KF_OK;
    if ((rc = check_ptr(nullptr, seed_state, 4, "")) || (rc = check_ptr(nullptr, seed_cov, 4, "")) ||
        (rc = check_ptr(nullptr, charge, 1, "")) || (rc = check_ptr(nullptr, hit_pos, 4, "")) ||
        (rc = check_ptr(nullptr, hit_cov, 4, "")) || (rc = check_ptr(nullptr, hit_mask, 4, "")) ||
        (rc = check_ptr(nullptr, out_state, 4, "")) || (rc = check_ptr(nullptr, out_cov, 4, "")) ||
        (rc = check_ptr(nullptr, out_chi2, 4, "")) || (rc = check_ptr(nullptr, out_ndof, 2, "")) ||
        (rc = check_ptr(nullptr, out_flags, 4, "")))
        return rc;
    int device = -1, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return KF_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return KF_ERR_CUDA;
    unsigned *counter = nullptr;
    if (scratch_address(device, &counter) != cudaSuccess) return KF_ERR_CUDA;

    // fixed launch shape (no tuning runs here): the caller's choice, else 64
    // tracks per block without a register cap, hits prefetched into registers
    const int block = o.tracks_per_block ? o.tracks_per_block : 64;
    const int cap = o.reg_cap > 0 ? o.reg_cap : 0;
    const int depth = o.hit_prefetch ? o.hit_prefetch : 1;
    const int per_sm = persistent_blocks_per_sm(block, cap, depth);
    if (per_sm == 0) return KF_ERR_ARG;  // this (block, cap, depth) combination is not compiled in
    if (per_sm < 0) return KF_ERR_CUDA;
    const int64_t units = (n_tracks + 31) / 32;
    const int64_t want = (units * 32 + block - 1) / block;
    const int grid = (int)std::min<int64_t>((int64_t)sms * per_sm, want);
    // every resident warp makes one claim past the last unit before it stops:
    // the counter stays below 2^32 while units + resident warps do
    if ((int64_t)grid * (block / 32) > kNoallocMaxWarps) return KF_ERR_TOO_LARGE;
    const FitIO io{n_tracks, seed_state, seed_cov, charge, hit_pos, hit_cov, hit_mask,
                   out_state, out_cov, out_chi2, out_ndof, out_flags};
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned), stream) != cudaSuccess) return KF_ERR_CUDA;
    if (launch_fit_persistent(g, make_routing(o), io, block, cap, depth, grid, counter, stream) != cudaSuccess)
        return KF_ERR_CUDA;
    return KF_OK;
}
