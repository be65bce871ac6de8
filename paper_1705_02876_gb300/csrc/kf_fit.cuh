// Track-fit kernels: shared declarations between the kernels and the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kf_math.cuh"

namespace kf {

constexpr int kMaxLayers = 32;

struct FitGeom {
    int L;
    float z_half;
    float qk;  // k * Bz; a track's curvature is charge * qk / pT
    float r[kMaxLayers];
    float inv_r[kMaxLayers];
    float xx0[kMaxLayers];
};

struct FitIO {
    int64_t T;  // row stride of every [..][T] array (tracks in the batch)
    const float *seed_state;
    const float *seed_cov;
    const int8_t *charge;
    const float *hit_pos;
    const float *hit_cov;
    const uint32_t *hit_mask;
    float *out_state;
    float *out_cov;
    float *out_chi2;
    int16_t *out_ndof;
    uint32_t *out_flags;
};

// A persistent-fit launch shape: threads per block, register cap (0 = none)
// and hit prefetch depth (layers ahead).
struct FitShape {
    int block, cap, depth;
};

// status word bits written by the persistent kernels (device scratch)
constexpr unsigned kStatusTimeout = 1u;

// Launchers (kf_fit.cu).  All enqueue on `stream` and return the launch error.
cudaError_t launch_fit_plain(const FitGeom &g, const Routing &rt, const FitIO &io, int64_t t_begin,
                             int64_t t_end, int block, cudaStream_t stream);
// Persistent kernel: grid = `grid` blocks of `block` threads with registers
// capped at `cap` per thread (0 = no cap), hits loaded `depth` layers ahead
// (1: registers; 2, 4: a cp.async ring in shared memory); warps claim 32-track
// units from *counter, which must read 0 at launch.
cudaError_t launch_fit_persistent(const FitGeom &g, const Routing &rt, const FitIO &io, int block, int cap,
                                  int depth, int grid, unsigned *counter, cudaStream_t stream);
// Blocks of the persistent kernel of this shape that fit on one SM at once on
// the current device: 0 if the shape is not compiled in, -1 if a CUDA call
// (the shared-memory opt-in or the occupancy query) failed.
int persistent_blocks_per_sm(int block, int cap, int depth);
// The (block, cap, depth) shapes compiled in; returns how many were written.
int persistent_shapes(int *blocks, int *caps, int *depths, int max_n);

}  // namespace kf
