// Internal helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kf.h"
#include "kf_fit.cuh"

namespace kf {

struct BuildState;  // device scratch of the build step (kf_build.cu)
void destroy_build_state(BuildState *s);
struct MlpState;  // proposal network scratch and weights (kf_mlp.cu)
void destroy_mlp_state(MlpState *s);
struct HostPipe;  // staging buffers and streams of the host-buffer fit (kf_host.cu)
void destroy_host_state(HostPipe *s);
struct SmoothState;  // per-layer scratch of the smoother (kf_smooth.cu)
void destroy_smooth_state(SmoothState *s);
struct SeedState;  // binned seed-layer hits and found triplets (kf_seed.cu)
void destroy_seed_state(SeedState *s);
bool proposal_loaded(kf_context *ctx);
// device copies of the loaded weights (the layouts of kf_mlp.cuh)
void proposal_weights(kf_context *ctx, const __nv_bfloat16 **W1, const __nv_bfloat16 **W2, const float **w32);

int set_error(kf_context *ctx, int code, const char *fmt, ...);
int cuda_error(kf_context *ctx, cudaError_t e, const char *what);
int check_geometry(kf_context *ctx, const kf_geometry *geom, FitGeom *g);
int check_ptr(kf_context *ctx, const void *p, size_t align, const char *name);
int check_options(kf_context *ctx, const kf_options &o);
Routing make_routing(const kf_options &o);
int context_device(const kf_context *ctx);
int context_sm_count(const kf_context *ctx);
BuildState *&context_build_state(kf_context *ctx);
MlpState *&context_mlp_state(kf_context *ctx);
HostPipe *&context_host_state(kf_context *ctx);
SmoothState *&context_smooth_state(kf_context *ctx);
SeedState *&context_seed_state(kf_context *ctx);

// Make `dev` current for a scope, restoring the caller's device after.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};


}  // namespace kf
