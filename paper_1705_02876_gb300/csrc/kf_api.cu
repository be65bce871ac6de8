// C interface (include/kf.h): argument checks, launch-shape selection (an
// autotuner over tracks per block), CUDA-graph capture of the persistent fit
// launch, and the context that owns scratch memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "kf.h"
#include "kf_api_internal.h"
#include "kf_fit.cuh"

using namespace kf;

namespace {

struct GraphEntry {
    FitGeom g;
    Routing rt;
    FitIO io;
    FitShape shape;
    int grid;
    cudaGraphExec_t exec;
    uint64_t last_use;
};

bool same_bytes(const void *a, const void *b, size_t n) { return std::memcmp(a, b, n) == 0; }

}  // namespace

struct kf_context {
    int device = 0;
    int sm_count = 0;
    unsigned *d_counter = nullptr;  // persistent-kernel work counter
    cudaStream_t capture_stream = nullptr;
    std::string err;
    // (L, log2 size, precision, fixed block, fixed cap, fixed depth) -> shape
    std::map<std::tuple<int, int, int, int, int, int>, kf::FitShape> tuned;
    std::vector<GraphEntry> graphs;
    uint64_t clock = 0;
    kf::BuildState *build = nullptr;
    kf::MlpState *mlp = nullptr;
    kf::HostPipe *host = nullptr;
    kf::SmoothState *smooth = nullptr;
    kf::SeedState *seed = nullptr;
};

namespace kf {

int set_error(kf_context *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

int cuda_error(kf_context *ctx, cudaError_t e, const char *what)
{
    return set_error(ctx, KF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int context_device(const kf_context *ctx) { return ctx->device; }
int context_sm_count(const kf_context *ctx) { return ctx->sm_count; }
BuildState *&context_build_state(kf_context *ctx) { return ctx->build; }
MlpState *&context_mlp_state(kf_context *ctx) { return ctx->mlp; }
HostPipe *&context_host_state(kf_context *ctx) { return ctx->host; }
SmoothState *&context_smooth_state(kf_context *ctx) { return ctx->smooth; }
SeedState *&context_seed_state(kf_context *ctx) { return ctx->seed; }

int check_geometry(kf_context *ctx, const kf_geometry *geom, FitGeom *g)
{
    if (!geom) return set_error(ctx, KF_ERR_ARG, "geometry is NULL");
    if (geom->n_layers < 1 || geom->n_layers > KF_MAX_LAYERS)
        return set_error(ctx, KF_ERR_ARG, "n_layers %d outside 1..%d", geom->n_layers, KF_MAX_LAYERS);
    if (!geom->r || !geom->x_over_x0) return set_error(ctx, KF_ERR_ARG, "geometry arrays are NULL");
    if (!(geom->z_half > 0.0f) || !std::isfinite(geom->z_half))
        return set_error(ctx, KF_ERR_ARG, "z_half must be positive and finite");
    if (!std::isfinite(geom->bz_tesla)) return set_error(ctx, KF_ERR_ARG, "bz_tesla is not finite");
    std::memset(g, 0, sizeof *g);
    g->L = geom->n_layers;
    g->z_half = geom->z_half;
    g->qk = kField * geom->bz_tesla;
    for (int l = 0; l < geom->n_layers; ++l) {
        const float r = geom->r[l], x = geom->x_over_x0[l];
        if (!(r > 0.0f) || !std::isfinite(r) || (l > 0 && !(r > geom->r[l - 1])))
            return set_error(ctx, KF_ERR_ARG, "radii must be positive, finite and increasing (layer %d)", l);
        if (!(x >= 0.0f) || !std::isfinite(x))
            return set_error(ctx, KF_ERR_ARG, "x_over_x0[%d] must be finite and >= 0", l);
        g->r[l] = r;
        g->inv_r[l] = 1.0f / r;
        g->xx0[l] = x;
    }
    return KF_OK;
}

int check_ptr(kf_context *ctx, const void *p, size_t align, const char *name)
{
    if (!p) return set_error(ctx, KF_ERR_ARG, "%s is NULL", name);
    if (reinterpret_cast<uintptr_t>(p) % align)
        return set_error(ctx, KF_ERR_ARG, "%s is not %zu-byte aligned", name, align);
    return KF_OK;
}

Routing make_routing(const kf_options &o)
{
    Routing rt;
    rt.mode = o.precision_mode;
    rt.det_min = 6.75f / o.cond_max;
    rt.pt_lo = o.pt_lo;
    rt.pt_hi = o.pt_hi;
    rt.gain_max = o.gain_max;
    return rt;
}

int check_options(kf_context *ctx, const kf_options &o)
{
    if (o.precision_mode != KF_PRECISION_FP32 && o.precision_mode != KF_PRECISION_ROUTED)
        return set_error(ctx, KF_ERR_ARG, "precision_mode %d", o.precision_mode);
    if (o.precision_mode == KF_PRECISION_ROUTED &&
        (!(o.cond_max > 1.0f) || !(o.pt_lo >= 0.0f) || !(o.pt_hi > o.pt_lo) || !(o.gain_max >= 0.0f)))
        return set_error(ctx, KF_ERR_ARG, "routing thresholds: cond_max > 1, 0 <= pt_lo < pt_hi, gain_max >= 0");
    if (o.launch_mode < KF_LAUNCH_AUTO || o.launch_mode > KF_LAUNCH_FLAT)
        return set_error(ctx, KF_ERR_ARG, "launch_mode %d", o.launch_mode);
    if (o.tracks_per_block != 0 && o.tracks_per_block != 32 && o.tracks_per_block != 64 &&
        o.tracks_per_block != 128 && o.tracks_per_block != 256)
        return set_error(ctx, KF_ERR_ARG, "tracks_per_block must be 0, 32, 64, 128 or 256");
    if (o.reg_cap != 0 && o.reg_cap != -1 && o.reg_cap != 168 && o.reg_cap != 128 && o.reg_cap != 96 &&
        o.reg_cap != 80)
        return set_error(ctx, KF_ERR_ARG, "reg_cap must be 0, -1, 168, 128, 96 or 80");
    if (o.hit_prefetch != 0 && o.hit_prefetch != 1 && o.hit_prefetch != 2 && o.hit_prefetch != 4)
        return set_error(ctx, KF_ERR_ARG, "hit_prefetch must be 0, 1, 2 or 4");
    return KF_OK;
}

}  // namespace kf

extern "C" {

void kf_options_default(kf_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision_mode = KF_PRECISION_ROUTED;
    o->cond_max = 1e4f;
    o->pt_lo = 0.25f;
    o->pt_hi = 200.0f;
    o->gain_max = 0.0f;
    o->launch_mode = KF_LAUNCH_AUTO;
    o->tracks_per_block = 0;
    o->reg_cap = 0;
    o->hit_prefetch = 0;
    o->max_cands = 6;
    o->chi2_cut = 30.0f;
    o->window_nsigma = 3.0f;
    o->hit_sigma_rphi = 0.01f;
    o->hit_sigma_z = 0.1f;
    o->window_max_dphi = 0.05f;
    o->window_max_dz = 5.0f;
    o->n_phi_bins = 0;
    o->n_z_bins = 0;
    o->use_proposal = 0;
    o->topk = 4;
    o->build_variant = -1;
}

int kf_context_create(kf_context **out, int device)
{
    if (!out) return KF_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return KF_ERR_UNSUPPORTED;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return KF_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return KF_ERR_UNSUPPORTED;  // built for sm_103a only
    DeviceGuard dg(device);
    kf_context *ctx = new kf_context;
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    if (cudaMalloc(&ctx->d_counter, 256) != cudaSuccess) {
        delete ctx;
        return KF_ERR_NOMEM;
    }
    if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(ctx->d_counter);
        delete ctx;
        return KF_ERR_CUDA;
    }
    *out = ctx;
    return KF_OK;
}

void kf_context_destroy(kf_context *ctx)
{
    if (!ctx) return;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    for (auto &e : ctx->graphs) cudaGraphExecDestroy(e.exec);
    kf::destroy_build_state(ctx->build);
    kf::destroy_mlp_state(ctx->mlp);
    kf::destroy_host_state(ctx->host);
    kf::destroy_smooth_state(ctx->smooth);
    kf::destroy_seed_state(ctx->seed);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    cudaFree(ctx->d_counter);
    delete ctx;
}

const char *kf_last_error(const kf_context *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

}  // extern "C"

namespace {

int size_class(int64_t n)
{
    int c = 0;
    while ((int64_t(1) << (c + 1)) <= n && c < 40) ++c;
    return c;
}

// Enqueue the persistent fit: counter reset + kernel, replayed from a cached
// CUDA graph when this exact launch was captured before.
cudaError_t enqueue_persistent(kf_context *ctx, const FitGeom &g, const Routing &rt, const FitIO &io,
                               const FitShape &sh, cudaStream_t stream, bool use_graph)
{
    const int block = sh.block;
    const int per_sm = persistent_blocks_per_sm(block, sh.cap, sh.depth);
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const int64_t units = (io.T + 31) / 32;
    const int64_t want = (units * 32 + block - 1) / block;
    const int grid = (int)std::min<int64_t>((int64_t)ctx->sm_count * per_sm, std::max<int64_t>(want, 1));
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(stream, &capst);
    if (!use_graph || capst != cudaStreamCaptureStatusNone) {
        cudaError_t e = cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned), stream);
        if (e != cudaSuccess) return e;
        return launch_fit_persistent(g, rt, io, block, sh.cap, sh.depth, grid, ctx->d_counter, stream);
    }
    for (auto &e : ctx->graphs) {
        if (e.shape.block == block && e.shape.cap == sh.cap && e.shape.depth == sh.depth && e.grid == grid &&
            same_bytes(&e.g, &g, sizeof g) &&
            same_bytes(&e.rt, &rt, sizeof rt) && same_bytes(&e.io, &io, sizeof io)) {
            e.last_use = ++ctx->clock;
            return cudaGraphLaunch(e.exec, stream);
        }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e1 = cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned), ctx->capture_stream);
    cudaError_t e2 = e1 == cudaSuccess
                         ? launch_fit_persistent(g, rt, io, block, sh.cap, sh.depth, grid, ctx->d_counter,
                                                 ctx->capture_stream)
                         : e1;
    e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (e2 != cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (ctx->graphs.size() >= 16) {  // evict the least recently used
        size_t lru = 0;
        for (size_t i = 1; i < ctx->graphs.size(); ++i)
            if (ctx->graphs[i].last_use < ctx->graphs[lru].last_use) lru = i;
        cudaGraphExecDestroy(ctx->graphs[lru].exec);
        ctx->graphs.erase(ctx->graphs.begin() + lru);
    }
    ctx->graphs.push_back(GraphEntry{g, rt, io, sh, grid, exec, ++ctx->clock});
    return cudaGraphLaunch(exec, stream);
}

// Time every compiled (tracks per block, register cap, hit prefetch depth)
// shape on the caller's own buffers (the fit is idempotent: it reads its
// inputs and overwrites its outputs) and keep the fastest for this layer
// count, size class and precision.  Skipped while the stream is being
// captured.  fixed (fields 0 = free; cap -1 = uncapped) restricts the search
// to matching shapes.
FitShape tune_shape(kf_context *ctx, const FitGeom &g, const Routing &rt, const FitIO &io, cudaStream_t stream,
                    const FitShape &fixed)
{
    const auto key = std::make_tuple(g.L, size_class(io.T), rt.mode, fixed.block, fixed.cap, fixed.depth);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) return it->second;
    FitShape cand[64];
    int n = 0;
    {
        int all_b[64], all_c[64], all_d[64];
        const int m = persistent_shapes(all_b, all_c, all_d, 64);
        for (int i = 0; i < m; ++i)
            if ((!fixed.block || all_b[i] == fixed.block) &&
                (!fixed.cap || all_c[i] == (fixed.cap < 0 ? 0 : fixed.cap)) &&
                (!fixed.depth || all_d[i] == fixed.depth))
                cand[n++] = FitShape{all_b[i], all_c[i], all_d[i]};
    }
    if (n == 0)
        return FitShape{fixed.block ? fixed.block : 128, fixed.cap > 0 ? fixed.cap : 0, fixed.depth ? fixed.depth : 1};
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(stream, &capst);
    if (capst != cudaStreamCaptureStatusNone) return cand[0];
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    FitShape best = cand[0];
    float best_ms = 1e30f;
    for (int i = 0; i < n; ++i) {
        if (enqueue_persistent(ctx, g, rt, io, cand[i], stream, false) != cudaSuccess) continue;
        cudaEventRecord(a, stream);
        for (int rep = 0; rep < 3; ++rep) enqueue_persistent(ctx, g, rt, io, cand[i], stream, false);
        cudaEventRecord(b, stream);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
            best_ms = ms;
            best = cand[i];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->tuned[key] = best;
    return best;
}

}  // namespace

extern "C" {

int kf_fit_tracks(kf_context *ctx, const kf_geometry *geom, int64_t n_tracks, const int64_t *event_offsets,
                  int n_events, const float *seed_state, const float *seed_cov, const int8_t *charge,
                  const float *hit_pos, const float *hit_cov, const uint32_t *hit_mask, float *out_state,
                  float *out_cov, float *out_chi2, int16_t *out_ndof, uint32_t *out_flags, const kf_options *opt,
                  kf_stream stream_)
{
    if (!ctx) return KF_ERR_ARG;
    ctx->err.clear();
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    kf_options o;
    if (opt) o = *opt;
    else kf_options_default(&o);
    int rc;
    FitGeom g;
    if ((rc = check_geometry(ctx, geom, &g))) return rc;
    if ((rc = check_options(ctx, o))) return rc;
    if (n_tracks < 0 || n_tracks > (int64_t(1) << 36))
        return set_error(ctx, KF_ERR_ARG, "n_tracks %lld out of range", (long long)n_tracks);
    if (n_tracks == 0) return KF_OK;
    if ((rc = check_ptr(ctx, seed_state, 4, "seed_state")) || (rc = check_ptr(ctx, seed_cov, 4, "seed_cov")) ||
        (rc = check_ptr(ctx, charge, 1, "charge")) || (rc = check_ptr(ctx, hit_pos, 4, "hit_pos")) ||
        (rc = check_ptr(ctx, hit_cov, 4, "hit_cov")) || (rc = check_ptr(ctx, hit_mask, 4, "hit_mask")) ||
        (rc = check_ptr(ctx, out_state, 4, "out_state")) || (rc = check_ptr(ctx, out_cov, 4, "out_cov")) ||
        (rc = check_ptr(ctx, out_chi2, 4, "out_chi2")) || (rc = check_ptr(ctx, out_ndof, 2, "out_ndof")) ||
        (rc = check_ptr(ctx, out_flags, 4, "out_flags")))
        return rc;
    if (o.launch_mode == KF_LAUNCH_PER_EVENT) {
        if (!event_offsets || n_events < 1)
            return set_error(ctx, KF_ERR_ARG, "per-event launches need event_offsets and n_events >= 1");
        if (event_offsets[0] != 0 || event_offsets[n_events] != n_tracks)
            return set_error(ctx, KF_ERR_ARG, "event_offsets must run from 0 to n_tracks");
        for (int e = 0; e < n_events; ++e)
            if (event_offsets[e + 1] < event_offsets[e])
                return set_error(ctx, KF_ERR_ARG, "event_offsets decrease at event %d", e);
    }
    DeviceGuard dg(ctx->device);
    FitIO io{n_tracks, seed_state, seed_cov, charge, hit_pos, hit_cov, hit_mask,
             out_state, out_cov, out_chi2, out_ndof, out_flags};
    const Routing rt = make_routing(o);
    cudaError_t e = cudaSuccess;
    const int block = o.tracks_per_block ? o.tracks_per_block : 0;
    switch (o.launch_mode) {
    case KF_LAUNCH_FLAT:
        e = launch_fit_plain(g, rt, io, 0, n_tracks, block ? block : 128, stream);
        break;
    case KF_LAUNCH_PER_EVENT:
        for (int ev = 0; ev < n_events && e == cudaSuccess; ++ev)
            e = launch_fit_plain(g, rt, io, event_offsets[ev], event_offsets[ev + 1], block ? block : 128, stream);
        break;
    default: {
        FitShape shape{block, o.reg_cap < 0 ? 0 : o.reg_cap, o.hit_prefetch};
        if (!block || !o.reg_cap || !o.hit_prefetch)
            shape = tune_shape(ctx, g, rt, io, stream, FitShape{block, o.reg_cap, o.hit_prefetch});
        e = enqueue_persistent(ctx, g, rt, io, shape, stream, true);
    }
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "fit launch");
    return KF_OK;
}

int kf_fit_tuned_shape(kf_context *ctx, int n_layers, int64_t n_tracks, int *tracks_per_block, int *reg_cap,
                       int *hit_prefetch)
{
    if (!ctx || !tracks_per_block || !reg_cap || !hit_prefetch) return KF_ERR_ARG;
    for (int mode = 1; mode >= 0; --mode) {
        auto it = ctx->tuned.find(std::make_tuple(n_layers, size_class(n_tracks), mode, 0, 0, 0));
        if (it != ctx->tuned.end()) {
            *tracks_per_block = it->second.block;
            *reg_cap = it->second.cap ? it->second.cap : -1;
            *hit_prefetch = it->second.depth;
            return KF_OK;
        }
    }
    return set_error(ctx, KF_ERR_ARG, "no fit of %d layers and this size has been tuned yet", n_layers);
}

}  // extern "C"
