// The fit from host buffers (the paper's multi-stream event transfers, Section
// 4.2; its builds spent about half their wall time on host-device transfers,
// Section 4.3).  Page-locked buffers the device can address are read and
// written in place by one persistent launch: on this part the kernel's loads
// over the host link run as fast as the copy engines (about 210 GB/s), and the
// inputs' reads and the outputs' writes share the link in both directions
// with no pipeline fill or drain.  Other buffers go through chunks copied in,
// fitted and copied out on a ring of streams, so that the copies of one chunk
// overlap the fit of the next.
#include <algorithm>

#include "kf.h"
#include "kf_api_internal.h"
#include "kf_fit.cuh"

namespace kf {

constexpr int kHostStreams = 3;

struct HostPipe {
    cudaStream_t stream[kHostStreams] = {};
    unsigned *counter = nullptr;  // one work counter per stream
    char *buf[kHostStreams] = {};  // staging for one chunk per stream
    size_t buf_bytes = 0;
};

void destroy_host_state(HostPipe *s)
{
    if (!s) return;
    for (int i = 0; i < kHostStreams; ++i) {
        if (s->stream[i]) cudaStreamDestroy(s->stream[i]);
        cudaFree(s->buf[i]);
    }
    cudaFree(s->counter);
    delete s;
}

namespace {

// Bytes of one chunk's staging for n tracks of L layers, each array padded to
// 256 bytes.
struct ChunkLayout {
    size_t seed_state, seed_cov, charge, hit_pos, hit_cov, mask, out_state, out_cov, out_chi2, out_ndof, out_flags,
        total;
    ChunkLayout(int64_t n, int L)
    {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o += (bytes + 255) / 256 * 256;
            return at;
        };
        seed_state = take(6 * n * 4);
        seed_cov = take(21 * n * 4);
        charge = take(n);
        hit_pos = take((size_t)L * 3 * n * 4);
        hit_cov = take((size_t)L * 6 * n * 4);
        mask = take(n * 4);
        out_state = take(6 * n * 4);
        out_cov = take(21 * n * 4);
        out_chi2 = take(n * 4);
        out_ndof = take(n * 2);
        out_flags = take(n * 4);
        total = o;
    }
};

}  // namespace
}  // namespace kf

using namespace kf;

extern "C" int kf_fit_tracks_host(kf_context *ctx, const kf_geometry *geom, int64_t n_tracks, const float *seed_state,
                                  const float *seed_cov, const int8_t *charge, const float *hit_pos,
                                  const float *hit_cov, const uint32_t *hit_mask, float *out_state, float *out_cov,
                                  float *out_chi2, int16_t *out_ndof, uint32_t *out_flags, int64_t chunk_tracks,
                                  const kf_options *opt)
{
    if (!ctx) return KF_ERR_ARG;
    kf_options o;
    if (opt) o = *opt;
    else kf_options_default(&o);
    int rc;
    FitGeom g;
    if ((rc = check_geometry(ctx, geom, &g))) return rc;
    if ((rc = check_options(ctx, o))) return rc;
    if (n_tracks < 0 || n_tracks > (int64_t(1) << 36))
        return set_error(ctx, KF_ERR_ARG, "n_tracks %lld out of range", (long long)n_tracks);
    if (chunk_tracks < 0) return set_error(ctx, KF_ERR_ARG, "chunk_tracks must be >= 0");
    if (n_tracks == 0) return KF_OK;
    if ((rc = check_ptr(ctx, seed_state, 4, "seed_state")) || (rc = check_ptr(ctx, seed_cov, 4, "seed_cov")) ||
        (rc = check_ptr(ctx, charge, 1, "charge")) || (rc = check_ptr(ctx, hit_pos, 4, "hit_pos")) ||
        (rc = check_ptr(ctx, hit_cov, 4, "hit_cov")) || (rc = check_ptr(ctx, hit_mask, 4, "hit_mask")) ||
        (rc = check_ptr(ctx, out_state, 4, "out_state")) || (rc = check_ptr(ctx, out_cov, 4, "out_cov")) ||
        (rc = check_ptr(ctx, out_chi2, 4, "out_chi2")) || (rc = check_ptr(ctx, out_ndof, 2, "out_ndof")) ||
        (rc = check_ptr(ctx, out_flags, 4, "out_flags")))
        return rc;
    const int block = o.tracks_per_block ? o.tracks_per_block : 64;
    const int cap = o.reg_cap < 0 ? 0 : (o.reg_cap ? o.reg_cap : 128);
    DeviceGuard dg(context_device(ctx));
    const int depth = o.hit_prefetch ? o.hit_prefetch : 1;
    const int per_sm = persistent_blocks_per_sm(block, cap, depth);
    if (per_sm < 1)
        return set_error(ctx, KF_ERR_ARG, "no persistent fit of %d tracks per block, cap %d, hit prefetch %d", block,
                         cap, depth);
    const int grid = per_sm * context_sm_count(ctx);
    int64_t C = chunk_tracks ? chunk_tracks : (int64_t(1) << 18);
    C = std::min<int64_t>(C, n_tracks);
    C = (C + 31) / 32 * 32;
    const int L = g.L;
    const ChunkLayout lay(C, L);

    HostPipe *&hp = context_host_state(ctx);
    if (!hp) {
        hp = new HostPipe;
        bool ok = cudaMalloc(&hp->counter, kHostStreams * sizeof(unsigned)) == cudaSuccess;
        for (int i = 0; ok && i < kHostStreams; ++i)
            ok = cudaStreamCreateWithFlags(&hp->stream[i], cudaStreamNonBlocking) == cudaSuccess;
        if (!ok) {
            destroy_host_state(hp);
            hp = nullptr;
            return set_error(ctx, KF_ERR_NOMEM, "could not create the host pipeline's streams");
        }
    }
    const Routing rt = make_routing(o);
    // page-locked buffers the device addresses in place: one launch, the
    // transfers happen inside the kernel's loads and stores
    if (chunk_tracks == 0) {
        const void *host[11] = {seed_state, seed_cov, charge, hit_pos, hit_cov, hit_mask,
                                out_state, out_cov, out_chi2, out_ndof, out_flags};
        void *dev[11] = {};
        bool mapped = true;
        for (int i = 0; i < 11 && mapped; ++i) {
            cudaPointerAttributes a{};
            if (cudaPointerGetAttributes(&a, host[i]) != cudaSuccess) {
                cudaGetLastError();  // clear: an unknown pointer is an answer, not an error
                mapped = false;
            } else {
                mapped = a.type == cudaMemoryTypeHost && a.devicePointer != nullptr;
                dev[i] = a.devicePointer;
            }
        }
        if (mapped) {
            const FitIO io{n_tracks,
                           static_cast<const float *>(dev[0]),
                           static_cast<const float *>(dev[1]),
                           static_cast<const int8_t *>(dev[2]),
                           static_cast<const float *>(dev[3]),
                           static_cast<const float *>(dev[4]),
                           static_cast<const uint32_t *>(dev[5]),
                           static_cast<float *>(dev[6]),
                           static_cast<float *>(dev[7]),
                           static_cast<float *>(dev[8]),
                           static_cast<int16_t *>(dev[9]),
                           static_cast<uint32_t *>(dev[10])};
            cudaStream_t s = hp->stream[0];
            const int64_t units = (n_tracks + 31) / 32;
            const int grid_n = (int)std::min<int64_t>(grid, std::max<int64_t>((units * 32 + block - 1) / block, 1));
            cudaError_t e = cudaMemsetAsync(hp->counter, 0, sizeof(unsigned), s);
            if (e == cudaSuccess) e = launch_fit_persistent(g, rt, io, block, cap, depth, grid_n, hp->counter, s);
            const cudaError_t e2 = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_error(ctx, e, "host-buffer fit");
            if (e2 != cudaSuccess) return cuda_error(ctx, e2, "host-buffer fit");
            return KF_OK;
        }
    }
    if (hp->buf_bytes < lay.total) {
        for (int i = 0; i < kHostStreams; ++i) {
            cudaStreamSynchronize(hp->stream[i]);
            cudaFree(hp->buf[i]);
            hp->buf[i] = nullptr;
        }
        hp->buf_bytes = 0;
        for (int i = 0; i < kHostStreams; ++i)
            if (cudaMalloc(&hp->buf[i], lay.total) != cudaSuccess)
                return set_error(ctx, KF_ERR_NOMEM, "could not allocate %zu bytes of staging", lay.total);
        hp->buf_bytes = lay.total;
    }

    const int64_t T = n_tracks;
    const int64_t n_chunks = (T + C - 1) / C;
    cudaError_t e = cudaSuccess;
    for (int64_t c = 0; c < n_chunks && e == cudaSuccess; ++c) {
        const int k = (int)(c % kHostStreams);
        cudaStream_t s = hp->stream[k];
        char *b = hp->buf[k];
        const int64_t t0 = c * C, n = std::min<int64_t>(C, T - t0);
        // rows of a host [rows][T] array from track t0, to or from a device
        // [rows][n] block: one strided copy per array
        auto in = [&](size_t off, const void *host, size_t elem, size_t rows) {
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(b + off, n * elem, (const char *)host + t0 * elem, T * elem, n * elem, rows,
                                      cudaMemcpyHostToDevice, s);
        };
        auto out = [&](void *host, size_t off, size_t elem, size_t rows) {
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync((char *)host + t0 * elem, T * elem, b + off, n * elem, n * elem, rows,
                                      cudaMemcpyDeviceToHost, s);
        };
        in(lay.seed_state, seed_state, 4, 6);
        in(lay.seed_cov, seed_cov, 4, 21);
        in(lay.charge, charge, 1, 1);
        in(lay.hit_pos, hit_pos, 4, (size_t)L * 3);
        in(lay.hit_cov, hit_cov, 4, (size_t)L * 6);
        in(lay.mask, hit_mask, 4, 1);
        if (e == cudaSuccess) e = cudaMemsetAsync(hp->counter + k, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) {
            FitIO io{n,
                     reinterpret_cast<const float *>(b + lay.seed_state),
                     reinterpret_cast<const float *>(b + lay.seed_cov),
                     reinterpret_cast<const int8_t *>(b + lay.charge),
                     reinterpret_cast<const float *>(b + lay.hit_pos),
                     reinterpret_cast<const float *>(b + lay.hit_cov),
                     reinterpret_cast<const uint32_t *>(b + lay.mask),
                     reinterpret_cast<float *>(b + lay.out_state),
                     reinterpret_cast<float *>(b + lay.out_cov),
                     reinterpret_cast<float *>(b + lay.out_chi2),
                     reinterpret_cast<int16_t *>(b + lay.out_ndof),
                     reinterpret_cast<uint32_t *>(b + lay.out_flags)};
            e = launch_fit_persistent(g, rt, io, block, cap, depth, grid, hp->counter + k, s);
        }
        out(out_state, lay.out_state, 4, 6);
        out(out_cov, lay.out_cov, 4, 21);
        out(out_chi2, lay.out_chi2, 4, 1);
        out(out_ndof, lay.out_ndof, 2, 1);
        out(out_flags, lay.out_flags, 4, 1);
    }
    cudaError_t e2 = cudaSuccess;
    for (int i = 0; i < kHostStreams; ++i) {
        const cudaError_t ei = cudaStreamSynchronize(hp->stream[i]);
        if (e2 == cudaSuccess) e2 = ei;
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "host-buffer fit");
    if (e2 != cudaSuccess) return cuda_error(ctx, e2, "host-buffer fit");
    return KF_OK;
}
