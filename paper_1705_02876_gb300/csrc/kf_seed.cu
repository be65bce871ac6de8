// Seeding from hits on sm_103a: triplets of hits on the first three layers of
// every event that a track from the beam line above a pT threshold could have
// made, and the seed-fit inputs built from them.  The paper seeds from the
// true hits of each simulated track and says realistic seeding is under
// development (Section 2); this search replaces the truth.
//
// A triplet (h0, h1, h2) is a seed when (all with the hits' own radii r_i,
// azimuths phi_i and z_i):
//   (a), (e) |phi_1 - phi_0| <= w01 and |phi_2 - phi_1| <= w12, with
//            w_ab = asin(R_b / 2 R_min) - asin(R_a / 2 R_min) + d0_max (1/R_a + 1/R_b),
//            R_a the layers' radii, R_min = pt_min / (k |Bz|);
//   (b)      the line through (r_0, z_0), (r_1, z_1) meets r = 0 within z0_max;
//   (d)      it predicts z at r_2 within dz_max;
//   (c)      the circle through the three (x, y) points has |kappa| <=
//            k |Bz| / pt_min and passes within d0_max of the beam line:
//            kappa = 2 orient / (|P1-P0| |P2-P1| |P2-P0|), orient = (P1-P0) x (P2-P0),
//            F = -incircle(P0, P1, P2, O) / orient (the origin's power),
//            d0 = |F| |kappa| / (1 + sqrt(max(0, 1 + F kappa^2))).
// Charge: q = +1 when orient Bz < 0 (a positive charge turns clockwise in
// Bz > 0); a triplet with pT above pt_both_charges (|kappa| the hits cannot
// resolve) seeds both charges.
//
// One warp per hit of the middle layer scans the binned hits of layer 0 in
// its window, and for every doublet passing (a) and (b) the binned hits of
// layer 2 in theirs; the windows' z ranges are widened for hit radii within
// 0.1 cm of the layer radius, and every candidate is then tested exactly.
#include <algorithm>
#include <vector>

#include "kf.h"
#include "kf_api_internal.h"
#include "kf_bins.cuh"

namespace kf {

struct SeedState {
    float4 *bkey = nullptr;
    size_t key_cap = 0;
    int32_t *bin_off = nullptr;
    size_t bin_cap = 0;
    int32_t *hit_rank = nullptr;  // the binning's rank of each hit within its bin
    size_t rank_cap = 0;
    int64_t *seg_off = nullptr;
    size_t seg_cap = 0;
    int32_t *trip = nullptr;  // [5][trip_cap]: event, h0, h1, h2 (global), charge
    int64_t trip_cap = 0;
    unsigned long long *count = nullptr;
    int64_t n = 0;  // triplets found by the last search
    int64_t n_hits = 0;
};

void destroy_seed_state(SeedState *s)
{
    if (!s) return;
    cudaFree(s->bkey);
    cudaFree(s->bin_off);
    cudaFree(s->hit_rank);
    cudaFree(s->seg_off);
    cudaFree(s->trip);
    cudaFree(s->count);
    delete s;
}

namespace {

constexpr float kKField = 0.00299792458f;
constexpr float kRadialSlack = 0.1f;  // cm: hit radii within this of the layer radius

struct SeedParams {
    BinGrid bg;
    float R[3];
    float w01, w12, kmax, kamb, d0_max, z0_max, dz_max, bz;
    int64_t H;
    const float *hit_pos;
    const int64_t *seg_off;  // [3 E + 1]
    const float4 *bkey;
    const int32_t *bin_off;
    int32_t *trip;
    int64_t cap;
    unsigned long long *count;
};

struct Circle {
    float kappa, d0, orient;
};

__device__ __forceinline__ bool triplet_circle(float x0, float y0, float x1, float y1, float x2, float y2, Circle *c)
{
    const float ax = x1 - x0, ay = y1 - y0, bx = x2 - x1, by = y2 - y1, cx = x2 - x0, cy = y2 - y0;
    const float orient = ax * cy - ay * cx;
    if (orient == 0.0f) return false;
    const float k = 2.0f * orient * rsqrtf((ax * ax + ay * ay) * (bx * bx + by * by)) * rsqrtf(cx * cx + cy * cy);
    const float s0 = x0 * x0 + y0 * y0, s1 = x1 * x1 + y1 * y1, s2 = x2 * x2 + y2 * y2;
    const float inc = x0 * (y1 * s2 - s1 * y2) - y0 * (x1 * s2 - s1 * x2) + s0 * (x1 * y2 - y1 * x2);
    const float F = -inc / orient;
    const float q = fmaf(F * k, k, 1.0f);
    c->kappa = k;
    c->d0 = fabsf(F) * fabsf(k) / (1.0f + sqrtf(fmaxf(q, 0.0f)));
    c->orient = orient;
    return true;
}

// The bins of a window as contiguous key runs: for each z row iz0..iz1 the
// phi bins a0..b0-1, and a1..b1-1 when the window wraps past +-pi (keys are
// stored bin by bin, bin = iz * n_phi + iphi, so each run is one key range).
struct Runs {
    int iz0, iz1, a0, b0, a1, b1;
};

__device__ __forceinline__ Runs window_runs(const BinGrid &bg, float phic, float w, float zlo, float zhi)
{
    Runs r;
    r.iz0 = z_bin(zlo, bg);
    r.iz1 = z_bin(zhi, bg);
    r.a1 = r.b1 = 0;
    if (w >= kPi) {
        r.a0 = 0;
        r.b0 = bg.n_phi;
        return r;
    }
    const float pm = 1e-5f, scale = (float)bg.n_phi * (1.0f / (2.0f * kPi));
    int ip0 = (int)floorf((phic - w - pm + kPi) * scale);
    const int ip1 = (int)floorf((phic + w + pm + kPi) * scale);
    const int nphi = min(ip1 - ip0 + 1, bg.n_phi);
    if (ip0 < 0) ip0 += bg.n_phi;  // phic in [-pi, pi], w < pi: ip0 >= -n_phi
    r.a0 = ip0;
    if (ip0 + nphi <= bg.n_phi) {
        r.b0 = ip0 + nphi;
    } else {
        r.b0 = bg.n_phi;
        r.b1 = ip0 + nphi - bg.n_phi;
    }
    return r;
}

constexpr int kSeedWarps = 4;      // warps per block, one middle-layer hit each at a time
constexpr int kDoubletQueue = 64;  // doublets a warp collects before scanning layer 2 for them

// One warp per hit h1 of the middle layer: the lanes stride over the key runs
// of h1's layer-0 window and queue the doublets passing (a) and (b) in shared
// memory; for each queued doublet the lanes stride over the key runs of its
// layer-2 window and apply (d), (e) and (c).  Triplets are appended with one
// atomic per warp and ballot (a triplet seeded with both charges takes two
// slots); the count keeps growing past the capacity so that the host can
// size a rerun.
__global__ void __launch_bounds__(32 * kSeedWarps) triplet_kernel(const SeedParams p)
{
    __shared__ int32_t queue[kSeedWarps][kDoubletQueue];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int e = blockIdx.y;
    const int64_t lo0 = p.seg_off[3 * e], s1 = p.seg_off[3 * e + 1], lo2 = p.seg_off[3 * e + 2];
    const int n_phi = p.bg.n_phi, nb = n_phi * p.bg.n_z;
    const int32_t *bo0 = p.bin_off + (int64_t)(3 * e) * (nb + 1);
    const int32_t *bo2 = p.bin_off + (int64_t)(3 * e + 2) * (nb + 1);
    const int64_t H = p.H;
    for (int64_t h1 = s1 + (int64_t)blockIdx.x * kSeedWarps + wq; h1 < lo2;
         h1 += (int64_t)gridDim.x * kSeedWarps) {
        const float x1 = p.hit_pos[h1], y1 = p.hit_pos[H + h1], z1 = p.hit_pos[2 * H + h1];
        const float r1 = sqrtf(x1 * x1 + y1 * y1), f1 = atan2f(y1, x1);
        // layer 0: z0 = (z_0 r_1 - z_1 r_0) / (r_1 - r_0) within z0_max, for r_0 near R_0
        float zlo = INFINITY, zhi = -INFINITY;
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
            const float r0 = p.R[0] + sg * kRadialSlack;
            zlo = fminf(zlo, (z1 * r0 - p.z0_max * (r1 - r0)) / r1);
            zhi = fmaxf(zhi, (z1 * r0 + p.z0_max * (r1 - r0)) / r1);
        }
        const float zm = 1e-3f * (1.0f + fabsf(zlo) + fabsf(zhi));
        const Runs w0 = window_runs(p.bg, f1, p.w01, zlo - zm, zhi + zm);
        int nq = 0;  // queued doublets (warp-uniform)

        auto drain = [&]() {
            for (int d = 0; d < nq; ++d) {
                const int64_t h0 = queue[wq][d];
                const float x0 = p.hit_pos[h0], y0 = p.hit_pos[H + h0], z0 = p.hit_pos[2 * H + h0];
                const float r0 = sqrtf(x0 * x0 + y0 * y0);
                const float slope = (z1 - z0) / (r1 - r0);
                const float zaa = fmaf(slope, p.R[2] - kRadialSlack - r1, z1);
                const float zbb = fmaf(slope, p.R[2] + kRadialSlack - r1, z1);
                const float z2lo = fminf(zaa, zbb) - p.dz_max, z2hi = fmaxf(zaa, zbb) + p.dz_max;
                const float zm2 = 1e-3f * (1.0f + fabsf(z2lo) + fabsf(z2hi));
                const Runs w2 = window_runs(p.bg, f1, p.w12, z2lo - zm2, z2hi + zm2);
                for (int iz = w2.iz0; iz <= w2.iz1; ++iz)
                    for (int run = 0; run < 2; ++run) {
                        const int a = run ? w2.a1 : w2.a0, b = run ? w2.b1 : w2.b0;
                        if (a >= b) continue;
                        const int ka = bo2[iz * n_phi + a], kb = bo2[iz * n_phi + b];
                        for (int base = ka; base < kb; base += 32) {
                            const int j = base + lane;
                            bool pass = false;
                            int q = 0, nqq = 0;
                            int32_t h2 = 0;
                            if (j < kb) {
                                const float4 k2 = p.bkey[lo2 + j];
                                if (fabsf(wrap_pi(k2.x - f1)) <= p.w12) {
                                    // the key holds z and r: x and y are read only for a
                                    // candidate within dz_max
                                    const float zp = z1 + (z1 - z0) * (k2.w - r1) / (r1 - r0);
                                    Circle c;
                                    if (fabsf(k2.y - zp) <= p.dz_max) {
                                        h2 = (int32_t)(lo2 + __float_as_int(k2.z));
                                        const float x2 = p.hit_pos[h2], y2 = p.hit_pos[H + h2];
                                        pass = triplet_circle(x0, y0, x1, y1, x2, y2, &c) &&
                                               fabsf(c.kappa) <= p.kmax && c.d0 <= p.d0_max;
                                    }
                                    if (pass) {
                                        q = c.orient * p.bz < 0.0f ? 1 : -1;
                                        nqq = fabsf(c.kappa) <= p.kamb ? 2 : 1;
                                    }
                                }
                            }
                            const unsigned m1 = __ballot_sync(~0u, pass), m2 = __ballot_sync(~0u, nqq == 2);
                            if (m1) {
                                unsigned long long i0 = 0;
                                if (lane == 0)
                                    i0 = atomicAdd(p.count, (unsigned long long)(__popc(m1) + __popc(m2)));
                                i0 = __shfl_sync(~0u, i0, 0) + __popc(m1 & lt) + __popc(m2 & lt);
                                for (int jj = 0; jj < nqq; ++jj) {
                                    const unsigned long long i = i0 + jj;
                                    if (i >= (unsigned long long)p.cap) break;
                                    p.trip[0 * p.cap + i] = e;
                                    p.trip[1 * p.cap + i] = (int32_t)h0;
                                    p.trip[2 * p.cap + i] = (int32_t)h1;
                                    p.trip[3 * p.cap + i] = h2;
                                    p.trip[4 * p.cap + i] = jj == 0 ? q : -q;
                                }
                            }
                        }
                    }
            }
            nq = 0;
            __syncwarp();  // the queue is read before it is refilled
        };

        for (int iz = w0.iz0; iz <= w0.iz1; ++iz)
            for (int run = 0; run < 2; ++run) {
                const int a = run ? w0.a1 : w0.a0, b = run ? w0.b1 : w0.b0;
                if (a >= b) continue;
                const int ka = bo0[iz * n_phi + a], kb = bo0[iz * n_phi + b];
                for (int base = ka; base < kb; base += 32) {
                    const int j = base + lane;
                    bool ok = false;
                    int32_t h0 = 0;
                    if (j < kb) {
                        const float4 k0 = p.bkey[lo0 + j];
                        if (fabsf(wrap_pi(f1 - k0.x)) <= p.w01) {
                            h0 = (int32_t)(lo0 + __float_as_int(k0.z));
                            const float zv = (k0.y * r1 - z1 * k0.w) / (r1 - k0.w);  // key: z_0, r_0
                            ok = fabsf(zv) <= p.z0_max;
                        }
                    }
                    const unsigned m = __ballot_sync(~0u, ok);
                    const int c = __popc(m);
                    if (nq + c > kDoubletQueue) drain();
                    if (ok) queue[wq][nq + __popc(m & lt)] = h0;
                    __syncwarp();
                    nq += c;
                }
            }
        drain();
    }
}

struct FetchParams {
    int64_t n, cap, H;
    float bz, kamb, pt_unres, rel_res, rel_unres;
    const int32_t *trip;
    const float *hit_pos, *hit_cov;
    int32_t *out_event, *out_hits;
    float *out_state, *out_cov;
    int8_t *out_charge;
    float *out_hit_pos, *out_hit_cov;
    uint32_t *out_mask;
};

// The seed fit's inputs of triplet i: the state 1 cm before the first hit
// along the circle's tangent there (so that the fit's first propagation
// reaches layer 0 forwards), pT from the circle (pt_unresolved for a triplet
// seeded with both charges: 1/curvature of a triplet straighter than the hits
// resolve is noise, and a start far above the track's pT leaves the
// linearised fit there), pz from the chord's slope, and a diagonal covariance
// (sigma 10% of each position component, p_sigma_resolved or
// p_sigma_unresolved of each momentum component, floors 1e-4 cm and 1e-3
// GeV); the three hits.
__global__ void __launch_bounds__(256) fetch_kernel(const FetchParams p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int64_t H = p.H, n = p.n;
    const int e = p.trip[i];
    const int32_t h[3] = {p.trip[p.cap + i], p.trip[2 * p.cap + i], p.trip[3 * p.cap + i]};
    const int q = p.trip[4 * p.cap + i];
    float x[3], y[3], z[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        x[l] = p.hit_pos[h[l]];
        y[l] = p.hit_pos[H + h[l]];
        z[l] = p.hit_pos[2 * H + h[l]];
    }
    Circle c;
    if (!triplet_circle(x[0], y[0], x[1], y[1], x[2], y[2], &c)) c.kappa = 0.0f;
    const bool both = fabsf(c.kappa) <= p.kamb;
    const float pt = both ? p.pt_unres : kKField * fabsf(p.bz) / fabsf(c.kappa);
    const float ka = both ? kKField * fabsf(p.bz) / p.pt_unres : fabsf(c.kappa);
    const float ax = x[1] - x[0], ay = y[1] - y[0], alen = sqrtf(ax * ax + ay * ay);
    // turning sense of charge q: counter-clockwise (+1) when q Bz < 0
    const float turn = (float)q * p.bz < 0.0f ? 1.0f : -1.0f;
    const float half = asinf(fminf(1.0f, 0.5f * alen * ka)) * turn;  // half the turning angle over the chord
    float sh, ch;
    sincosf(-half, &sh, &ch);
    const float cx = ax / alen, cy = ay / alen;
    const float tx = ch * cx - sh * cy, ty = sh * cx + ch * cy;
    const float tanl = (z[1] - z[0]) / alen;
    const float st[6] = {x[0] - tx, y[0] - ty, z[0] - tanl, pt * tx, pt * ty, pt * tanl};
    const float rel_p = both ? p.rel_unres : p.rel_res;
#pragma unroll
    for (int k = 0; k < 6; ++k) p.out_state[k * n + i] = st[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) p.out_cov[k * n + i] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float rel = k < 3 ? 0.1f : rel_p, fl = k < 3 ? 1e-4f : 1e-3f;
        p.out_cov[(k * (k + 1) / 2 + k) * n + i] = rel * rel * st[k] * st[k] + fl * fl;
    }
    p.out_charge[i] = (int8_t)q;
    p.out_event[i] = e;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        p.out_hits[l * n + i] = h[l];
        p.out_hit_pos[(l * 3 + 0) * n + i] = x[l];
        p.out_hit_pos[(l * 3 + 1) * n + i] = y[l];
        p.out_hit_pos[(l * 3 + 2) * n + i] = z[l];
#pragma unroll
        for (int k = 0; k < 6; ++k) p.out_hit_cov[(l * 6 + k) * n + i] = p.hit_cov[k * H + h[l]];
    }
    p.out_mask[i] = 7u;
}

float dphi_window(float ra, float rb, float rmin, float d0_max)
{
    return asinf(std::min(1.0f, rb / (2.0f * rmin))) - asinf(std::min(1.0f, ra / (2.0f * rmin))) +
           d0_max * (1.0f / ra + 1.0f / rb);
}

}  // namespace
}  // namespace kf

using namespace kf;

extern "C" void kf_seeding_default(kf_seeding *s)
{
    if (!s) return;
    s->pt_min = 0.3f;
    s->d0_max = 0.15f;
    s->z0_max = 4.0f;
    s->dz_max = 0.8f;
    s->pt_both_charges = 2.0f;
    s->pt_unresolved = 6.0f;
    s->p_sigma_resolved = 0.3f;
    s->p_sigma_unresolved = 1.0f;
    s->n_phi_bins = 256;
    s->n_z_bins = 64;
}

extern "C" int kf_seed_triplets(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
                                const float *hit_pos, int64_t n_hits, const kf_seeding *opt, int64_t *n_seeds,
                                kf_stream stream_)
{
    if (!ctx || !n_seeds) return KF_ERR_ARG;
    kf_seeding o;
    if (opt) o = *opt;
    else kf_seeding_default(&o);
    int rc;
    FitGeom g;
    if ((rc = check_geometry(ctx, geom, &g))) return rc;
    if (g.L != 3) return set_error(ctx, KF_ERR_ARG, "seeding needs the three seed layers (got %d)", g.L);
    if (!(o.pt_min > 0.0f) || !(o.d0_max >= 0.0f) || !(o.z0_max >= 0.0f) || !(o.dz_max >= 0.0f) ||
        !(o.pt_both_charges > 0.0f))
        return set_error(ctx, KF_ERR_ARG, "seeding cuts: pt_min > 0, d0_max, z0_max, dz_max >= 0, pt_both_charges > 0");
    if (o.n_phi_bins < 1 || o.n_z_bins < 1 || (int64_t)o.n_phi_bins * o.n_z_bins > 16384)
        return set_error(ctx, KF_ERR_ARG, "n_phi_bins x n_z_bins must be 1..16384");
    if (!(g.qk != 0.0f)) return set_error(ctx, KF_ERR_ARG, "seeding needs a magnetic field");
    if (n_events < 0 || n_hits < 0 || n_hits >= (int64_t(1) << 31))
        return set_error(ctx, KF_ERR_ARG, "n_events must be >= 0 and n_hits < 2^31");
    *n_seeds = 0;
    SeedState *&st = context_seed_state(ctx);
    if (!st) st = new SeedState;
    st->n = 0;
    if (n_events == 0) return KF_OK;
    if (!hit_offsets) return set_error(ctx, KF_ERR_ARG, "hit_offsets is NULL");
    int max_l1 = 0;
    for (int e = 0; e < n_events; ++e) {
        const int64_t *r = hit_offsets + (int64_t)e * 4;
        if (e > 0 && r[0] != hit_offsets[(int64_t)(e - 1) * 4 + 3])
            return set_error(ctx, KF_ERR_ARG, "events must be stored back to back (event %d)", e);
        for (int l = 0; l < 3; ++l)
            if (r[l] < 0 || r[l + 1] < r[l] || r[l + 1] > n_hits)
                return set_error(ctx, KF_ERR_ARG, "hit_offsets row %d is not a non-decreasing run within n_hits", e);
        max_l1 = std::max<int>(max_l1, (int)(r[2] - r[1]));
    }
    if (n_hits > 0 && (rc = check_ptr(ctx, hit_pos, 4, "hit_pos"))) return rc;
    DeviceGuard dg(context_device(ctx));
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const int nb = o.n_phi_bins * o.n_z_bins;
    const size_t n_seg = (size_t)n_events * 3;
    auto grow = [&](void **ptr, size_t &cap, size_t need, size_t elem) -> bool {
        if (need <= cap) return true;
        cudaFree(*ptr);
        *ptr = nullptr;
        cap = 0;
        if (cudaMalloc(ptr, std::max<size_t>(need, 1) * elem) != cudaSuccess) return false;
        cap = need;
        return true;
    };
    bool ok = grow((void **)&st->bkey, st->key_cap, (size_t)n_hits, sizeof(float4)) &&
              grow((void **)&st->bin_off, st->bin_cap, n_seg * (nb + 1), sizeof(int32_t)) &&
              grow((void **)&st->hit_rank, st->rank_cap, (size_t)n_hits, sizeof(int32_t)) &&
              grow((void **)&st->seg_off, st->seg_cap, n_seg + 1, sizeof(int64_t));
    if (ok && !st->count) ok = cudaMalloc(&st->count, sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) return set_error(ctx, KF_ERR_NOMEM, "could not allocate the seeding scratch");
    std::vector<int64_t> seg(n_seg + 1);
    for (int e = 0; e < n_events; ++e)
        for (int l = 0; l < 3; ++l) seg[(size_t)e * 3 + l] = hit_offsets[(int64_t)e * 4 + l];
    seg[n_seg] = hit_offsets[(int64_t)(n_events - 1) * 4 + 3];
    cudaError_t e = cudaMemcpyAsync(st->seg_off, seg.data(), (n_seg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                    stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // the host vector must outlive the copy
    if (e != cudaSuccess) return cuda_error(ctx, e, "seeding offsets copy");
    BinGrid bg{o.n_phi_bins, o.n_z_bins, g.z_half};
    int64_t max_seg = 0;
    for (size_t i = 0; i < n_seg; ++i) max_seg = std::max<int64_t>(max_seg, seg[i + 1] - seg[i]);
    if ((e = bin_hits(st->seg_off, (int64_t)n_seg, max_seg, hit_pos, n_hits, bg, st->bkey, st->bin_off, st->hit_rank,
                      context_sm_count(ctx), stream)) != cudaSuccess)
        return cuda_error(ctx, e, "seeding binning");

    SeedParams p;
    p.bg = bg;
    for (int l = 0; l < 3; ++l) p.R[l] = g.r[l];
    const float bz = g.qk / kKField;
    const float rmin = o.pt_min / (kKField * fabsf(bz));
    p.w01 = dphi_window(p.R[0], p.R[1], rmin, o.d0_max);
    p.w12 = dphi_window(p.R[1], p.R[2], rmin, o.d0_max);
    p.kmax = kKField * fabsf(bz) / o.pt_min;
    p.kamb = kKField * fabsf(bz) / o.pt_both_charges;
    p.d0_max = o.d0_max;
    p.z0_max = o.z0_max;
    p.dz_max = o.dz_max;
    p.bz = bz;
    p.H = n_hits;
    p.hit_pos = hit_pos;
    p.seg_off = st->seg_off;
    p.bkey = st->bkey;
    p.bin_off = st->bin_off;
    p.count = st->count;
    if (st->trip_cap == 0) {
        const int64_t want = std::max<int64_t>(1 << 16, 4 * (int64_t)n_hits);
        if (cudaMalloc(&st->trip, (size_t)want * 5 * sizeof(int32_t)) != cudaSuccess)
            return set_error(ctx, KF_ERR_NOMEM, "could not allocate the triplet buffer");
        st->trip_cap = want;
    }
    for (int pass = 0; pass < 2; ++pass) {
        p.trip = st->trip;
        p.cap = st->trip_cap;
        if ((e = cudaMemsetAsync(st->count, 0, sizeof(unsigned long long), stream)) != cudaSuccess)
            return cuda_error(ctx, e, "seeding counter");
        if (max_l1 > 0) {
            const dim3 grid((unsigned)((max_l1 + kSeedWarps - 1) / kSeedWarps), (unsigned)n_events);
            triplet_kernel<<<grid, 32 * kSeedWarps, 0, stream>>>(p);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(ctx, e, "triplet search");
        }
        unsigned long long cnt = 0;
        e = cudaMemcpyAsync(&cnt, st->count, sizeof cnt, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_error(ctx, e, "triplet count");
        if ((int64_t)cnt <= st->trip_cap) {
            st->n = (int64_t)cnt;
            st->n_hits = n_hits;
            *n_seeds = (int64_t)cnt;
            return KF_OK;
        }
        cudaFree(st->trip);
        st->trip = nullptr;
        st->trip_cap = 0;
        const int64_t want = (int64_t)cnt + (int64_t)cnt / 4;
        if (cudaMalloc(&st->trip, (size_t)want * 5 * sizeof(int32_t)) != cudaSuccess)
            return set_error(ctx, KF_ERR_NOMEM, "could not allocate %lld triplets", (long long)want);
        st->trip_cap = want;
    }
    return set_error(ctx, KF_ERR_CUDA, "triplet count changed between passes");
}

extern "C" int kf_seed_fetch(kf_context *ctx, const kf_geometry *geom, const float *hit_pos, const float *hit_cov,
                             const kf_seeding *opt, int64_t n, int32_t *out_event, int32_t *out_hits,
                             float *out_state, float *out_cov, int8_t *out_charge, float *out_hit_pos,
                             float *out_hit_cov, uint32_t *out_mask, kf_stream stream_)
{
    if (!ctx) return KF_ERR_ARG;
    kf_seeding o;
    if (opt) o = *opt;
    else kf_seeding_default(&o);
    if (!(o.pt_both_charges > 0.0f) || !(o.pt_unresolved > 0.0f) || !(o.p_sigma_resolved >= 0.0f) ||
        !(o.p_sigma_unresolved >= 0.0f))
        return set_error(ctx, KF_ERR_ARG, "seed start: pt_both_charges, pt_unresolved > 0, momentum sigmas >= 0");
    int rc;
    FitGeom g;
    if ((rc = check_geometry(ctx, geom, &g))) return rc;
    SeedState *st = context_seed_state(ctx);
    const int64_t have = st ? st->n : 0;
    if (n < 0 || n > have)
        return set_error(ctx, KF_ERR_ARG, "n = %lld but the last search found %lld", (long long)n, (long long)have);
    if (n == 0) return KF_OK;
    if ((rc = check_ptr(ctx, hit_pos, 4, "hit_pos")) || (rc = check_ptr(ctx, hit_cov, 4, "hit_cov")) ||
        (rc = check_ptr(ctx, out_event, 4, "out_event")) || (rc = check_ptr(ctx, out_hits, 4, "out_hits")) ||
        (rc = check_ptr(ctx, out_state, 4, "out_state")) || (rc = check_ptr(ctx, out_cov, 4, "out_cov")) ||
        (rc = check_ptr(ctx, out_charge, 1, "out_charge")) || (rc = check_ptr(ctx, out_hit_pos, 4, "out_hit_pos")) ||
        (rc = check_ptr(ctx, out_hit_cov, 4, "out_hit_cov")) || (rc = check_ptr(ctx, out_mask, 4, "out_mask")))
        return rc;
    DeviceGuard dg(context_device(ctx));
    const float bz = g.qk / kKField;
    FetchParams p{n, st->trip_cap, st->n_hits, bz, kKField * fabsf(bz) / o.pt_both_charges, o.pt_unresolved,
                  o.p_sigma_resolved, o.p_sigma_unresolved, st->trip, hit_pos, hit_cov, out_event, out_hits,
                  out_state, out_cov, out_charge, out_hit_pos, out_hit_cov, out_mask};
    fetch_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream_)>>>(p);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : cuda_error(ctx, e, "seed fetch");
}
