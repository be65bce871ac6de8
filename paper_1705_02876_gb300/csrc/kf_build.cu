// Combinatorial track building on sm_103a (Sections 3, 3.1 and 4.3):
//   bin_hits          - counting sort of every (event, layer)'s hits into
//                       phi x z bins (Section 3: hits partitioned spatially
//                       for a fast look-up of the compatible ones), a
//                       shared-memory count per segment and a scatter over
//                       all segments (kf_bins.cuh);
//   build_kernel      - the clone engine, all layers in one launch: each
//                       seed's candidates occupy a group of G >= N lanes of
//                       a warp (G in 1, 2, 4, 6, 8); every lane propagates
//                       its candidate, scans the bins its window overlaps
//                       and keeps its N best compatible hits; the group
//                       merges its lanes' lists into the N best children by
//                       warp shuffles (in place of the paper's shared-memory
//                       heaps, Section 4.3) and each lane takes over one
//                       child and updates it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "kf.h"
#include "kf_api_internal.h"
#include "kf_fit.cuh"
#include "kf_bins.cuh"
#include "kf_mlp.cuh"

namespace kf {

struct BuildState {
    size_t hit_capacity = 0, bin_capacity = 0, seg_capacity = 0, rank_capacity = 0;
    float4 *bkey = nullptr;  // binned hits: (phi, z, index within the segment as bits, radius)
    int32_t *bin_off = nullptr;
    int32_t *hit_rank = nullptr;  // the binning's rank of each hit within its bin
    int64_t *seg_off = nullptr;  // device copy of the segment bounds [n_seg + 1]
    int64_t *ev_off = nullptr;   // device copy of hit_offsets [n_events][L + 1]
    size_t ev_capacity = 0;
    // the host-buffer build's pipeline: streams, and per ring slot the batch's device buffers,
    // its pinned offset staging and the events that order the slot's reuse
    cudaStream_t hs_in = nullptr, hs_run = nullptr, hs_out = nullptr;
    struct Slot {
        char *dev = nullptr;
        size_t dev_bytes = 0;
        int64_t *pin = nullptr;  // pinned: segment bounds, then the batch's offsets rows
        size_t pin_elems = 0;
        cudaEvent_t in_done = nullptr, built = nullptr, out_done = nullptr;
        bool used = false;
    } slot[3];
    // autotuned shapes: (L, N, mode, seeds' size class, hits' size class, fixed n_phi, fixed n_z,
    // fixed form of the learned build)
    // -> (n_phi, n_z, speculative: the learned build as a flagging plain pass plus a proposal pass)
    std::map<std::tuple<int, int, int, int, int, int, int, int>, std::tuple<int, int, int>> tuned;
    // the speculative learned build's per-seed flags, flagged-seed list and its length
    int32_t *seed_flag = nullptr, *seed_list = nullptr;
    unsigned *list_count = nullptr;
    size_t flag_capacity = 0, list_capacity = 0, count_capacity = 0;
};

void destroy_build_state(BuildState *s)
{
    if (!s) return;
    for (auto &sl : s->slot) {
        cudaFree(sl.dev);
        cudaFreeHost(sl.pin);
        if (sl.in_done) cudaEventDestroy(sl.in_done);
        if (sl.built) cudaEventDestroy(sl.built);
        if (sl.out_done) cudaEventDestroy(sl.out_done);
    }
    for (cudaStream_t h : {s->hs_in, s->hs_run, s->hs_out})
        if (h) cudaStreamDestroy(h);
    cudaFree(s->bkey);
    cudaFree(s->bin_off);
    cudaFree(s->hit_rank);
    cudaFree(s->seg_off);
    cudaFree(s->ev_off);
    cudaFree(s->seed_flag);
    cudaFree(s->seed_list);
    cudaFree(s->list_count);
    delete s;
}

namespace {

constexpr int kModePlain = 0, kModeLog = 1, kModeProposal = 2;
constexpr int kKeyBatch = 4;  // window keys loaded together in the collecting scan (8 was slower)

struct BuildParams {
    FitGeom g;
    Routing rt;
    BinGrid bg;
    int N;
    float chi2_cut, nsigma, sig_rphi2, sig_z2, max_dphi, max_dz;
    int64_t S, H;
    int n_events;
    int event_base;    // seed_event values are event_base + the event's index in ev_off
    int64_t hit_base;  // added to the written hit indices (ev_off holds batch-local offsets)
    const int64_t *ev_off;  // [E][L + 1]
    const float *hit_pos, *hit_cov;
    const float4 *bkey;
    const int32_t *bin_off;
    const int32_t *seed_event;
    const float *seed_state, *seed_cov;
    const int8_t *seed_charge;
    int32_t *out_hit;
    float *out_chi2;
    int16_t *out_nhits;
    float *out_state, *out_cov;
    uint32_t *out_flags;
    // training log of the plain build (null when off)
    float *log_f, *log_y;
    int32_t *log_ref;
    unsigned long long *log_n;
    unsigned long long log_cap;
    // learned proposal
    int topk;
    const __nv_bfloat16 *mlp_W1, *mlp_W2;
    const float *mlp_w32;
    // the learned build in two passes: the plain pass flags (flag_over > 0)
    // every seed one of whose windows held more than flag_over hits; the
    // proposal pass builds only the seeds of seed_list (*list_count of them)
    int flag_over;
    int32_t *seed_flag;
    const int32_t *seed_list;
    const unsigned *list_count;
};

constexpr int kMaxN = 8;
constexpr uint32_t kNoKey = 0xffffffffu;

// Chi2 increment of a hit (m, packed V) against the predicted candidate, in
// the layer's local frame (n, t, z) with the radial row of C projected out
// (the same arithmetic as the update): ctt = C_tt, ctz = C_tz, czz = C_zz.
// f3 receives the residual in that frame divided by the square roots of S's
// diagonal (the proposal's first three inputs).
__device__ __forceinline__ bool hit_eval(const float x[3], float nx, float ny, float ctt, float ctz, float czz,
                                         const float m[3], const float v[6], float *out, float f3[3])
{
    const float vnn = fmaf(nx * nx, v[0], fmaf(2.0f * nx * ny, v[1], ny * ny * v[2]));
    const float vnt = fmaf(nx * ny, v[2] - v[0], (nx * nx - ny * ny) * v[1]);
    const float vtt = fmaf(ny * ny, v[0], fmaf(-2.0f * nx * ny, v[1], nx * nx * v[2]));
    const float vnz = fmaf(nx, v[3], ny * v[4]), vtz = fmaf(nx, v[4], -ny * v[3]);
    const float a = vnn, b = vnt, cc = ctt + vtt, d = vnz, e = ctz + vtz, f = czz + v[5];
    const float i00 = cc * f - e * e, i10 = d * e - b * f, i11 = a * f - d * d;
    const float i20 = b * e - cc * d, i21 = b * d - a * e, i22 = a * cc - b * b;
    const float det = fmaf(a, i00, fmaf(b, i10, d * i20));
    const float d0 = m[0] - x[0], d1 = m[1] - x[1];
    const float rn = fmaf(nx, d0, ny * d1), rt = fmaf(nx, d1, -ny * d0), rz = m[2] - x[2];
    f3[0] = rn * rsqrtf(fmaxf(a, 1e-30f));
    f3[1] = rt * rsqrtf(fmaxf(cc, 1e-30f));
    f3[2] = rz * rsqrtf(fmaxf(f, 1e-30f));
    if (!(a > 0.0f && i22 > 0.0f && det > 0.0f)) return false;
    const float q0 = fmaf(i00, rn, fmaf(i10, rt, i20 * rz));
    const float q1 = fmaf(i10, rn, fmaf(i11, rt, i21 * rz));
    const float q2 = fmaf(i20, rn, fmaf(i21, rt, i22 * rz));
    *out = __fdividef(fmaf(rn, q0, fmaf(rt, q1, rz * q2)), det);
    return true;
}

// The window of a candidate at the predicted crossing and the bins it overlaps.
struct Window {
    float phic, dphi, z, dz;
    int iz0, iz1, ip0, nphi;
    const int32_t *bo;
    int64_t seg_lo;
};

// Resumable walk over the in-window hits of a candidate: next() returns the
// next hit's index within its (event, layer), or kNoKey at the end.
struct WindowCursor {
    int iz, k, hb, h1;
    __device__ __forceinline__ void start(const Window &w)
    {
        iz = w.iz0;
        k = -1;
        hb = h1 = 0;
    }
    __device__ __forceinline__ uint32_t next(const BuildParams &p, const Window &w)
    {
        for (;;) {
            while (hb < h1) {
                const int64_t q = w.seg_lo + hb++;
                const float4 k = p.bkey[q];
                if (fabsf(wrap_pi(k.x - w.phic)) <= w.dphi && fabsf(k.y - w.z) <= w.dz)
                    return (uint32_t)__float_as_int(k.z);
            }
            if (iz > w.iz1) return kNoKey;
            if (++k >= w.nphi) {
                k = 0;
                if (++iz > w.iz1) return kNoKey;
            }
            int ip = w.ip0 + k;
            ip = ip < 0 ? ip + p.bg.n_phi : (ip >= p.bg.n_phi ? ip - p.bg.n_phi : ip);
            const int b = iz * p.bg.n_phi + ip;
            hb = w.bo[b];
            h1 = w.bo[b + 1];
        }
    }
};


// Shared memory: back-pointers [L][128], update slots [kSlotSize][128], then
// (proposal only) the parking columns [kWcWords][128] and each warp's 32
// staged input rows (FP32, kStageLd floats each).
constexpr int kStageLd = 12;
__host__ __device__ constexpr size_t build_smem_base(int L) { return ((size_t)(L + kSlotSize) * 128 * 4 + 127) / 128 * 128; }

// Proposal mode: where a lane parks, in shared memory, what walking the wide
// windows needs ([kWcWords][128] words, one column per thread; the candidate
// state x, C goes to the thread's update slot, idle at that point).  While
// the warp walks the wide windows the candidate state is out of the
// registers, so that the scoring's fragments do not spill it.
constexpr int kWcHb = 0;                        // [kMaxN] collected (or ranked) hits
constexpr int kWcNx = 8, kWcNy = 9, kWcCtt = 10, kWcCtz = 11, kWcCzz = 12;
constexpr int kWcSegLo = 13;                    // 2 words
constexpr int kWcBo = 15;                       // 2 words
constexpr int kWcPhic = 17, kWcDphi = 18, kWcZ = 19, kWcDz = 20;
constexpr int kWcIz0 = 21, kWcIz1 = 22, kWcIp0 = 23, kWcNphi = 24;
constexpr int kWcNhits = 25, kWcQkb = 26;      // the candidate's hit count, its charge x field term
constexpr int kWcWords = 27;
constexpr size_t kBuildSmemMlp = (size_t)(kWcWords * 128 + 4 * 32 * kStageLd) * sizeof(float);

// What scan_wide reads besides the parked columns.
struct WideArgs {
    const float4 *bkey;
    const float *hit_pos, *hit_cov;
    int64_t H;
    int n_phi, topk, l, L;
    const __nv_bfloat16 *W1, *W2;
    const float *w32;
};

// The windows of one warp wider than topk, walked by the whole warp
// (warp-collective: every lane calls it, converged; every lane has parked its
// columns).  Each wide lane walks its own window, and the warp's other lanes
// join the wide lanes as helpers, spread evenly: an owner served by R lanes
// has its window's key sequence (each z row's key runs, in order) split by
// position modulo R, so that every key is visited once.  Each round every
// lane advances to its next in-window hit and the warp scores the round's 32
// rows together on the tensor cores (weights read through L1); a wide lane
// keeps its own pairs in its top-k list, (logit desc, hit index asc), and a
// helper's pair goes to its owner by shuffle only if it beats the owner's
// current topk-th entry.  The owner's list is written back to its hit
// column.  Few wide lanes with long windows take about one round per 32 keys;
// many wide lanes take about one round per hit of the longest window.  The
// proposal's candidate inputs are computed here from the owner's parked
// state, as the kernel computes them: log10 of the covariance diagonal,
// q/pT, the layer's fraction l / L and the layers missed so far.
__device__ __forceinline__ void scan_wide(const WideArgs p, bool wide, const float *slots_w, float *wc_w, float *xs)
{
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wbase = threadIdx.x - lane;
    const unsigned wmask = __ballot_sync(kAll, wide);
    const int W = __popc(wmask), nh = 32 - W;
    // this lane's owner, its position among the owner's R serving lanes
    int oi, sub;
    if (wide) {
        oi = __popc(wmask & ((1u << lane) - 1u));
        sub = 0;
    } else {
        const int h = __popc(~wmask & ((1u << lane) - 1u));
        oi = h % W;
        sub = 1 + h / W;
    }
    unsigned om = wmask;
    for (int i = 0; i < oi; ++i) om &= om - 1u;
    const int owner = __ffs(om) - 1;
    const int R = 1 + (oi < nh ? (nh - oi + W - 1) / W : 0);
    volatile const float *oc = wc_w + wbase + owner;
    volatile const float *os = slots_w + wbase + owner;
    auto col = [&](int f) { return oc[f * 128]; };
    auto icol = [&](int f) { return __float_as_int(oc[f * 128]); };
    // the owner's candidate inputs, staged once in this lane's row
    {
        float *row = xs + lane * kStageLd;
#pragma unroll
        for (int i = 0; i < 6; ++i) row[3 + i] = log10f(fmaxf(os[(kSlotC + pk(i, i)) * 128], 1e-30f));
        const float px3 = os[(kSlotX + 3) * 128], px4 = os[(kSlotX + 4) * 128];
        row[9] = copysignf(rsqrtf(px3 * px3 + px4 * px4), col(kWcQkb));
        row[10] = __fdiv_rn((float)p.l, (float)p.L);  // correctly rounded, whatever the division flags
        row[11] = (float)(p.l - icol(kWcNhits));
    }
    // the owner's key runs: z rows iz0..iz1, each one contiguous run of bins
    // (two past the wrap at +-pi), run index ri = 2 (iz - iz0) + r
    const int nphi = p.n_phi;
    const int ip0 = icol(kWcIp0), iz0 = icol(kWcIz0), iz1 = icol(kWcIz1);
    const int a0 = ip0 < 0 ? ip0 + nphi : (ip0 >= nphi ? ip0 - nphi : ip0);
    const int e0 = a0 + icol(kWcNphi);
    const int b0 = min(e0, nphi), b1 = e0 > nphi ? e0 - nphi : 0;
    const int32_t *bo = reinterpret_cast<const int32_t *>(((unsigned long long)(uint32_t)icol(kWcBo + 1) << 32) |
                                                          (uint32_t)icol(kWcBo));
    const int64_t seg_lo =
        (int64_t)(((unsigned long long)(uint32_t)icol(kWcSegLo + 1) << 32) | (uint32_t)icol(kWcSegLo));
    // q: the next key to visit; while q >= kb, q - kb keys remain to skip past
    // the current run's end
    int ri = -1, q = sub, kb = 0;
    auto next_hit = [&]() -> uint32_t {
        for (;;) {
            while (q >= kb) {
                const int over = q - kb;
                ++ri;
                const int iz = iz0 + (ri >> 1);
                if (iz > iz1) {
                    q = kb = 0;
                    return kNoKey;
                }
                const int r = ri & 1;
                const int ra = r ? 0 : a0, rb = r ? b1 : b0;
                if (ra >= rb) {
                    q = over;
                    kb = 0;
                    continue;
                }
                const int32_t *rowp = bo + iz * nphi;
                const int ka = rowp[ra];
                kb = rowp[rb];
                q = ka + over;
            }
            const float4 k = p.bkey[seg_lo + q];
            q += R;
            if (fabsf(wrap_pi(k.x - col(kWcPhic))) <= col(kWcDphi) && fabsf(k.y - col(kWcZ)) <= col(kWcDz))
                return (uint32_t)__float_as_int(k.z);
        }
    };
    float tz[kMaxN];
    uint32_t hk[kMaxN];
#pragma unroll
    for (int k = 0; k < kMaxN; ++k) {
        tz[k] = -INFINITY;
        hk[k] = kNoKey;
    }
    auto insert_top = [&](float cv, uint32_t hv) {
#pragma unroll
        for (int k2 = 0; k2 < kMaxN; ++k2) {
            const bool before = k2 < p.topk && (cv > tz[k2] || (cv == tz[k2] && hv < hk[k2]));
            const float t1 = tz[k2];
            const uint32_t t2 = hk[k2];
            tz[k2] = before ? cv : t1;
            hk[k2] = before ? hv : t2;
            cv = before ? t1 : cv;
            hv = before ? t2 : hv;
        }
    };
    bool more = true;
    while (__any_sync(kAll, more)) {
        const uint32_t hl = more ? next_hit() : kNoKey;
        more = hl != kNoKey;
        float f3[3] = {0.0f, 0.0f, 0.0f};
        if (more) {
            float m[3], v[6], dc;
            const int64_t hg = seg_lo + hl;
#pragma unroll
            for (int i = 0; i < 3; ++i) m[i] = p.hit_pos[i * p.H + hg];
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = p.hit_cov[i * p.H + hg];
            const float xp[3] = {os[(kSlotX + 0) * 128], os[(kSlotX + 1) * 128], os[(kSlotX + 2) * 128]};
            hit_eval(xp, col(kWcNx), col(kWcNy), col(kWcCtt), col(kWcCtz), col(kWcCzz), m, v, &dc, f3);
        }
        __syncwarp();  // the previous round's rows are read
#pragma unroll
        for (int i = 0; i < 3; ++i) xs[lane * kStageLd + i] = f3[i];
        const MlpWeightsRef mw{reinterpret_cast<const uint32_t *>(p.W1), reinterpret_cast<const uint32_t *>(p.W2),
                               p.w32 + kOffB1, p.w32 + kOffB2, p.w32 + kOffW3, p.w32[kOffB3]};
        const float z = mlp_score_warp_split(mw, xs, kStageLd);
        if (more && wide) insert_top(z, hl);
        // a helper's pair goes to its owner if it beats the owner's topk-th
        float tl = -INFINITY;
        uint32_t th = kNoKey;
#pragma unroll
        for (int k = 0; k < kMaxN; ++k)
            if (k == p.topk - 1) {
                tl = tz[k];
                th = hk[k];
            }
        tl = __shfl_sync(kAll, tl, owner);
        th = __shfl_sync(kAll, th, owner);
        const bool offer = more && !wide && (z > tl || (z == tl && hl < th));
        for (unsigned mo = __ballot_sync(kAll, offer); mo; mo &= mo - 1u) {
            const int j = __ffs(mo) - 1;
            const float cv = __shfl_sync(kAll, z, j);
            const uint32_t hv = __shfl_sync(kAll, hl, j);
            const int oj = __shfl_sync(kAll, owner, j);
            if (lane == oj) insert_top(cv, hv);
        }
    }
    if (wide) {
        volatile float *mine = wc_w + threadIdx.x;
#pragma unroll
        for (int k = 0; k < kMaxN; ++k) mine[(kWcHb + k) * 128] = __int_as_float((int)hk[k]);
    }
    __syncwarp();
}

// The seeds the plain pass flagged, appended to list in no fixed order.
__global__ void flagged_seeds_kernel(const int32_t *flag, int64_t S, int32_t *list, unsigned *count)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
        if (flag[s]) list[atomicAdd(count, 1u)] = (int32_t)s;
}

// At most 128 registers (four blocks per SM) in every mode.
template <int G, int MODE>
__global__ void __launch_bounds__(128, 4) build_kernel(const BuildParams p)
{
    constexpr int SEEDS_PER_WARP = 32 / G;
    // a lane's child list (it gives at most N <= kMaxN hit children) and the
    // first scan's buffer: kMaxN entries each (lists sized to G measured no
    // faster: their shorter loops cost the plain kernel spills at 128 registers)
    constexpr int NL = kMaxN, HB = kMaxN;
    extern __shared__ __align__(128) int32_t smem[];
    const int L = p.g.L;
    int32_t *bp = smem;                                   // [L][128] back-pointers
    float *slots = reinterpret_cast<float *>(smem + L * 128);  // [kSlotSize][128]
    // (proposal only) this thread's parking columns [kWcWords][128] and this
    // warp's staged input rows [32][kStageLd]
    float *wc = nullptr, *xs = nullptr;
    if (MODE == kModeProposal) {
        wc = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(smem) + build_smem_base(L));
        xs = wc + kWcWords * 128 + (threadIdx.x >> 5) * 32 * kStageLd;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = lane % G, gbase = lane - slot;
    // G = 6: five groups per warp; lanes 30 and 31 form an idle group of two
    const bool lane_ok = lane < SEEDS_PER_WARP * G;
    const int64_t k_seed = ((int64_t)blockIdx.x * 4 + warp) * SEEDS_PER_WARP + lane / G;
    int64_t s = k_seed;
    bool seed_ok = lane_ok && k_seed < p.S;
    if (p.seed_list) {  // the listed seeds only; a warp without one has nothing to do
        seed_ok = lane_ok && k_seed < (int64_t)*p.list_count;
        s = seed_ok ? p.seed_list[k_seed] : 0;
        if (!__any_sync(0xffffffffu, seed_ok)) return;
    }
    const int N = p.N;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);

    float x[6], c[21];
    float chi2 = 0.0f;
    int nhits = 0;
    bool stopped = false;
    uint32_t flags = 0;
    bool over = false;  // a window of this lane's candidates held more than flag_over hits
    int nc = 1;
    const int ev_in = seed_ok ? p.seed_event[s] - p.event_base : 0;
    const bool ev_ok = ev_in >= 0 && ev_in < p.n_events;  // a seed of an unknown event builds nothing
    const int ev = ev_ok ? ev_in : 0;
    const float qkb = seed_ok ? (float)p.seed_charge[s] * p.g.qk : 0.0f;
    if (seed_ok && ev_ok) {
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = p.seed_state[i * p.S + s];
#pragma unroll
        for (int i = 0; i < 21; ++i) c[i] = p.seed_cov[i * p.S + s];
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 21; ++i) c[i] = 0.0f;
        nc = 0;
    }
    const int nbins = p.bg.n_phi * p.bg.n_z;
    for (int l = 0; l < L; ++l) {
        const bool valid = slot < nc;
        bool reached = false;
        if (valid && !stopped) {
            float xn[6], sd;
            Jac J;
            if (!propagate(x, qkb, p.g.r[l], xn, sd, &J)) {
                stopped = true;
                flags |= KF_FLAG_UNREACHABLE;
            } else if (fabsf(xn[2]) > p.g.z_half) {
                stopped = true;
                flags |= KF_FLAG_LEFT_BARREL;
            } else {
                transport(J, c);
                add_scattering(xn, p.g.inv_r[l], p.g.xx0[l], c);
#pragma unroll
                for (int i = 0; i < 6; ++i) x[i] = xn[i];
                reached = true;
            }
        }
        // this candidate's best compatible hits, sorted by (chi2, hit index);
        // lr = each entry's row in the training log (logging only)
        float lc[NL];
        uint32_t lh[NL], lr[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            lc[k] = INFINITY;
            lh[k] = kNoKey;
            lr[k] = kNoKey;
        }
        auto insert = [&](float dc, uint32_t hl, uint32_t row) {
            if (!(dc < lc[NL - 1] || (dc == lc[NL - 1] && hl < lh[NL - 1]))) return;
            float cv = dc;
            uint32_t hv = hl, rv = row;
#pragma unroll
            for (int k2 = 0; k2 < NL; ++k2) {
                const bool before = cv < lc[k2] || (cv == lc[k2] && hv < lh[k2]);
                const float tc = lc[k2];
                const uint32_t th = lh[k2], tr = lr[k2];
                lc[k2] = before ? cv : tc;
                lh[k2] = before ? hv : th;
                lr[k2] = before ? rv : tr;
                cv = before ? tc : cv;
                hv = before ? th : hv;
                rv = before ? tr : rv;
            }
        };
        const int64_t seg = (int64_t)ev * (L + 1) + l;
        int64_t seg_lo = seed_ok ? p.ev_off[seg] : 0;
        Window win{};
        float nx = 0.0f, ny = 0.0f, ctt = 0.0f, ctz = 0.0f, czz = 0.0f;
        if (reached) {
            const float ir = rsqrtf(x[0] * x[0] + x[1] * x[1]);
            nx = x[0] * ir;
            ny = x[1] * ir;
            ctt = fmaf(ny * ny, c[pk(0, 0)], fmaf(-2.0f * nx * ny, c[pk(1, 0)], nx * nx * c[pk(1, 1)]));
            ctz = fmaf(nx, c[pk(2, 1)], -ny * c[pk(2, 0)]);
            czz = c[pk(2, 2)];
            win.dphi = fminf(p.nsigma * sqrtf(ctt + p.sig_rphi2) * p.g.inv_r[l], p.max_dphi);
            win.dz = fminf(p.nsigma * sqrtf(czz + p.sig_z2), p.max_dz);
            win.phic = atan2f(x[1], x[0]);
            win.z = x[2];
            win.bo = p.bin_off + (((int64_t)ev * L + l) * (nbins + 1));
            win.seg_lo = seg_lo;
            // bin ranges widened by a rounding margin: a hit that passes the
            // exact window test always lies in a scanned bin
            const float zm = 1e-4f * (1.0f + fabsf(x[2])), pm = 1e-5f;
            win.iz0 = z_bin(x[2] - win.dz - zm, p.bg);
            win.iz1 = z_bin(x[2] + win.dz + zm, p.bg);
            int ip0, ip1;
            if (win.dphi >= kPi - pm) {
                ip0 = 0;
                ip1 = p.bg.n_phi - 1;
            } else {
                ip0 = (int)floorf((win.phic - win.dphi - pm + kPi) * (float)p.bg.n_phi * (1.0f / (2.0f * kPi)));
                ip1 = (int)floorf((win.phic + win.dphi + pm + kPi) * (float)p.bg.n_phi * (1.0f / (2.0f * kPi)));
            }
            win.ip0 = ip0;
            win.nphi = min(ip1 - ip0 + 1, p.bg.n_phi);
        }
        auto load_hit = [&](uint32_t hl, float m[3], float v[6]) {
            const int64_t hg = seg_lo + hl;
#pragma unroll
            for (int i = 0; i < 3; ++i) m[i] = p.hit_pos[i * p.H + hg];
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = p.hit_cov[i * p.H + hg];
        };
        // inputs of the proposal shared by every hit of this candidate
        auto cand_features = [&](float f[kMlpIn]) {
#pragma unroll
            for (int i = 0; i < 6; ++i) f[3 + i] = log10f(fmaxf(c[pk(i, i)], 1e-30f));
            f[9] = copysignf(rsqrtf(x[3] * x[3] + x[4] * x[4]), qkb);
            f[10] = __fdiv_rn((float)l, (float)L);  // correctly rounded, whatever the division flags
            f[11] = (float)(l - nhits);
        };
        if (MODE != kModeLog) {
            // first pass: the window's hits are collected (cheap bin reads
            // only) while there are at most `cap`; one more marks the window
            // as wide
            const int cap = MODE == kModeProposal ? p.topk : HB;
            uint32_t hb[HB];
#pragma unroll
            for (int k = 0; k < HB; ++k) hb[k] = kNoKey;
            int n_in = 0;
            if (reached) {
                // each z row's bins are one contiguous key run (two past the
                // wrap at +-pi): one pair of bin-offset loads per run, then
                // the keys kKeyBatch at a time with their loads issued together
                const int nphi = p.bg.n_phi;
                int a0 = win.ip0;
                a0 = a0 < 0 ? a0 + nphi : (a0 >= nphi ? a0 - nphi : a0);
                const int e0 = a0 + win.nphi;
                const int b0 = min(e0, nphi), b1 = e0 > nphi ? e0 - nphi : 0;
                for (int iz = win.iz0; iz <= win.iz1 && n_in <= cap; ++iz) {
                    const int32_t *row = win.bo + iz * nphi;
                    for (int r = 0; r < 2 && n_in <= cap; ++r) {
                        const int ra = r ? 0 : a0, rb = r ? b1 : b0;
                        if (ra >= rb) continue;
                        const int ka = row[ra], kb = row[rb];
                        for (int q = ka; q < kb && n_in <= cap; q += kKeyBatch) {
                            float4 kk[kKeyBatch];
#pragma unroll
                            for (int j = 0; j < kKeyBatch; ++j)
                                if (q + j < kb) kk[j] = p.bkey[seg_lo + q + j];
#pragma unroll
                            for (int j = 0; j < kKeyBatch; ++j) {
                                if (q + j < kb && n_in <= cap && fabsf(wrap_pi(kk[j].x - win.phic)) <= win.dphi &&
                                    fabsf(kk[j].y - win.z) <= win.dz) {
                                    const uint32_t hl = (uint32_t)__float_as_int(kk[j].z);
#pragma unroll
                                    for (int k = 0; k < HB; ++k)
                                        if (k == n_in && n_in < cap) hb[k] = hl;
                                    ++n_in;
                                }
                            }
                        }
                    }
                }
            }
            const bool wide = n_in > cap;
            if (MODE == kModePlain && p.flag_over > 0) over |= n_in > p.flag_over;
            if (MODE == kModeProposal && __any_sync(0xffffffffu, wide)) {
                // a wide window keeps its topk best hits by logit: park this
                // lane's state, walk the warp's wide windows, take it back
                volatile float *vs = slots + threadIdx.x;
                volatile float *vw = wc + threadIdx.x;
#pragma unroll
                for (int i = 0; i < 6; ++i) vs[(kSlotX + i) * 128] = x[i];
#pragma unroll
                for (int i = 0; i < 21; ++i) vs[(kSlotC + i) * 128] = c[i];
#pragma unroll
                for (int k = 0; k < kMaxN; ++k) vw[(kWcHb + k) * 128] = __int_as_float((int)hb[k]);
                vw[kWcNx * 128] = nx;
                vw[kWcNy * 128] = ny;
                vw[kWcCtt * 128] = ctt;
                vw[kWcCtz * 128] = ctz;
                vw[kWcCzz * 128] = czz;
                vw[kWcSegLo * 128] = __int_as_float((int)(uint32_t)(unsigned long long)seg_lo);
                vw[(kWcSegLo + 1) * 128] = __int_as_float((int)(uint32_t)((unsigned long long)seg_lo >> 32));
                const unsigned long long bo_bits = reinterpret_cast<unsigned long long>(win.bo);
                vw[kWcBo * 128] = __int_as_float((int)(uint32_t)bo_bits);
                vw[(kWcBo + 1) * 128] = __int_as_float((int)(uint32_t)(bo_bits >> 32));
                vw[kWcPhic * 128] = win.phic;
                vw[kWcDphi * 128] = win.dphi;
                vw[kWcZ * 128] = win.z;
                vw[kWcDz * 128] = win.dz;
                vw[kWcIz0 * 128] = __int_as_float(win.iz0);
                vw[kWcIz1 * 128] = __int_as_float(win.iz1);
                vw[kWcIp0 * 128] = __int_as_float(win.ip0);
                vw[kWcNphi * 128] = __int_as_float(win.nphi);
                vw[kWcNhits * 128] = __int_as_float(nhits);
                vw[kWcQkb * 128] = qkb;
                __syncwarp();
                const WideArgs wa{p.bkey,    p.hit_pos, p.hit_cov, p.H,       p.bg.n_phi,
                                  p.topk,    l,         L,         p.mlp_W1, p.mlp_W2, p.mlp_w32};
                scan_wide(wa, wide, slots, wc, xs);
#pragma unroll
                for (int i = 0; i < 6; ++i) x[i] = vs[(kSlotX + i) * 128];
#pragma unroll
                for (int i = 0; i < 21; ++i) c[i] = vs[(kSlotC + i) * 128];
#pragma unroll
                for (int k = 0; k < kMaxN; ++k) hb[k] = (uint32_t)__float_as_int(vw[(kWcHb + k) * 128]);
                nx = vw[kWcNx * 128];
                ny = vw[kWcNy * 128];
                ctt = vw[kWcCtt * 128];
                ctz = vw[kWcCtz * 128];
                czz = vw[kWcCzz * 128];
                seg_lo = (int64_t)(((unsigned long long)(uint32_t)__float_as_int(vw[(kWcSegLo + 1) * 128]) << 32) |
                                   (uint32_t)__float_as_int(vw[kWcSegLo * 128]));
            }
            if (MODE == kModeProposal || !wide) {
                // the full chi2 for the collected (or ranked) hits, loads
                // issued together
#pragma unroll
                for (int k2 = 0; k2 < HB; ++k2) {
                    if (hb[k2] == kNoKey) continue;
                    float m[3], v[6], dc, f3[3];
                    load_hit(hb[k2], m, v);
                    if (hit_eval(x, nx, ny, ctt, ctz, czz, m, v, &dc, f3) && dc <= p.chi2_cut)
                        insert(dc, hb[k2], kNoKey);
                }
            } else if (!(MODE == kModePlain && p.flag_over > 0)) {
                // exhaustive search of a window wider than the buffer (the
                // flagging pass leaves it: its seed is built again by the
                // proposal pass)
                WindowCursor cur;
                cur.start(win);
                for (uint32_t hl = cur.next(p, win); hl != kNoKey; hl = cur.next(p, win)) {
                    float m[3], v[6], dc, f3[3];
                    load_hit(hl, m, v);
                    if (hit_eval(x, nx, ny, ctt, ctz, czz, m, v, &dc, f3) && dc <= p.chi2_cut) insert(dc, hl, kNoKey);
                }
            }
        } else if (reached) {
            // training log: every in-window pair's features now, label 1 once
            // the pair survives the merge
            WindowCursor cur;
            cur.start(win);
            for (uint32_t hl = cur.next(p, win); hl != kNoKey; hl = cur.next(p, win)) {
                float m[3], v[6], dc, feat[kMlpIn];
                load_hit(hl, m, v);
                const bool ok = hit_eval(x, nx, ny, ctt, ctz, czz, m, v, &dc, feat);
                uint32_t row = kNoKey;
                const unsigned long long r = atomicAdd(p.log_n, 1ull);
                if (r < p.log_cap) {
                    cand_features(feat);
                    row = (uint32_t)r;
#pragma unroll
                    for (int i = 0; i < kMlpIn; ++i) p.log_f[(int64_t)r * kMlpIn + i] = feat[i];
                    p.log_y[r] = 0.0f;
                    int32_t *ref = p.log_ref + (int64_t)r * 4;
                    ref[0] = (int32_t)s;
                    ref[1] = slot;
                    ref[2] = l;
                    ref[3] = (int32_t)(seg_lo + hl);
                }
                if (ok && dc <= p.chi2_cut) insert(dc, hl, row);
            }
        }
        // merge the group's lists: N rounds of a group arg-min; the head of a
        // lane is its best hit child, then its hole child.  A round's offers
        // come from distinct slots, so (hits desc, chi2 asc, slot asc) orders
        // them totally and fits one 64-bit key, (63 - hits) << 35 | the bits
        // of chi2 (non-negative floats order as their bit patterns) << 3 |
        // slot; ~0 offers nothing.  The taker of the round's child reads the
        // winner's hit by one more shuffle.
        int taken = 0;  // hit children of this lane already selected
        bool hole_taken = false;
        int new_parent = -1;
        uint32_t new_hit = 0;  // hit index + 1, 0 = hole
        float new_chi2 = 0.0f;
        int new_nhits = 0;
        int n_new = 0;
        for (int r = 0; r < N; ++r) {
            const bool offer_hit = valid && taken < N && lh[0] != kNoKey;
            const bool offer = offer_hit || (valid && !hole_taken);
            const int kh = offer_hit ? nhits + 1 : nhits;
            const float kc = offer_hit ? chi2 + lc[0] : chi2;
            unsigned long long bk = offer ? ((unsigned long long)(63 - kh) << 35) |
                                                ((unsigned long long)__float_as_uint(kc) << 3) | (unsigned)slot
                                          : ~0ull;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                unsigned long long o;
                if constexpr ((G & (G - 1)) == 0) {  // butterfly within a power-of-two group
                    o = __shfl_xor_sync(gmask, bk, d, G);
                } else {  // G = 6: pairs, then slots 0-3, then the two halves crossed
                    const int ps = d == 1 ? (slot ^ 1) : d == 2 ? (slot < 4 ? slot ^ 2 : slot)
                                                                : (slot < 4 ? 4 + (slot & 1) : slot - 4);
                    const int src_lane = lane_ok ? gbase + ps : lane;
                    o = __shfl_sync(gmask, bk, src_lane, 32);
                }
                bk = o < bk ? o : bk;
            }
            if (bk == ~0ull) break;
            const int win_slot = (int)(bk & 7u);
            const uint32_t whit = __shfl_sync(gmask, offer_hit ? lh[0] + 1u : 0u, gbase + win_slot, 32);
            if (slot == r) {
                new_parent = win_slot;
                new_hit = whit;
                new_nhits = 63 - (int)(bk >> 35);
                new_chi2 = __uint_as_float((uint32_t)(bk >> 3));
            }
            if (slot == win_slot) {
                if (offer_hit) {  // pop the head of the list
                    if (MODE == kModeLog && lr[0] != kNoKey) p.log_y[lr[0]] = 1.0f;  // the pair survives
#pragma unroll
                    for (int k = 0; k < NL - 1; ++k) {
                        lc[k] = lc[k + 1];
                        lh[k] = lh[k + 1];
                        lr[k] = lr[k + 1];
                    }
                    lc[NL - 1] = INFINITY;
                    lh[NL - 1] = kNoKey;
                    lr[NL - 1] = kNoKey;
                    ++taken;
                } else {
                    hole_taken = true;
                }
            }
            ++n_new;
        }
        // each lane takes over child `slot` from its parent lane
        const int src = gbase + (new_parent >= 0 ? new_parent : slot);
        float px[6], pc[21];
#pragma unroll
        for (int i = 0; i < 6; ++i) px[i] = __shfl_sync(gmask, x[i], src, 32);
#pragma unroll
        for (int i = 0; i < 21; ++i) pc[i] = __shfl_sync(gmask, c[i], src, 32);
        const int pstop = __shfl_sync(gmask, (int)stopped, src, 32);
        const uint32_t pflags = __shfl_sync(gmask, flags, src, 32);
        nc = n_new;
        if (slot < nc) {
#pragma unroll
            for (int i = 0; i < 6; ++i) x[i] = px[i];
#pragma unroll
            for (int i = 0; i < 21; ++i) c[i] = pc[i];
            stopped = pstop != 0;
            flags = pflags;
            chi2 = new_chi2;
            nhits = new_nhits;
            if (new_hit) {
                const int64_t hg = seg_lo + (new_hit - 1u);
                float m[3], v[6], d;
#pragma unroll
                for (int i = 0; i < 3; ++i) m[i] = p.hit_pos[i * p.H + hg];
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = p.hit_cov[i * p.H + hg];
                const int st = update(x, c, m, v, p.rt, &d, slots + threadIdx.x, 128);
                if (st == 1) flags |= KF_FLAG_INVERSION_FAILED;
                if (st >= 2) flags |= KF_FLAG_FP64_PATH;
                if (st == 3) flags |= KF_FLAG_PSD_REPAIRED;
            }
            bp[l * 128 + threadIdx.x] = (int32_t)(((uint32_t)new_parent << 27) | new_hit);
        }
        __syncwarp();
    }
    if (MODE == kModePlain && p.flag_over > 0) {
        // OR over the seed's lanes (the group's lanes are contiguous)
        const unsigned ov = __ballot_sync(0xffffffffu, over && seed_ok);
        if (seed_ok && slot == 0) p.seed_flag[s] = (ov >> gbase) & ((G == 32 ? 0xffffffffu : (1u << G) - 1u)) ? 1 : 0;
    }
    if (!seed_ok) return;
    const int N_ = p.N;
    const int64_t sj = s * N_ + slot;
    if (slot < N_) {
        const bool have = slot < nc;
#pragma unroll
        for (int i = 0; i < 6; ++i) p.out_state[i * p.S * N_ + sj] = have ? x[i] : 0.0f;
#pragma unroll
        for (int i = 0; i < 21; ++i) p.out_cov[i * p.S * N_ + sj] = have ? c[i] : 0.0f;
        p.out_chi2[sj] = have ? chi2 : 0.0f;
        p.out_nhits[sj] = (int16_t)(have ? nhits : -1);
        p.out_flags[sj] = have ? flags : 0u;
        int cur = slot;
        for (int l = L - 1; l >= 0; --l) {
            int32_t out = -1;
            if (have) {
                const uint32_t e = (uint32_t)bp[l * 128 + (threadIdx.x - slot) + cur];
                const uint32_t h = e & 0x7ffffffu;
                if (h) out = (int32_t)(p.hit_base + p.ev_off[(int64_t)ev * (L + 1) + l] + (h - 1u));
                cur = (int)(e >> 27);
            }
            p.out_hit[sj * L + l] = out;
        }
    }
}

}  // namespace
}  // namespace kf

using namespace kf;

namespace {

// (n_phi, n_z) bin grids the build autotuner tries (at most 16,384 bins)
constexpr int kBinGrids[][2] = {{256, 64}, {512, 32}, {128, 64}, {256, 32}, {128, 128}};

int size_class(int64_t n)
{
    int c = 0;
    while ((int64_t(1) << (c + 1)) <= n && c < 40) ++c;
    return c;
}

struct BuildLog {
    float *features, *labels;
    int32_t *ref;
    int64_t capacity;
    uint64_t *count;
};

template <class T>
bool grow(T **ptr, size_t &cap, size_t need)
{
    if (need <= cap) return true;
    cudaFree(*ptr);
    *ptr = nullptr;
    cap = 0;
    if (cudaMalloc((void **)ptr, std::max<size_t>(need, 1) * sizeof(T)) != cudaSuccess) return false;
    cap = need;
    return true;
}

// Segment bounds of the n_events rows of hit_offsets [n_events][L + 1], less
// `shift`: out [n_events L + 1].  Returns the largest segment.
int64_t segment_bounds(const int64_t *hit_offsets, int n_events, int L, int64_t shift, int64_t *out)
{
    const size_t n_seg = (size_t)n_events * L;
    for (int e = 0; e < n_events; ++e)
        for (int l = 0; l < L; ++l) out[(size_t)e * L + l] = hit_offsets[(int64_t)e * (L + 1) + l] - shift;
    out[n_seg] = hit_offsets[(int64_t)(n_events - 1) * (L + 1) + L] - shift;
    int64_t m = 0;
    for (size_t i = 0; i < n_seg; ++i) m = std::max<int64_t>(m, out[i + 1] - out[i]);
    return m;
}

// Bins per (event, layer) the build needs room for: the grid asked for, else
// the largest the tuner tries.
int bins_needed(const kf_options &o)
{
    int nb = 0;
    for (const auto &gr : kBinGrids)
        if ((!o.n_phi_bins || o.n_phi_bins == gr[0]) && (!o.n_z_bins || o.n_z_bins == gr[1]))
            nb = std::max(nb, gr[0] * gr[1]);
    return std::max(nb, std::max(o.n_phi_bins, 1) * std::max(o.n_z_bins, 1));
}

// Grow the binning scratch for n_events events of L layers and n_hits hits.
bool reserve_bins(BuildState *st, const kf_options &o, int n_events, int L, int64_t n_hits)
{
    const size_t n_seg = (size_t)n_events * L;
    const int nb = bins_needed(o);
    return grow(&st->bkey, st->hit_capacity, (size_t)n_hits) &&
           grow(&st->bin_off, st->bin_capacity, n_seg * (nb + 1)) &&
           grow(&st->hit_rank, st->rank_capacity, (size_t)n_hits);
}

// One build on device buffers: events [0, n_events) of the batch (ev_off, the
// batch's rows of hit_offsets less its first hit, and their segment bounds,
// both on the device), its hits and seeds; written hit indices gain hit_base.
struct BuildBatch {
    int n_events;
    const int64_t *ev_off, *seg_off;
    int64_t max_seg;
    const float *hit_pos, *hit_cov;
    int64_t n_hits, n_seeds;
    const int32_t *seed_event;
    const float *seed_state, *seed_cov;
    const int8_t *seed_charge;
    int32_t *out_hit;
    float *out_chi2;
    int16_t *out_nhits;
    float *out_state, *out_cov;
    uint32_t *out_flags;
    int event_base;
    int64_t hit_base;
};

// Binning and the clone engine for one batch, in the tuned shape (tuned now,
// synchronously, for a new workload class).
int build_run(kf_context *ctx, const FitGeom &g, const kf_options &o, const BuildBatch &b, const BuildLog *log,
              cudaStream_t stream)
{
    BuildState *st = context_build_state(ctx);
    const int L = g.L;
    const size_t n_seg = (size_t)b.n_events * L;
    if (!reserve_bins(st, o, b.n_events, L, b.n_hits))
        return set_error(ctx, KF_ERR_NOMEM, "could not allocate the build's scratch");
    const __nv_bfloat16 *W1 = nullptr, *W2 = nullptr;
    const float *w32 = nullptr;
    if (o.use_proposal) proposal_weights(ctx, &W1, &W2, &w32);
    BuildParams p;
    p.g = g;
    p.rt = make_routing(o);
    p.N = o.max_cands;
    p.chi2_cut = o.chi2_cut;
    p.nsigma = o.window_nsigma;
    p.sig_rphi2 = o.hit_sigma_rphi * o.hit_sigma_rphi;
    p.sig_z2 = o.hit_sigma_z * o.hit_sigma_z;
    p.max_dphi = o.window_max_dphi;
    p.max_dz = o.window_max_dz;
    p.S = b.n_seeds;
    p.H = b.n_hits;
    p.n_events = b.n_events;
    p.event_base = b.event_base;
    p.hit_base = b.hit_base;
    p.ev_off = b.ev_off;
    p.hit_pos = b.hit_pos;
    p.hit_cov = b.hit_cov;
    p.bkey = st->bkey;
    p.bin_off = st->bin_off;
    p.seed_event = b.seed_event;
    p.seed_state = b.seed_state;
    p.seed_cov = b.seed_cov;
    p.seed_charge = b.seed_charge;
    p.out_hit = b.out_hit;
    p.out_chi2 = b.out_chi2;
    p.out_nhits = b.out_nhits;
    p.out_state = b.out_state;
    p.out_cov = b.out_cov;
    p.out_flags = b.out_flags;
    p.log_f = log ? log->features : nullptr;
    p.log_y = log ? log->labels : nullptr;
    p.log_ref = log ? log->ref : nullptr;
    p.log_n = log ? reinterpret_cast<unsigned long long *>(log->count) : nullptr;
    p.log_cap = log ? (unsigned long long)log->capacity : 0ull;
    p.topk = o.topk;
    p.mlp_W1 = W1;
    p.mlp_W2 = W2;
    p.mlp_w32 = w32;
    p.flag_over = 0;
    p.seed_flag = nullptr;
    p.seed_list = nullptr;
    p.list_count = nullptr;
    // lanes per seed: the smallest group that holds N candidates (6 for N = 5
    // or 6, so that a warp holds five seeds instead of four)
    const int G = p.N == 1 ? 1 : p.N <= 2 ? 2 : p.N <= 4 ? 4 : p.N <= 6 ? 6 : 8;
    const int64_t seeds_per_block = 4 * (32 / G);
    const unsigned grid = (unsigned)((b.n_seeds + seeds_per_block - 1) / seeds_per_block);
    const int mode = o.use_proposal ? kModeProposal : log ? kModeLog : kModePlain;
    const int smem_plain = (int)build_smem_base(L);
    const int smem = (int)(mode == kModeProposal ? smem_plain + kBuildSmemMlp : smem_plain);
    using Kernel = void (*)(const BuildParams);
    static const Kernel table[5][3] = {
        {build_kernel<1, kModePlain>, build_kernel<1, kModeLog>, build_kernel<1, kModeProposal>},
        {build_kernel<2, kModePlain>, build_kernel<2, kModeLog>, build_kernel<2, kModeProposal>},
        {build_kernel<4, kModePlain>, build_kernel<4, kModeLog>, build_kernel<4, kModeProposal>},
        {build_kernel<6, kModePlain>, build_kernel<6, kModeLog>, build_kernel<6, kModeProposal>},
        {build_kernel<8, kModePlain>, build_kernel<8, kModeLog>, build_kernel<8, kModeProposal>}};
    const int gi = G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : G == 6 ? 3 : 4;
    const Kernel kern = table[gi][mode];
    if (mode == kModeProposal && (!grow(&st->seed_flag, st->flag_capacity, (size_t)b.n_seeds) ||
                                  !grow(&st->seed_list, st->list_capacity, (size_t)b.n_seeds) ||
                                  !grow(&st->list_count, st->count_capacity, 1)))
        return set_error(ctx, KF_ERR_NOMEM, "could not allocate the build's scratch");
    // one build: the binning for the grid (n_phi, n_z), then the kernel; the
    // speculative learned build runs the plain kernel, flagging every seed one
    // of whose windows held more than topk hits, then the proposal kernel on
    // the flagged seeds only (the others' builds are the same either way)
    auto enqueue = [&](int nphi, int nz, int spec) -> cudaError_t {
        const BinGrid bgr{nphi, nz, g.z_half};
        cudaError_t e1 = bin_hits(b.seg_off, (int64_t)n_seg, b.max_seg, b.hit_pos, b.n_hits, bgr, st->bkey,
                                  st->bin_off, st->hit_rank, context_sm_count(ctx), stream);
        if (e1 != cudaSuccess) return e1;
        BuildParams q = p;
        q.bg = bgr;
        // the dynamic shared memory opt-in is a per-device attribute: set it
        // on every call (a host-side attribute write, no stream work)
        if ((e1 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e1;
        if (log && (e1 = cudaMemsetAsync(log->count, 0, sizeof(uint64_t), stream)) != cudaSuccess) return e1;
        if (b.n_seeds == 0) return cudaGetLastError();
        if (mode == kModeProposal && spec) {
            const Kernel kp = table[gi][kModePlain];
            if ((e1 = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_plain)) !=
                cudaSuccess)
                return e1;
            BuildParams q1 = q;
            q1.flag_over = o.topk;
            q1.seed_flag = st->seed_flag;
            kp<<<grid, 128, smem_plain, stream>>>(q1);
            if ((e1 = cudaMemsetAsync(st->list_count, 0, sizeof(unsigned), stream)) != cudaSuccess) return e1;
            const unsigned cg = (unsigned)std::min<int64_t>((b.n_seeds + 255) / 256, (int64_t)context_sm_count(ctx) * 8);
            flagged_seeds_kernel<<<cg, 256, 0, stream>>>(st->seed_flag, b.n_seeds, st->seed_list, st->list_count);
            q.seed_list = st->seed_list;
            q.list_count = st->list_count;
        }
        kern<<<grid, 128, smem, stream>>>(q);
        return cudaGetLastError();
    };
    // the shape: the one tuned for this workload class, or tuned now on the
    // caller's own buffers (a build only reads its inputs and overwrites its
    // outputs; the training log restarts its count)
    const int fixed_spec = mode == kModeProposal ? o.build_variant : -1;
    const auto key = std::make_tuple(L, p.N, mode, size_class(b.n_seeds), size_class(b.n_hits), o.n_phi_bins, o.n_z_bins,
                                     fixed_spec);
    std::tuple<int, int, int> shape;
    cudaError_t e = cudaSuccess;
    auto it = st->tuned.find(key);
    if (it != st->tuned.end()) {
        shape = it->second;
    } else {
        std::vector<std::tuple<int, int, int>> cand;
        for (int spec = 0; spec <= (mode == kModeProposal ? 1 : 0); ++spec) {
            if (fixed_spec >= 0 && spec != fixed_spec) continue;
            for (const auto &gr : kBinGrids)
                if ((!o.n_phi_bins || o.n_phi_bins == gr[0]) && (!o.n_z_bins || o.n_z_bins == gr[1]))
                    cand.emplace_back(gr[0], gr[1], spec);
            if (!o.n_phi_bins && !o.n_z_bins) continue;
            bool listed = false;
            for (const auto &c : cand) listed |= std::get<2>(c) == spec;
            if (!listed)  // a fixed grid outside the tuner's list
                cand.emplace_back(o.n_phi_bins ? o.n_phi_bins : 256, o.n_z_bins ? o.n_z_bins : 64, spec);
        }
        shape = cand[0];
        if (cand.size() > 1) {
            cudaEvent_t ta, tb;
            cudaEventCreate(&ta);
            cudaEventCreate(&tb);
            float best = 1e30f;
            for (const auto &c : cand) {
                if ((e = enqueue(std::get<0>(c), std::get<1>(c), std::get<2>(c))) != cudaSuccess) break;
                cudaEventRecord(ta, stream);
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
                    e = enqueue(std::get<0>(c), std::get<1>(c), std::get<2>(c));
                cudaEventRecord(tb, stream);
                if (e != cudaSuccess || (e = cudaEventSynchronize(tb)) != cudaSuccess) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, ta, tb);
                if (ms < best) {
                    best = ms;
                    shape = c;
                }
            }
            cudaEventDestroy(ta);
            cudaEventDestroy(tb);
            if (e != cudaSuccess) return cuda_error(ctx, e, "build tuning");
        }
        st->tuned[key] = shape;
    }
    if ((e = enqueue(std::get<0>(shape), std::get<1>(shape), std::get<2>(shape))) != cudaSuccess)
        return cuda_error(ctx, e, "build launch");
    return KF_OK;
}

// Argument checks shared by the build entry points (pointers apart): the
// geometry into *g, the options, the log, the sizes and, when there are
// seeds, the offsets table (host).
int check_build_args(kf_context *ctx, const kf_geometry *geom, const kf_options &o, int n_events,
                     const int64_t *hit_offsets, int64_t n_hits, int64_t n_seeds, const BuildLog *log, FitGeom *g)
{
    int rc;
    if ((rc = check_geometry(ctx, geom, g))) return rc;
    if ((rc = check_options(ctx, o))) return rc;
    if (o.max_cands < 1 || o.max_cands > 8) return set_error(ctx, KF_ERR_ARG, "max_cands must be 1..8");
    if (!(o.chi2_cut > 0.0f) || !(o.window_nsigma > 0.0f) || !(o.hit_sigma_rphi >= 0.0f) || !(o.hit_sigma_z >= 0.0f) ||
        !(o.window_max_dphi > 0.0f) || !(o.window_max_dz > 0.0f))
        return set_error(ctx, KF_ERR_ARG,
                         "chi2_cut, window_nsigma and the window caps must be positive, hit sigmas non-negative");
    if (o.n_phi_bins < 0 || o.n_z_bins < 0 || (int64_t)o.n_phi_bins * o.n_z_bins > 16384)
        return set_error(ctx, KF_ERR_ARG, "n_phi_bins x n_z_bins must be 1..16384 (0: tuned)");
    if (o.build_variant < -1 || o.build_variant > 1)
        return set_error(ctx, KF_ERR_ARG, "build_variant must be -1 (tuned), 0 or 1");
    if (o.use_proposal) {
        if (log) return set_error(ctx, KF_ERR_ARG, "the training log records the plain build: use_proposal must be 0");
        if (o.topk < 1 || o.topk > kMaxN) return set_error(ctx, KF_ERR_ARG, "topk must be 1..8");
        if (!proposal_loaded(ctx)) return set_error(ctx, KF_ERR_ARG, "use_proposal needs weights (kf_proposal_load)");
    }
    if (log) {
        if (log->capacity < 0) return set_error(ctx, KF_ERR_ARG, "log capacity must be >= 0");
        if ((rc = check_ptr(ctx, log->count, 8, "log_count"))) return rc;
        if (log->capacity > 0 && ((rc = check_ptr(ctx, log->features, 4, "log_features")) ||
                                  (rc = check_ptr(ctx, log->labels, 4, "log_labels")) ||
                                  (rc = check_ptr(ctx, log->ref, 4, "log_ref"))))
            return rc;
    }
    if (n_events < 0 || n_seeds < 0 || n_hits < 0 || n_hits >= (int64_t(1) << 31))
        return set_error(ctx, KF_ERR_ARG, "n_events, n_seeds must be >= 0 and n_hits < 2^31");
    if (n_seeds == 0) return KF_OK;
    if (n_events < 1 || !hit_offsets) return set_error(ctx, KF_ERR_ARG, "hit_offsets (host) needs n_events >= 1 rows");
    const int L = g->L;
    for (int e = 0; e < n_events; ++e) {
        const int64_t *row = hit_offsets + (int64_t)e * (L + 1);
        if (e > 0 && row[0] != hit_offsets[(int64_t)(e - 1) * (L + 1) + L])
            return set_error(ctx, KF_ERR_ARG, "events must be stored back to back (event %d)", e);
        for (int l = 0; l < L; ++l)
            if (row[l] < 0 || row[l + 1] < row[l] || row[l + 1] > n_hits)
                return set_error(ctx, KF_ERR_ARG, "hit_offsets row %d is not a non-decreasing run within n_hits", e);
        if (row[L] - row[0] >= (int64_t(1) << 27))
            return set_error(ctx, KF_ERR_ARG, "event %d holds 2^27 or more hits", e);
    }
    return KF_OK;
}

int build_impl(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
               const float *hit_pos, const float *hit_cov, int64_t n_hits, int64_t n_seeds, const int32_t *seed_event,
               const float *seed_state, const float *seed_cov, const int8_t *seed_charge, int32_t *out_hit_idx,
               float *out_chi2, int16_t *out_nhits, float *out_state, float *out_cov, uint32_t *out_flags,
               const kf_options *opt, kf_stream stream_, const BuildLog *log)
{
    if (!ctx) return KF_ERR_ARG;
    kf_options o;
    if (opt) o = *opt;
    else kf_options_default(&o);
    int rc;
    FitGeom g;
    if ((rc = check_build_args(ctx, geom, o, n_events, hit_offsets, n_hits, n_seeds, log, &g))) return rc;
    if (n_seeds == 0) {
        if (log) {
            const cudaError_t e0 = cudaMemsetAsync(log->count, 0, sizeof(uint64_t), reinterpret_cast<cudaStream_t>(stream_));
            if (e0 != cudaSuccess) return cuda_error(ctx, e0, "log counter");
        }
        return KF_OK;
    }
    const int L = g.L;
    if (n_hits > 0 && ((rc = check_ptr(ctx, hit_pos, 4, "hit_pos")) || (rc = check_ptr(ctx, hit_cov, 4, "hit_cov"))))
        return rc;
    if ((rc = check_ptr(ctx, seed_event, 4, "seed_event")) || (rc = check_ptr(ctx, seed_state, 4, "seed_state")) ||
        (rc = check_ptr(ctx, seed_cov, 4, "seed_cov")) || (rc = check_ptr(ctx, seed_charge, 1, "seed_charge")) ||
        (rc = check_ptr(ctx, out_hit_idx, 4, "out_hit_idx")) || (rc = check_ptr(ctx, out_chi2, 4, "out_chi2")) ||
        (rc = check_ptr(ctx, out_nhits, 2, "out_nhits")) || (rc = check_ptr(ctx, out_state, 4, "out_state")) ||
        (rc = check_ptr(ctx, out_cov, 4, "out_cov")) || (rc = check_ptr(ctx, out_flags, 4, "out_flags")))
        return rc;
    DeviceGuard dg(context_device(ctx));
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    BuildState *&st = context_build_state(ctx);
    if (!st) st = new BuildState;
    const size_t n_seg = (size_t)n_events * L;
    if (!grow(&st->seg_off, st->seg_capacity, n_seg + 1) || !grow(&st->ev_off, st->ev_capacity, (size_t)n_events * (L + 1)))
        return set_error(ctx, KF_ERR_NOMEM, "could not allocate the build's scratch");
    std::vector<int64_t> seg(n_seg + 1);
    const int64_t max_seg = segment_bounds(hit_offsets, n_events, L, 0, seg.data());
    cudaError_t e = cudaMemcpyAsync(st->seg_off, seg.data(), (n_seg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                    stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st->ev_off, hit_offsets, (size_t)n_events * (L + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "offsets copy");
    // the host vector must outlive the asynchronous copy
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(ctx, e, "offsets copy");
    const BuildBatch bt{n_events, st->ev_off, st->seg_off, max_seg, hit_pos, hit_cov, n_hits, n_seeds, seed_event,
                        seed_state, seed_cov, seed_charge, out_hit_idx, out_chi2, out_nhits, out_state, out_cov,
                        out_flags, 0, 0};
    return build_run(ctx, g, o, bt, log, stream);
}

}  // namespace

extern "C" int kf_build_tracks(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
                               const float *hit_pos, const float *hit_cov, int64_t n_hits, int64_t n_seeds,
                               const int32_t *seed_event, const float *seed_state, const float *seed_cov,
                               const int8_t *seed_charge, int32_t *out_hit_idx, float *out_chi2, int16_t *out_nhits,
                               float *out_state, float *out_cov, uint32_t *out_flags, const kf_options *opt,
                               kf_stream stream)
{
    return build_impl(ctx, geom, n_events, hit_offsets, hit_pos, hit_cov, n_hits, n_seeds, seed_event, seed_state,
                      seed_cov, seed_charge, out_hit_idx, out_chi2, out_nhits, out_state, out_cov, out_flags, opt,
                      stream, nullptr);
}

extern "C" int kf_build_tracks_logged(kf_context *ctx, const kf_geometry *geom, int n_events,
                                      const int64_t *hit_offsets, const float *hit_pos, const float *hit_cov,
                                      int64_t n_hits, int64_t n_seeds, const int32_t *seed_event,
                                      const float *seed_state, const float *seed_cov, const int8_t *seed_charge,
                                      int32_t *out_hit_idx, float *out_chi2, int16_t *out_nhits, float *out_state,
                                      float *out_cov, uint32_t *out_flags, const kf_options *opt, float *log_features,
                                      float *log_labels, int32_t *log_ref, int64_t log_capacity, uint64_t *log_count,
                                      kf_stream stream)
{
    if (!ctx) return KF_ERR_ARG;
    const BuildLog log{log_features, log_labels, log_ref, log_capacity, log_count};
    return build_impl(ctx, geom, n_events, hit_offsets, hit_pos, hit_cov, n_hits, n_seeds, seed_event, seed_state,
                      seed_cov, seed_charge, out_hit_idx, out_chi2, out_nhits, out_state, out_cov, out_flags, opt,
                      stream, &log);
}

extern "C" int kf_build_tuned_shape(kf_context *ctx, int n_layers, int max_cands, int mode, int64_t n_seeds,
                                    int64_t n_hits, int *n_phi_bins, int *n_z_bins, int *speculative)
{
    if (!ctx || !n_phi_bins || !n_z_bins) return KF_ERR_ARG;
    BuildState *st = context_build_state(ctx);
    if (st) {
        auto it =
            st->tuned.find(std::make_tuple(n_layers, max_cands, mode, size_class(n_seeds), size_class(n_hits), 0, 0, -1));
        if (it != st->tuned.end()) {
            *n_phi_bins = std::get<0>(it->second);
            *n_z_bins = std::get<1>(it->second);
            if (speculative) *speculative = std::get<2>(it->second);
            return KF_OK;
        }
    }
    return set_error(ctx, KF_ERR_ARG, "no build of this class has been tuned yet");
}

namespace {

// Byte offsets of one batch's device buffers (hits, seeds, outputs), each
// array aligned to 256 bytes.
struct HostBatchLayout {
    size_t hit_pos, hit_cov, seed_event, seed_state, seed_cov, seed_charge, ev_off, seg_off, out_hit, out_chi2,
        out_nhits, out_state, out_cov, out_flags, total;
    HostBatchLayout(int64_t H, int64_t S, int E, int L, int N)
    {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o += (bytes + 255) / 256 * 256;
            return at;
        };
        hit_pos = take(3 * H * 4);
        hit_cov = take(6 * H * 4);
        seed_event = take(S * 4);
        seed_state = take(6 * S * 4);
        seed_cov = take(21 * S * 4);
        seed_charge = take(S);
        ev_off = take((size_t)E * (L + 1) * 8);
        seg_off = take(((size_t)E * L + 1) * 8);
        out_hit = take((size_t)S * N * L * 4);
        out_chi2 = take((size_t)S * N * 4);
        out_nhits = take((size_t)S * N * 2);
        out_state = take((size_t)6 * S * N * 4);
        out_cov = take((size_t)21 * S * N * 4);
        out_flags = take((size_t)S * N * 4);
        total = o;
    }
};

// rows [r0, r0 + n) of `rows` arrays of row length `pitch` elements, between
// host and device (dst pitch n); one strided copy
template <class T>
cudaError_t copy_rows(T *dst, size_t dpitch, const T *src, size_t spitch, int64_t n, int rows, cudaMemcpyKind kind,
                      cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst, dpitch * sizeof(T), src, spitch * sizeof(T), (size_t)n * sizeof(T), rows, kind,
                             stream);
}

}  // namespace

extern "C" int kf_build_tracks_host(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
                                    const float *hit_pos, const float *hit_cov, int64_t n_hits, int64_t n_seeds,
                                    const int32_t *seed_event, const float *seed_state, const float *seed_cov,
                                    const int8_t *seed_charge, int32_t *out_hit_idx, float *out_chi2,
                                    int16_t *out_nhits, float *out_state, float *out_cov, uint32_t *out_flags,
                                    int events_per_batch, const kf_options *opt)
{
    if (!ctx) return KF_ERR_ARG;
    kf_options o;
    if (opt) o = *opt;
    else kf_options_default(&o);
    int rc;
    FitGeom g;
    if ((rc = check_build_args(ctx, geom, o, n_events, hit_offsets, n_hits, n_seeds, nullptr, &g))) return rc;
    if (events_per_batch < 0) return set_error(ctx, KF_ERR_ARG, "events_per_batch must be >= 0");
    if (n_seeds == 0) return KF_OK;
    if (n_hits > 0 && ((rc = check_ptr(ctx, hit_pos, 4, "hit_pos")) || (rc = check_ptr(ctx, hit_cov, 4, "hit_cov"))))
        return rc;
    if ((rc = check_ptr(ctx, seed_event, 4, "seed_event")) || (rc = check_ptr(ctx, seed_state, 4, "seed_state")) ||
        (rc = check_ptr(ctx, seed_cov, 4, "seed_cov")) || (rc = check_ptr(ctx, seed_charge, 1, "seed_charge")) ||
        (rc = check_ptr(ctx, out_hit_idx, 4, "out_hit_idx")) || (rc = check_ptr(ctx, out_chi2, 4, "out_chi2")) ||
        (rc = check_ptr(ctx, out_nhits, 2, "out_nhits")) || (rc = check_ptr(ctx, out_state, 4, "out_state")) ||
        (rc = check_ptr(ctx, out_cov, 4, "out_cov")) || (rc = check_ptr(ctx, out_flags, 4, "out_flags")))
        return rc;
    for (int64_t i = 0; i < n_seeds; ++i)
        if (seed_event[i] < 0 || seed_event[i] >= n_events || (i > 0 && seed_event[i] < seed_event[i - 1]))
            return set_error(ctx, KF_ERR_ARG, "seed_event must be non-decreasing within 0..n_events-1 (seed %lld)",
                             (long long)i);
    const int L = g.L, N = o.max_cands;
    const int B = events_per_batch ? events_per_batch : 16;
    // batches of B events: their seed and hit ranges
    struct Batch {
        int e0, e1;
        int64_t s0, s1, h0, h1;
    };
    std::vector<Batch> batches;
    int64_t max_h = 0, max_s = 0;
    for (int e0 = 0, si = 0; e0 < n_events; e0 += B) {
        Batch bt;
        bt.e0 = e0;
        bt.e1 = std::min(e0 + B, n_events);
        bt.s0 = si;
        while (si < n_seeds && seed_event[si] < bt.e1) ++si;
        bt.s1 = si;
        bt.h0 = hit_offsets[(int64_t)bt.e0 * (L + 1)];
        bt.h1 = hit_offsets[(int64_t)(bt.e1 - 1) * (L + 1) + L];
        max_h = std::max(max_h, bt.h1 - bt.h0);
        max_s = std::max(max_s, bt.s1 - bt.s0);
        if (bt.s1 > bt.s0) batches.push_back(bt);
    }
    DeviceGuard dg(context_device(ctx));
    BuildState *&st = context_build_state(ctx);
    if (!st) st = new BuildState;
    const HostBatchLayout lay(std::max<int64_t>(max_h, 1), std::max<int64_t>(max_s, 1), B, L, N);
    const size_t pin_elems = ((size_t)B * L + 1) + (size_t)B * (L + 1);
    bool ok = reserve_bins(st, o, B, L, max_h);
    for (cudaStream_t *h : {&st->hs_in, &st->hs_run, &st->hs_out})
        if (ok && !*h) ok = cudaStreamCreateWithFlags(h, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &sl : st->slot) {
        if (!ok) break;
        if (sl.dev_bytes < lay.total) {
            cudaFree(sl.dev);
            sl.dev = nullptr;
            sl.dev_bytes = 0;
            ok = cudaMalloc(&sl.dev, lay.total) == cudaSuccess;
            if (ok) sl.dev_bytes = lay.total;
        }
        if (ok && sl.pin_elems < pin_elems) {
            cudaFreeHost(sl.pin);
            sl.pin = nullptr;
            sl.pin_elems = 0;
            ok = cudaMallocHost(&sl.pin, pin_elems * sizeof(int64_t)) == cudaSuccess;
            if (ok) sl.pin_elems = pin_elems;
        }
        for (cudaEvent_t *ev : {&sl.in_done, &sl.built, &sl.out_done})
            if (ok && !*ev) ok = cudaEventCreateWithFlags(ev, cudaEventDisableTiming) == cudaSuccess;
        sl.used = false;
    }
    if (!ok) return set_error(ctx, KF_ERR_NOMEM, "could not allocate the host-buffer build's staging");
    cudaError_t e = cudaSuccess;
    for (size_t bi = 0; bi < batches.size() && e == cudaSuccess; ++bi) {
        const Batch &bt = batches[bi];
        BuildState::Slot &sl = st->slot[bi % 3];
        const int E = bt.e1 - bt.e0;
        const int64_t H = bt.h1 - bt.h0, S = bt.s1 - bt.s0;
        char *d = sl.dev;
        if (sl.used) {
            // the slot's pinned offsets may be rewritten once their copy is done;
            // its device buffers once the previous batch in it is built and read out
            if ((e = cudaEventSynchronize(sl.in_done)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(st->hs_in, sl.built, 0)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(st->hs_run, sl.out_done, 0)) != cudaSuccess) break;
        }
        // host -> device: the batch's offsets (batch-local), hits and seeds
        int64_t *seg = sl.pin, *evo = sl.pin + ((size_t)E * L + 1);
        const int64_t max_seg = segment_bounds(hit_offsets + (int64_t)bt.e0 * (L + 1), E, L, bt.h0, seg);
        for (int64_t i = 0; i < (int64_t)E * (L + 1); ++i) evo[i] = hit_offsets[(int64_t)bt.e0 * (L + 1) + i] - bt.h0;
        cudaStream_t in = st->hs_in;
        e = cudaMemcpyAsync(d + lay.seg_off, seg, ((size_t)E * L + 1) * 8, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + lay.ev_off, evo, (size_t)E * (L + 1) * 8, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess)
            e = copy_rows((float *)(d + lay.hit_pos), H, hit_pos + bt.h0, n_hits, H, 3, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess)
            e = copy_rows((float *)(d + lay.hit_cov), H, hit_cov + bt.h0, n_hits, H, 6, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + lay.seed_event, seed_event + bt.s0, S * 4, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess)
            e = copy_rows((float *)(d + lay.seed_state), S, seed_state + bt.s0, n_seeds, S, 6, cudaMemcpyHostToDevice,
                          in);
        if (e == cudaSuccess)
            e = copy_rows((float *)(d + lay.seed_cov), S, seed_cov + bt.s0, n_seeds, S, 21, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + lay.seed_charge, seed_charge + bt.s0, S, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess) e = cudaEventRecord(sl.in_done, in);
        if (e != cudaSuccess) break;
        // the build, on the run stream (the binning scratch is shared: builds run in order)
        if ((e = cudaStreamWaitEvent(st->hs_run, sl.in_done, 0)) != cudaSuccess) break;
        const BuildBatch b{E,
                           (const int64_t *)(d + lay.ev_off),
                           (const int64_t *)(d + lay.seg_off),
                           max_seg,
                           (const float *)(d + lay.hit_pos),
                           (const float *)(d + lay.hit_cov),
                           H,
                           S,
                           (const int32_t *)(d + lay.seed_event),
                           (const float *)(d + lay.seed_state),
                           (const float *)(d + lay.seed_cov),
                           (const int8_t *)(d + lay.seed_charge),
                           (int32_t *)(d + lay.out_hit),
                           (float *)(d + lay.out_chi2),
                           (int16_t *)(d + lay.out_nhits),
                           (float *)(d + lay.out_state),
                           (float *)(d + lay.out_cov),
                           (uint32_t *)(d + lay.out_flags),
                           bt.e0,
                           bt.h0};
        if ((rc = build_run(ctx, g, o, b, nullptr, st->hs_run))) return rc;
        if ((e = cudaEventRecord(sl.built, st->hs_run)) != cudaSuccess) break;
        // device -> host: the batch's outputs into the caller's rows
        cudaStream_t out = st->hs_out;
        if ((e = cudaStreamWaitEvent(out, sl.built, 0)) != cudaSuccess) break;
        const int64_t SN = S * N, TN = n_seeds * N, s0N = bt.s0 * N;
        e = cudaMemcpyAsync(out_hit_idx + s0N * L, d + lay.out_hit, (size_t)SN * L * 4, cudaMemcpyDeviceToHost, out);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_chi2 + s0N, d + lay.out_chi2, (size_t)SN * 4, cudaMemcpyDeviceToHost, out);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_nhits + s0N, d + lay.out_nhits, (size_t)SN * 2, cudaMemcpyDeviceToHost, out);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_flags + s0N, d + lay.out_flags, (size_t)SN * 4, cudaMemcpyDeviceToHost, out);
        if (e == cudaSuccess)
            e = copy_rows(out_state + s0N, TN, (const float *)(d + lay.out_state), SN, SN, 6, cudaMemcpyDeviceToHost,
                          out);
        if (e == cudaSuccess)
            e = copy_rows(out_cov + s0N, TN, (const float *)(d + lay.out_cov), SN, SN, 21, cudaMemcpyDeviceToHost, out);
        if (e == cudaSuccess) e = cudaEventRecord(sl.out_done, out);
        sl.used = true;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->hs_out);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->hs_run);
    if (e != cudaSuccess) return cuda_error(ctx, e, "host-buffer build");
    return KF_OK;
}
