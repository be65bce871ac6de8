// Combinatorial track building on sm_103a (Sections 3, 3.1 and 4.3):
//   bin_hits          - counting sort of every (event, layer)'s hits into
//                       phi x z bins (Section 3: hits partitioned spatially
//                       for a fast look-up of the compatible ones), three
//                       kernels over all segments (kf_bins.cuh);
//   clone_kernel      - the clone engine, all layers in one launch: a block
//                       holds 32 seeds, warp w candidate slot w of each; per
//                       layer every candidate is propagated and its window's
//                       hits are tested, one lane per seed merges the
//                       candidates' children into the seed's N best (in place
//                       of the paper's per-seed heaps, Section 4.3), and every
//                       slot takes over its new child from shared memory and
//                       updates it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kf.h"
#include "kf_api_internal.h"
#include "kf_fit.cuh"
#include "kf_bins.cuh"
#include "kf_mlp.cuh"

namespace kf {

struct BuildState {
    size_t hit_capacity = 0, bin_capacity = 0, seg_capacity = 0, cnt_capacity = 0;
    float4 *bkey = nullptr;  // binned hits: (phi, z, index within the segment as bits, radius)
    int32_t *bin_off = nullptr;
    int32_t *bin_cnt = nullptr;  // per (segment, bin) counts, then cursors, of the binning
    int64_t *seg_off = nullptr;  // device copy of the segment bounds [n_seg + 1]
    int64_t *ev_off = nullptr;   // device copy of hit_offsets [n_events][L + 1]
    size_t ev_capacity = 0;
};

void destroy_build_state(BuildState *s)
{
    if (!s) return;
    cudaFree(s->bkey);
    cudaFree(s->bin_off);
    cudaFree(s->bin_cnt);
    cudaFree(s->seg_off);
    cudaFree(s->ev_off);
    delete s;
}

namespace {

constexpr int kModePlain = 0, kModeLog = 1, kModeProposal = 2;
constexpr int kKeyBatch = 4;  // window keys loaded together in the collecting scan (8 was slower)

// Shared memory of the clone-engine kernel: for N candidate slots (one warp
// each) of 32 seeds (one lane each) and L layers.  Every array is [..][32],
// the seed's lane fastest, so a warp's accesses fall in distinct banks.
// Offsets in bytes from the start of the dynamic shared memory.
struct CloneLayout {
    int st;        // float [N][kSlotSize][32]: slot w's predicted state (x: 0..5, c: 6..26) for the
                   // merge and the hand-over, then the update's slot of the extended-precision paths
    int flags;     // uint32 [N][32]: the candidate's flags, kStoppedBit = stopped
    int nh;        // int [N][32]: its hits
    int chi2;      // float [N][32]: its chi2
    int ncand;     // int [32]: candidates of each seed
    int bp;        // int32 [L][N][32]: back-pointers, parent slot << 27 | (hit index + 1)
    // union: the merge's inputs and outputs, or the proposal's staged input rows
    int lcnt;      // int [N][32]: hit children listed by slot w (at most N)
    int lc;        // float [N][N][32]: their summed chi2, ascending (then hit index)
    int lh;        // uint32 [N][N][32]: their hit indices within the (event, layer)
    int lr;        // uint32 [N][N][32]: their rows of the training log (logging only)
    int sel;       // uint32 [N][32]: child of new slot j, parent << 27 | (hit index + 1)
    int sel_chi2;  // float [N][32]
    int sel_nh;    // int [N][32]
    int stage;     // float [N][32][kStageLd]: input rows of the proposal (proposal only)
    int total;
};

struct BuildParams {
    FitGeom g;
    Routing rt;
    BinGrid bg;
    int N;
    float chi2_cut, nsigma, sig_rphi2, sig_z2, max_dphi, max_dz;
    int64_t S, H;
    int n_events;
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
    CloneLayout lay;
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

constexpr int kStageLd = 12;
constexpr uint32_t kStoppedBit = 0x80000000u;

CloneLayout clone_layout(int N, int L, int mode)
{
    CloneLayout o{};
    int off = 0;
    auto take = [&](int bytes) {
        const int at = off;
        off += (bytes + 15) / 16 * 16;
        return at;
    };
    const int col = 32 * 4;  // one [32] array of 4-byte words
    o.st = take(N * kSlotSize * col);
    o.flags = take(N * col);
    o.nh = take(N * col);
    o.chi2 = take(N * col);
    o.ncand = take(col);
    o.bp = take(L * N * col);
    const int base = off;
    o.lcnt = take(N * col);
    o.lc = take(N * N * col);
    o.lh = take(N * N * col);
    o.lr = mode == kModeLog ? take(N * N * col) : 0;
    o.sel = take(N * col);
    o.sel_chi2 = take(N * col);
    o.sel_nh = take(N * col);
    const int lists_end = off;
    o.stage = base;
    const int stage_end = mode == kModeProposal ? base + N * 32 * kStageLd * 4 : base;
    o.total = std::max(lists_end, stage_end);
    return o;
}

template <class T>
__device__ __forceinline__ T *sm_at(unsigned char *sm, int off)
{
    return reinterpret_cast<T *>(sm + off);
}

// The clone engine, all build layers in one launch.  Block = 32 seeds x N
// candidate slots: warp w holds slot w of the 32 seeds, lane i seed i, so every
// lane of every warp owns one candidate.  Per layer:
//   P  every live candidate is propagated, transported and scattered (fit
//      code); its predicted state goes to shared memory; its window is
//      scanned and the chi2 of its in-window hits taken; its N best hit
//      children (by chi2, then hit index) are listed in shared memory;
//      [proposal: windows holding more than topk hits are ranked first, the
//      warps scoring their rows on the tensor cores, and only the topk best
//      by logit get a chi2]
//   S  one lane per seed (warp 0) merges its candidates' lists and holes into
//      the seed's N best children (hits desc, chi2 asc, parent slot asc, hit
//      index asc, the hole first): N rounds of a minimum over at most N list
//      heads held in registers;
//   U  the thread of new slot j reads its child's parent state from shared
//      memory and applies the update with the child's hit; a back-pointer
//      (parent slot, hit) per (layer, slot) goes to shared memory.
// After the last layer each slot walks its back-pointers to write its hits.
template <int MODE>
__global__ void __launch_bounds__(256) clone_kernel(const BuildParams p)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const CloneLayout &ly = p.lay;
    const int N = p.N, L = p.g.L;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *st = sm_at<float>(sm, ly.st);
    uint32_t *s_flags = sm_at<uint32_t>(sm, ly.flags);
    int *s_nh = sm_at<int>(sm, ly.nh);
    float *s_chi2 = sm_at<float>(sm, ly.chi2);
    int *s_ncand = sm_at<int>(sm, ly.ncand);
    int32_t *s_bp = sm_at<int32_t>(sm, ly.bp);
    int *s_lcnt = sm_at<int>(sm, ly.lcnt);
    float *s_lc = sm_at<float>(sm, ly.lc);
    uint32_t *s_lh = sm_at<uint32_t>(sm, ly.lh);
    uint32_t *s_lr = sm_at<uint32_t>(sm, ly.lr);
    uint32_t *s_sel = sm_at<uint32_t>(sm, ly.sel);
    float *s_sel_chi2 = sm_at<float>(sm, ly.sel_chi2);
    int *s_sel_nh = sm_at<int>(sm, ly.sel_nh);
    const int me = w * 32 + lane;  // [w][lane] in the [N][32] arrays
    float *col = st + w * kSlotSize * 32 + lane;  // this slot's column: [k][32]

    const int64_t s = (int64_t)blockIdx.x * 32 + lane;
    const bool seed_ok = s < p.S;
    const int ev_in = seed_ok ? p.seed_event[s] : -1;
    const bool ev_ok = seed_ok && ev_in >= 0 && ev_in < p.n_events;  // a seed of an unknown event builds nothing
    const int ev = ev_ok ? ev_in : 0;
    const float qkb = ev_ok ? (float)p.seed_charge[s] * p.g.qk : 0.0f;

    float x[6], c[21];
    float chi2 = 0.0f;
    int nhits = 0;
    uint32_t flags = 0;
    int nc = ev_ok ? 1 : 0;
    if (ev_ok && w == 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = p.seed_state[i * p.S + s];
#pragma unroll
        for (int i = 0; i < 21; ++i) c[i] = p.seed_cov[i * p.S + s];
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 21; ++i) c[i] = 0.0f;
    }
    const int nbins = p.bg.n_phi * p.bg.n_z;
    for (int l = 0; l < L; ++l) {
        // ---------------------------------------------------------------- P
        const bool valid = w < nc;
        bool reached = false;
        if (valid && !(flags & kStoppedBit)) {
            float xn[6], sd;
            Jac J;
            if (!propagate(x, qkb, p.g.r[l], xn, sd, &J)) {
                flags |= kStoppedBit | KF_FLAG_UNREACHABLE;
            } else if (fabsf(xn[2]) > p.g.z_half) {
                flags |= kStoppedBit | KF_FLAG_LEFT_BARREL;
            } else {
                transport(J, c);
                add_scattering(xn, p.g.inv_r[l], p.g.xx0[l], c);
#pragma unroll
                for (int i = 0; i < 6; ++i) x[i] = xn[i];
                reached = true;
            }
        }
        if (valid) {  // the candidate (its predicted state) for the merge and the hand-over
#pragma unroll
            for (int i = 0; i < 6; ++i) col[(kSlotX + i) * 32] = x[i];
#pragma unroll
            for (int i = 0; i < 21; ++i) col[(kSlotC + i) * 32] = c[i];
            s_flags[me] = flags;
            s_nh[me] = nhits;
            s_chi2[me] = chi2;
        }
        const int64_t seg_lo = ev_ok ? p.ev_off[(int64_t)ev * (L + 1) + l] : 0;
        Window win{};
        float nx = 0.0f, ny = 0.0f, ctt = 0.0f, ctz = 0.0f, czz = 0.0f;
        float cf[kMlpIn];  // the proposal's inputs shared by every hit of this candidate (3..11)
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
            if (MODE != kModePlain) {
#pragma unroll
                for (int i = 0; i < 6; ++i) cf[3 + i] = log10f(fmaxf(c[pk(i, i)], 1e-30f));
                cf[9] = copysignf(rsqrtf(x[3] * x[3] + x[4] * x[4]), qkb);
                cf[10] = __fdiv_rn((float)l, (float)L);  // correctly rounded, whatever the division flags
                cf[11] = (float)(l - nhits);
            }
        }
        const float xp0 = x[0], xp1 = x[1], xp2 = x[2];  // the prediction the hits are tested against
        auto load_hit = [&](uint32_t hl, float m[3], float v[6]) {
            const int64_t hg = seg_lo + hl;
#pragma unroll
            for (int i = 0; i < 3; ++i) m[i] = p.hit_pos[i * p.H + hg];
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = p.hit_cov[i * p.H + hg];
        };
        auto eval = [&](uint32_t hl, float *dc, float f3[3]) {
            float m[3], v[6];
            load_hit(hl, m, v);
            const float xp[3] = {xp0, xp1, xp2};
            return hit_eval(xp, nx, ny, ctt, ctz, czz, m, v, dc, f3);
        };
        // this candidate's best hit children, sorted by (summed chi2, hit
        // index); lr = each entry's row in the training log (logging only)
        float lc[kMaxN];
        uint32_t lh[kMaxN], lr[kMaxN];
#pragma unroll
        for (int k = 0; k < kMaxN; ++k) {
            lc[k] = INFINITY;
            lh[k] = kNoKey;
            lr[k] = kNoKey;
        }
        int n_list = 0;
        auto insert = [&](float dc, uint32_t hl, uint32_t row) {
            const float cv0 = chi2 + dc;
            if (!(cv0 < lc[kMaxN - 1] || (cv0 == lc[kMaxN - 1] && hl < lh[kMaxN - 1]))) return;
            float cv = cv0;
            uint32_t hv = hl, rv = row;
#pragma unroll
            for (int k2 = 0; k2 < kMaxN; ++k2) {
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
            n_list = min(n_list + 1, kMaxN);
        };
        if (MODE != kModeLog) {
            // first pass: the window's hits are collected (cheap bin reads
            // only) while there are at most `cap`; one more marks the window
            // as wide
            const int cap = MODE == kModeProposal ? p.topk : kMaxN;
            uint32_t hb[kMaxN];
#pragma unroll
            for (int k = 0; k < kMaxN; ++k) hb[k] = kNoKey;
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
                                    for (int k = 0; k < kMaxN; ++k)
                                        if (k == n_in && n_in < cap) hb[k] = hl;
                                    ++n_in;
                                }
                            }
                        }
                    }
                }
            }
            const bool wide = n_in > cap;
            if (MODE == kModeProposal) {
                // windows holding more than topk hits keep their topk best by
                // logit (logit desc, hit index asc): the warps score one hit
                // per ranking lane per round.  Their input rows are staged over
                // the merge's lists, which are free until the lists are written
                if (__syncthreads_or(wide)) {
                    float *xs = sm_at<float>(sm, ly.stage) + w * 32 * kStageLd;
                    const MlpWeightsRef mw{reinterpret_cast<const uint32_t *>(p.mlp_W1),
                                           reinterpret_cast<const uint32_t *>(p.mlp_W2), p.mlp_w32 + kOffB1,
                                           p.mlp_w32 + kOffB2, p.mlp_w32 + kOffW3, p.mlp_w32[kOffB3]};
                    float tz[kMaxN];
#pragma unroll
                    for (int k = 0; k < kMaxN; ++k) tz[k] = -INFINITY;
                    WindowCursor cur;
                    if (wide) {
#pragma unroll
                        for (int k = 0; k < kMaxN; ++k) hb[k] = kNoKey;
                        cur.start(win);
                    }
                    bool more = wide;
                    while (__any_sync(0xffffffffu, more)) {
                        const uint32_t hr = more ? cur.next(p, win) : kNoKey;
                        more = hr != kNoKey;
                        float feat[kMlpIn];
#pragma unroll
                        for (int i = 0; i < kMlpIn; ++i) feat[i] = 0.0f;
                        if (more) {
                            float dc;
                            eval(hr, &dc, feat);
#pragma unroll
                            for (int i = 3; i < kMlpIn; ++i) feat[i] = cf[i];
                        }
#pragma unroll
                        for (int i = 0; i < kMlpIn; ++i) xs[lane * kStageLd + i] = feat[i];
                        const float z = mlp_score_warp_split(mw, xs, kStageLd);
                        if (more) {
                            float cv = z;
                            uint32_t hv = hr;
#pragma unroll
                            for (int k2 = 0; k2 < kMaxN; ++k2) {
                                const bool before = k2 < p.topk && (cv > tz[k2] || (cv == tz[k2] && hv < hb[k2]));
                                const float t1 = tz[k2];
                                const uint32_t t2 = hb[k2];
                                tz[k2] = before ? cv : t1;
                                hb[k2] = before ? hv : t2;
                                cv = before ? t1 : cv;
                                hv = before ? t2 : hv;
                            }
                        }
                    }
                    __syncthreads();  // every row is scored before the lists overwrite the staging
                }
            }
            if (MODE == kModeProposal || !wide) {
                // the full chi2 for the collected (or ranked) hits, loads
                // issued together
#pragma unroll
                for (int k2 = 0; k2 < kMaxN; ++k2) {
                    if (hb[k2] == kNoKey) continue;
                    float dc, f3[3];
                    if (eval(hb[k2], &dc, f3) && dc <= p.chi2_cut) insert(dc, hb[k2], kNoKey);
                }
            } else {
                // exhaustive search of a window wider than the buffer
                WindowCursor cur;
                cur.start(win);
                for (uint32_t hl = cur.next(p, win); hl != kNoKey; hl = cur.next(p, win)) {
                    float dc, f3[3];
                    if (eval(hl, &dc, f3) && dc <= p.chi2_cut) insert(dc, hl, kNoKey);
                }
            }
        } else if (reached) {
            // training log: every in-window pair's features now, label 1 once
            // the pair survives the merge
            WindowCursor cur;
            cur.start(win);
            for (uint32_t hl = cur.next(p, win); hl != kNoKey; hl = cur.next(p, win)) {
                float dc, feat[kMlpIn];
                const bool ok = eval(hl, &dc, feat);
                uint32_t row = kNoKey;
                const unsigned long long r = atomicAdd(p.log_n, 1ull);
                if (r < p.log_cap) {
#pragma unroll
                    for (int i = 3; i < kMlpIn; ++i) feat[i] = cf[i];
                    row = (uint32_t)r;
#pragma unroll
                    for (int i = 0; i < kMlpIn; ++i) p.log_f[(int64_t)r * kMlpIn + i] = feat[i];
                    p.log_y[r] = 0.0f;
                    int32_t *ref = p.log_ref + (int64_t)r * 4;
                    ref[0] = (int32_t)s;
                    ref[1] = w;
                    ref[2] = l;
                    ref[3] = (int32_t)(seg_lo + hl);
                }
                if (ok && dc <= p.chi2_cut) insert(dc, hl, row);
            }
        }
        if (valid) {  // the N best hit children for the merge
            const int cnt = min(n_list, N);
            s_lcnt[me] = cnt;
#pragma unroll
            for (int k = 0; k < kMaxN; ++k)
                if (k < cnt) {
                    s_lc[(w * N + k) * 32 + lane] = lc[k];
                    s_lh[(w * N + k) * 32 + lane] = lh[k];
                    if (MODE == kModeLog) s_lr[(w * N + k) * 32 + lane] = lr[k];
                }
        }
        __syncthreads();
        // ---------------------------------------------------------------- S
        if (w == 0) {
            // children keys: k64 = (63 - hits) << 32 | chi2 bits (non-negative
            // floats order as their bit patterns), k32 = parent slot << 27 |
            // (hit index + 1), 0 for the hole; the head of slot q is its best
            // listed hit child, then its hole child
            uint32_t khi[kMaxN], klo[kMaxN], k32[kMaxN];
            int head[kMaxN];
            auto head_key = [&](int q, int h, uint32_t &hi, uint32_t &lo, uint32_t &kk) {
                const int cnt = s_lcnt[q * 32 + lane];
                const int nh = s_nh[q * 32 + lane];
                if (h < cnt) {
                    hi = (uint32_t)(63 - (nh + 1));
                    lo = __float_as_uint(s_lc[(q * N + h) * 32 + lane]);
                    kk = ((uint32_t)q << 27) | (s_lh[(q * N + h) * 32 + lane] + 1u);
                } else if (h == cnt) {
                    hi = (uint32_t)(63 - nh);
                    lo = __float_as_uint(s_chi2[q * 32 + lane]);
                    kk = (uint32_t)q << 27;
                } else {
                    hi = lo = kk = kNoKey;
                }
            };
#pragma unroll
            for (int q = 0; q < kMaxN; ++q) {
                head[q] = 0;
                khi[q] = klo[q] = k32[q] = kNoKey;
                if (q < nc) head_key(q, 0, khi[q], klo[q], k32[q]);
            }
            int r = 0;
            for (; r < N; ++r) {
                uint32_t bhi = khi[0], blo = klo[0], b32 = k32[0];
#pragma unroll
                for (int q = 1; q < kMaxN; ++q) {
                    const bool less = khi[q] < bhi || (khi[q] == bhi && (klo[q] < blo || (klo[q] == blo && k32[q] < b32)));
                    bhi = less ? khi[q] : bhi;
                    blo = less ? klo[q] : blo;
                    b32 = less ? k32[q] : b32;
                }
                if (b32 == kNoKey) break;
                s_sel[r * 32 + lane] = b32;
                s_sel_chi2[r * 32 + lane] = __uint_as_float(blo);
                s_sel_nh[r * 32 + lane] = 63 - (int)bhi;
                const int q = (int)(b32 >> 27);
                int hq = 0;
#pragma unroll
                for (int k = 0; k < kMaxN; ++k) hq = k == q ? head[k] : hq;
                if (MODE == kModeLog && (b32 & 0x7ffffffu)) {
                    const uint32_t row = s_lr[(q * N + hq) * 32 + lane];
                    if (row != kNoKey) p.log_y[row] = 1.0f;  // the pair survives
                }
                uint32_t nhi, nlo, n32;
                head_key(q, hq + 1, nhi, nlo, n32);
#pragma unroll
                for (int k = 0; k < kMaxN; ++k)
                    if (k == q) {
                        head[k] = hq + 1;
                        khi[k] = nhi;
                        klo[k] = nlo;
                        k32[k] = n32;
                    }
            }
            s_ncand[lane] = r;
        }
        __syncthreads();
        // ---------------------------------------------------------------- U
        const int nn = s_ncand[lane];
        const uint32_t e = w < nn ? s_sel[me] : 0u;
        const int par = w < nn ? (int)(e >> 27) : w;
        {
            const float *pcol = st + par * kSlotSize * 32 + lane;
#pragma unroll
            for (int i = 0; i < 6; ++i) x[i] = pcol[(kSlotX + i) * 32];
#pragma unroll
            for (int i = 0; i < 21; ++i) c[i] = pcol[(kSlotC + i) * 32];
            flags = s_flags[par * 32 + lane];
            chi2 = s_sel_chi2[me];
            nhits = s_sel_nh[me];
        }
        __syncthreads();  // every parent state is read before a slot becomes an update's scratch
        if (w < nn) {
            const uint32_t h = e & 0x7ffffffu;
            if (h) {
                float m[3], v[6], d;
                load_hit(h - 1u, m, v);
                const int stt = update(x, c, m, v, p.rt, &d, col, 32);
                if (stt == 1) flags |= KF_FLAG_INVERSION_FAILED;
                if (stt >= 2) flags |= KF_FLAG_FP64_PATH;
                if (stt == 3) flags |= KF_FLAG_PSD_REPAIRED;
            }
            s_bp[(l * N + w) * 32 + lane] = (int32_t)e;
        }
        nc = nn;
    }
    __syncthreads();
    if (!seed_ok) return;
    const int64_t sj = s * N + w;
    const bool have = w < nc;
#pragma unroll
    for (int i = 0; i < 6; ++i) p.out_state[i * p.S * N + sj] = have ? x[i] : 0.0f;
#pragma unroll
    for (int i = 0; i < 21; ++i) p.out_cov[i * p.S * N + sj] = have ? c[i] : 0.0f;
    p.out_chi2[sj] = have ? chi2 : 0.0f;
    p.out_nhits[sj] = (int16_t)(have ? nhits : -1);
    p.out_flags[sj] = have ? (flags & ~kStoppedBit) : 0u;
    int cur = w;
    for (int l = L - 1; l >= 0; --l) {
        int32_t out = -1;
        if (have) {
            const uint32_t e = (uint32_t)s_bp[(l * N + cur) * 32 + lane];
            const uint32_t h = e & 0x7ffffffu;
            if (h) out = (int32_t)(p.ev_off[(int64_t)ev * (L + 1) + l] + (h - 1u));
            cur = (int)(e >> 27);
        }
        p.out_hit[sj * L + l] = out;
    }
}

}  // namespace
}  // namespace kf

using namespace kf;

namespace {

struct BuildLog {
    float *features, *labels;
    int32_t *ref;
    int64_t capacity;
    uint64_t *count;
};

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
    if ((rc = check_geometry(ctx, geom, &g))) return rc;
    if ((rc = check_options(ctx, o))) return rc;
    if (o.max_cands < 1 || o.max_cands > 8) return set_error(ctx, KF_ERR_ARG, "max_cands must be 1..8");
    if (!(o.chi2_cut > 0.0f) || !(o.window_nsigma > 0.0f) || !(o.hit_sigma_rphi >= 0.0f) || !(o.hit_sigma_z >= 0.0f) ||
        !(o.window_max_dphi > 0.0f) || !(o.window_max_dz > 0.0f))
        return set_error(ctx, KF_ERR_ARG,
                         "chi2_cut, window_nsigma and the window caps must be positive, hit sigmas non-negative");
    if (o.n_phi_bins < 1 || o.n_z_bins < 1 || (int64_t)o.n_phi_bins * o.n_z_bins > 16384)
        return set_error(ctx, KF_ERR_ARG, "n_phi_bins x n_z_bins must be 1..16384");
    const __nv_bfloat16 *W1 = nullptr, *W2 = nullptr;
    const float *w32 = nullptr;
    if (o.use_proposal) {
        if (log) return set_error(ctx, KF_ERR_ARG, "the training log records the plain build: use_proposal must be 0");
        if (o.topk < 1 || o.topk > kMaxN) return set_error(ctx, KF_ERR_ARG, "topk must be 1..8");
        if (!proposal_loaded(ctx)) return set_error(ctx, KF_ERR_ARG, "use_proposal needs weights (kf_proposal_load)");
        proposal_weights(ctx, &W1, &W2, &w32);
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
    if (n_seeds == 0) {
        if (log) {
            const cudaError_t e0 = cudaMemsetAsync(log->count, 0, sizeof(uint64_t), reinterpret_cast<cudaStream_t>(stream_));
            if (e0 != cudaSuccess) return cuda_error(ctx, e0, "log counter");
        }
        return KF_OK;
    }
    if (n_events < 1 || !hit_offsets) return set_error(ctx, KF_ERR_ARG, "hit_offsets (host) needs n_events >= 1 rows");
    const int L = g.L;
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
    if (n_hits > 0 && ((rc = check_ptr(ctx, hit_pos, 4, "hit_pos")) || (rc = check_ptr(ctx, hit_cov, 4, "hit_cov"))))
        return rc;
    if ((rc = check_ptr(ctx, seed_event, 4, "seed_event")) || (rc = check_ptr(ctx, seed_state, 4, "seed_state")) ||
        (rc = check_ptr(ctx, seed_cov, 4, "seed_cov")) || (rc = check_ptr(ctx, seed_charge, 1, "seed_charge")) ||
        (rc = check_ptr(ctx, out_hit_idx, 4, "out_hit_idx")) || (rc = check_ptr(ctx, out_chi2, 4, "out_chi2")) ||
        (rc = check_ptr(ctx, out_nhits, 2, "out_nhits")) || (rc = check_ptr(ctx, out_state, 4, "out_state")) ||
        (rc = check_ptr(ctx, out_cov, 4, "out_cov")) || (rc = check_ptr(ctx, out_flags, 4, "out_flags")))
        return rc;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != context_device(ctx)) cudaSetDevice(context_device(ctx));
    struct Restore {
        int prev;
        ~Restore()
        {
            int cur = -1;
            if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
        }
    } restore{prev};
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);

    // scratch: binned hits, bin offsets, segment and event offsets
    BuildState *&st = context_build_state(ctx);
    if (!st) st = new BuildState;
    const int nb = o.n_phi_bins * o.n_z_bins;
    const size_t n_seg = (size_t)n_events * L;
    auto grow = [&](void **ptr, size_t &cap, size_t need, size_t elem) -> bool {
        if (need <= cap) return true;
        cudaFree(*ptr);
        *ptr = nullptr;
        cap = 0;
        if (cudaMalloc(ptr, std::max<size_t>(need, 1) * elem) != cudaSuccess) return false;
        cap = need;
        return true;
    };
    bool ok = grow((void **)&st->bkey, st->hit_capacity, (size_t)n_hits, sizeof(float4));
    ok = ok && grow((void **)&st->bin_off, st->bin_capacity, n_seg * (nb + 1), sizeof(int32_t));
    ok = ok && grow((void **)&st->bin_cnt, st->cnt_capacity, n_seg * nb, sizeof(int32_t));
    ok = ok && grow((void **)&st->seg_off, st->seg_capacity, n_seg + 1, sizeof(int64_t));
    ok = ok && grow((void **)&st->ev_off, st->ev_capacity, (size_t)n_events * (L + 1), sizeof(int64_t));
    if (!ok) return set_error(ctx, KF_ERR_NOMEM, "could not allocate the build's scratch");
    std::vector<int64_t> seg(n_seg + 1);
    for (int e = 0; e < n_events; ++e)
        for (int l = 0; l < L; ++l) seg[(size_t)e * L + l] = hit_offsets[(int64_t)e * (L + 1) + l];
    seg[n_seg] = hit_offsets[(int64_t)(n_events - 1) * (L + 1) + L];
    int64_t max_seg = 0;
    for (size_t i = 0; i < n_seg; ++i) max_seg = std::max<int64_t>(max_seg, seg[i + 1] - seg[i]);
    cudaError_t e = cudaMemcpyAsync(st->seg_off, seg.data(), (n_seg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                    stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st->ev_off, hit_offsets, (size_t)n_events * (L + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "offsets copy");
    // the host vector must outlive the asynchronous copy
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(ctx, e, "offsets copy");

    BinGrid bg{o.n_phi_bins, o.n_z_bins, g.z_half};
    if ((e = bin_hits(st->seg_off, (int64_t)n_seg, max_seg, hit_pos, n_hits, bg, st->bkey, st->bin_off, st->bin_cnt,
                      context_sm_count(ctx), stream)) != cudaSuccess)
        return cuda_error(ctx, e, "binning launch");

    BuildParams p;
    p.g = g;
    p.rt = make_routing(o);
    p.bg = bg;
    p.N = o.max_cands;
    p.chi2_cut = o.chi2_cut;
    p.nsigma = o.window_nsigma;
    p.sig_rphi2 = o.hit_sigma_rphi * o.hit_sigma_rphi;
    p.sig_z2 = o.hit_sigma_z * o.hit_sigma_z;
    p.max_dphi = o.window_max_dphi;
    p.max_dz = o.window_max_dz;
    p.S = n_seeds;
    p.H = n_hits;
    p.n_events = n_events;
    p.ev_off = st->ev_off;
    p.hit_pos = hit_pos;
    p.hit_cov = hit_cov;
    p.bkey = st->bkey;
    p.bin_off = st->bin_off;
    p.seed_event = seed_event;
    p.seed_state = seed_state;
    p.seed_cov = seed_cov;
    p.seed_charge = seed_charge;
    p.out_hit = out_hit_idx;
    p.out_chi2 = out_chi2;
    p.out_nhits = out_nhits;
    p.out_state = out_state;
    p.out_cov = out_cov;
    p.out_flags = out_flags;
    p.log_f = log ? log->features : nullptr;
    p.log_y = log ? log->labels : nullptr;
    p.log_ref = log ? log->ref : nullptr;
    p.log_n = log ? reinterpret_cast<unsigned long long *>(log->count) : nullptr;
    p.log_cap = log ? (unsigned long long)log->capacity : 0ull;
    p.topk = o.topk;
    p.mlp_W1 = W1;
    p.mlp_W2 = W2;
    p.mlp_w32 = w32;
    if (log && (e = cudaMemsetAsync(log->count, 0, sizeof(uint64_t), stream)) != cudaSuccess)
        return cuda_error(ctx, e, "log counter");
    // one block per 32 seeds, one warp per candidate slot
    const int mode = o.use_proposal ? kModeProposal : log ? kModeLog : kModePlain;
    p.lay = clone_layout(p.N, L, mode);
    const unsigned grid = (unsigned)((n_seeds + 31) / 32);
    using Kernel = void (*)(const BuildParams);
    static const Kernel table[3] = {clone_kernel<kModePlain>, clone_kernel<kModeLog>, clone_kernel<kModeProposal>};
    // the dynamic shared memory opt-in is a per-device attribute: set it on
    // every call (a host-side attribute write, no stream work)
    if ((e = cudaFuncSetAttribute(table[mode], cudaFuncAttributeMaxDynamicSharedMemorySize, p.lay.total)) !=
        cudaSuccess)
        return cuda_error(ctx, e, "build kernel shared memory");
    table[mode]<<<grid, 32 * p.N, p.lay.total, stream>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(ctx, e, "build launch");
    return KF_OK;
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
