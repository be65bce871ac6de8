// The Kalman-filter arithmetic of kf_math.cuh for two tracks at once: every
// quantity is a float2 (track a in .x, track b in .y) and the arithmetic runs
// on the packed FP32x2 instructions of sm_100 and later (fma.rn.f32x2,
// mul.rn.f32x2, add.rn.f32x2 through __ffma2_rn, __fmul2_rn, __fadd2_rn): one
// issue slot computes both tracks' value.  Square roots, reciprocals,
// logarithms and comparisons have no packed form and run per track.
//
// The steps are those of propagate, transport, add_scattering and the FP32
// update of kf_math.cuh (Sections 2 and 2.1 of the paper: helix propagation,
// C' = J C J^T + Q, the Kalman update against a 3-D hit); the branches those
// take rarely -- a start moving inwards, a turn of more than about 28 degrees
// between layers, an update routed to extended precision, a failed inversion
// -- go back to the single-track code for the track that needs them.
#pragma once

#include <cuda_runtime.h>

#include "kf_math.cuh"

namespace kf {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b and c - a b as single packed instructions
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 fnma2(float2 a, float2 b, float2 c) { return __ffma2_rn(mul2(a, f2(-1.0f)), b, c); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)); }
__device__ __forceinline__ float lane_of(float2 a, int k) { return k ? a.y : a.x; }
__device__ __forceinline__ void set_lane(float2 &a, int k, float v)
{
    if (k) a.y = v;
    else a.x = v;
}

struct Jac2 {
    float2 T[4][4];
    float2 jz[4];
    float2 jzpz;
};

__device__ __forceinline__ void jac_lane_store(Jac2 &J2, int k, const Jac &J)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) set_lane(J2.T[i][j], k, J.T[i][j]);
        set_lane(J2.jz[i], k, J.jz[i]);
    }
    set_lane(J2.jzpz, k, J.jzpz);
}

// propagate() of both tracks to radius r.  Returns a 2-bit mask: bit k set =
// track k reached the cylinder.  A track whose start moves inwards, or that
// turns by more than 2 atan(1/4) before the crossing, is propagated by the
// single-track code.
__device__ __forceinline__ unsigned propagate2(const float2 x[6], float2 qkb, float r, float2 xn[6], Jac2 &J)
{
    const float2 px = x[3], py = x[4], pz = x[5];
    const float2 pt2 = fma2(px, px, mul2(py, py));
    const float2 ipt = rsqrt2(pt2);
    const float2 tx = mul2(px, ipt), ty = mul2(py, ipt);
    const float2 om = mul2(qkb, ipt);
    const float2 u = fma2(x[0], tx, mul2(x[1], ty));
    const float2 w = fnma2(x[1], tx, mul2(x[0], ty));
    const float2 D = fnma2(x[0], x[0], fnma2(x[1], x[1], f2(r * r)));
    const float2 omD = mul2(om, D);
    const float2 Bp = fnma2(mul2(f2(0.25f), om), omD, fma2(om, w, f2(1.0f)));
    const float2 Qd = fma2(D, Bp, mul2(u, u));
    unsigned ok = 0, slow = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool good = lane_of(Qd, k) >= 0.0f && lane_of(pt2, k) > 0.0f;
        ok |= good ? 1u << k : 0u;
    }
    const float2 sq = sqrt2(make_float2(fmaxf(Qd.x, 0.0f), fmaxf(Qd.y, 0.0f)));
    const float2 den = add2(u, sq);
    const float2 sigma = mul2(D, rcp2(den));
    const float2 tau = mul2(mul2(f2(0.5f), om), sigma);
    const float2 t2 = mul2(tau, tau);
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if ((ok >> k & 1u) && !(lane_of(den, k) > 0.0f && lane_of(t2, k) < 0.0625f)) slow |= 1u << k;
    // atan(tau)/tau: its Taylor series to t2^6 (|tau| < 1/4)
    float2 ratio = fnma2(t2, f2(1.0f / 13.0f), f2(1.0f / 11.0f));
    ratio = fnma2(t2, ratio, f2(1.0f / 9.0f));
    ratio = fnma2(t2, ratio, f2(1.0f / 7.0f));
    ratio = fnma2(t2, ratio, f2(1.0f / 5.0f));
    ratio = fnma2(t2, ratio, f2(1.0f / 3.0f));
    ratio = fnma2(t2, ratio, f2(1.0f));
    const float2 s = mul2(sigma, ratio);
    const float2 gg = rcp2(fma2(tau, tau, f2(1.0f)));
    const float2 a = mul2(sigma, gg);                   // sin(phi) / omega
    const float2 b = mul2(mul2(sigma, tau), gg);        // (1 - cos(phi)) / omega
    const float2 sn = mul2(mul2(f2(2.0f), tau), gg);    // sin(phi)
    const float2 c = fnma2(mul2(f2(2.0f), t2), gg, f2(1.0f));  // cos(phi)
    xn[0] = fma2(tx, a, fma2(ty, b, x[0]));
    xn[1] = fma2(ty, a, fnma2(tx, b, x[1]));
    const float2 lz = mul2(pz, ipt);  // dz/ds
    xn[2] = fma2(lz, s, x[2]);
    xn[3] = fma2(px, c, mul2(py, sn));
    xn[4] = fnma2(px, sn, mul2(py, c));
    xn[5] = pz;
    {
        const float2 phi = mul2(om, s);
        const float2 txn = mul2(xn[3], ipt), tyn = mul2(xn[4], ipt);
        const float2 stx = mul2(s, tx), sty = mul2(s, ty);
        const float2 d03 = mul2(fnma2(stx, txn, a), ipt), d04 = mul2(fnma2(sty, txn, b), ipt);
        const float2 d13 = mul2(fnma2(stx, tyn, mul2(b, f2(-1.0f))), ipt), d14 = mul2(fnma2(sty, tyn, a), ipt);
        const float2 ptx = mul2(phi, tx), pty = mul2(phi, ty);
        const float2 d33 = fnma2(ptx, tyn, c), d34 = fnma2(pty, tyn, sn);
        const float2 d43 = fma2(ptx, txn, mul2(sn, f2(-1.0f))), d44 = fma2(pty, txn, c);
        const float2 sli = mul2(mul2(s, lz), ipt);
        const float2 d23 = mul2(mul2(sli, tx), f2(-1.0f)), d24 = mul2(mul2(sli, ty), f2(-1.0f));
        // ds/dx0 from the constraint x'^2 + y'^2 = r^2
        const float2 iden = mul2(rcp2(fma2(xn[0], txn, mul2(xn[1], tyn))), f2(-1.0f));
        const float2 ds0 = mul2(xn[0], iden), ds1 = mul2(xn[1], iden);
        const float2 ds3 = mul2(fma2(xn[0], d03, mul2(xn[1], d13)), iden);
        const float2 ds4 = mul2(fma2(xn[0], d04, mul2(xn[1], d14)), iden);
        const float2 f0 = txn, f1 = tyn, f3 = mul2(om, xn[4]), f4 = mul2(mul2(om, xn[3]), f2(-1.0f));
        J.T[0][0] = fma2(f0, ds0, f2(1.0f));
        J.T[0][1] = mul2(f0, ds1);
        J.T[0][2] = fma2(f0, ds3, d03);
        J.T[0][3] = fma2(f0, ds4, d04);
        J.T[1][0] = mul2(f1, ds0);
        J.T[1][1] = fma2(f1, ds1, f2(1.0f));
        J.T[1][2] = fma2(f1, ds3, d13);
        J.T[1][3] = fma2(f1, ds4, d14);
        J.T[2][0] = mul2(f3, ds0);
        J.T[2][1] = mul2(f3, ds1);
        J.T[2][2] = fma2(f3, ds3, d33);
        J.T[2][3] = fma2(f3, ds4, d34);
        J.T[3][0] = mul2(f4, ds0);
        J.T[3][1] = mul2(f4, ds1);
        J.T[3][2] = fma2(f4, ds3, d43);
        J.T[3][3] = fma2(f4, ds4, d44);
        J.jz[0] = mul2(lz, ds0);
        J.jz[1] = mul2(lz, ds1);
        J.jz[2] = fma2(lz, ds3, d23);
        J.jz[3] = fma2(lz, ds4, d24);
        J.jzpz = mul2(s, ipt);
    }
    // the tracks the packed path does not cover: the single-track code
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!(slow >> k & 1u)) continue;
        float xs[6], xo[6], sd;
        Jac Jk;
#pragma unroll
        for (int i = 0; i < 6; ++i) xs[i] = lane_of(x[i], k);
        if (propagate(xs, lane_of(qkb, k), r, xo, sd, &Jk)) {
#pragma unroll
            for (int i = 0; i < 6; ++i) set_lane(xn[i], k, xo[i]);
            jac_lane_store(J, k, Jk);
        } else {
            ok &= ~(1u << k);
        }
    }
    return ok;
}

// transport() of both tracks' packed covariances: C <- J C J^T.
__device__ __forceinline__ void transport2(const Jac2 &J, float2 c[21])
{
    constexpr int P[4] = {0, 1, 3, 4};
    float2 A[4][4];  // A = T C[P][P]
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float2 acc = mul2(J.T[k][0], c[pk(P[0], P[m])]);
#pragma unroll
            for (int n = 1; n < 4; ++n) acc = fma2(J.T[k][n], c[pk(P[n], P[m])], acc);
            A[k][m] = acc;
        }
    float2 w[4];  // W = row z of J times C
    float2 w2 = fma2(J.jzpz, c[pk(5, 2)], c[pk(2, 2)]);
    float2 w5 = fma2(J.jzpz, c[pk(5, 5)], c[pk(5, 2)]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float2 acc = fma2(J.jzpz, c[pk(5, P[m])], c[pk(2, P[m])]);
#pragma unroll
        for (int n = 0; n < 4; ++n) acc = fma2(J.jz[n], c[pk(P[n], P[m])], acc);
        w[m] = acc;
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        w2 = fma2(J.jz[n], c[pk(P[n], 2)], w2);
        w5 = fma2(J.jz[n], c[pk(P[n], 5)], w5);
    }
    float2 c5[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float2 acc = mul2(c[pk(5, P[0])], J.T[m][0]);
#pragma unroll
        for (int n = 1; n < 4; ++n) acc = fma2(c[pk(5, P[n])], J.T[m][n], acc);
        c5[m] = acc;
    }
    float2 nc[21];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m <= k; ++m) {
            float2 acc = mul2(A[k][0], J.T[m][0]);
#pragma unroll
            for (int n = 1; n < 4; ++n) acc = fma2(A[k][n], J.T[m][n], acc);
            nc[pk(P[k], P[m])] = acc;
        }
    float2 c22 = w2;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float2 acc = mul2(w[0], J.T[m][0]);
#pragma unroll
        for (int n = 1; n < 4; ++n) acc = fma2(w[n], J.T[m][n], acc);
        nc[pk(2, P[m])] = acc;
        c22 = fma2(J.jz[m], w[m], c22);
    }
    nc[pk(2, 2)] = fma2(J.jzpz, w5, c22);
#pragma unroll
    for (int m = 0; m < 4; ++m) nc[pk(5, P[m])] = c5[m];
    nc[pk(5, 2)] = w5;
    nc[pk(5, 5)] = c[pk(5, 5)];
#pragma unroll
    for (int i = 0; i < 21; ++i) c[i] = nc[i];
}

// add_scattering() of both tracks at radius 1/inv_r (x_over_x0 > 0).
__device__ __forceinline__ void add_scattering2(const float2 xn[6], float inv_r, float x_over_x0, float2 c[21])
{
    const float2 px = xn[3], py = xn[4], pz = xn[5];
    const float2 p2 = fma2(px, px, fma2(py, py, mul2(pz, pz)));
    const float2 ip = rsqrt2(p2);
    const float2 pr = fma2(px, xn[0], mul2(py, xn[1]));
    float2 t2;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float cosi = fabsf(lane_of(pr, k)) * lane_of(ip, k) * inv_r;
        const float xx0 = __fdividef(x_over_x0, cosi);
        const float th = 0.0136f * lane_of(ip, k) * sqrtf(xx0) * (1.0f + 0.038f * __logf(xx0));
        set_lane(t2, k, th * th);
    }
    c[pk(3, 3)] = fma2(t2, fnma2(px, px, p2), c[pk(3, 3)]);
    c[pk(4, 3)] = fnma2(t2, mul2(px, py), c[pk(4, 3)]);
    c[pk(4, 4)] = fma2(t2, fnma2(py, py, p2), c[pk(4, 4)]);
    c[pk(5, 3)] = fnma2(t2, mul2(pz, px), c[pk(5, 3)]);
    c[pk(5, 4)] = fnma2(t2, mul2(pz, py), c[pk(5, 4)]);
    c[pk(5, 5)] = fma2(t2, fnma2(pz, pz, p2), c[pk(5, 5)]);
}

// update() of both tracks with their hits (Section 2.1: 3-D hits with a 3x3
// covariance), in the layer's local frame as the FP32 path of update() does.
// `active` (2 bits): the tracks that have a hit; the others keep their state.
// A track whose update update() would route to extended precision, or whose
// S is not positive definite, is updated by update() itself (slot: its
// per-thread shared-memory scratch).  st[k] receives update()'s status for
// track k (0 FP32, 1 failed, 2 extended precision, 3 PSD repaired), -1 for a
// track without a hit; dchi2 the chi2 increments.
__device__ __forceinline__ void update2(float2 x[6], float2 c[21], const float2 m[3], const float2 v[6],
                                        const Routing &rt, unsigned active, float2 &dchi2, int st[2], float *slot,
                                        int stride)
{
    const float2 ir = rsqrt2(fma2(x[0], x[0], mul2(x[1], x[1])));
    const float2 nx = mul2(x[0], ir), ny = mul2(x[1], ir);
    const float2 nny = mul2(ny, f2(-1.0f));
    const float2 nx2 = mul2(nx, nx), ny2 = mul2(ny, ny), nxy = mul2(nx, ny);
    const float2 m2nxy = mul2(nxy, f2(-2.0f));
    const float2 ctt = fma2(ny2, c[pk(0, 0)], fma2(m2nxy, c[pk(1, 0)], mul2(nx2, c[pk(1, 1)])));
    float2 ct[6];  // ct[i] = C_l[i][t] for i = 2..5
#pragma unroll
    for (int i = 2; i < 6; ++i) ct[i] = fma2(nx, c[pk(i, 1)], mul2(nny, c[pk(i, 0)]));
    const float2 vnn = fma2(nx2, v[0], fma2(mul2(nxy, f2(2.0f)), v[1], mul2(ny2, v[2])));
    const float2 vnt = fma2(nxy, sub2(v[2], v[0]), mul2(sub2(nx2, ny2), v[1]));
    const float2 vtt = fma2(ny2, v[0], fma2(m2nxy, v[1], mul2(nx2, v[2])));
    const float2 vnz = fma2(nx, v[3], mul2(ny, v[4])), vtz = fma2(nx, v[4], mul2(nny, v[3]));
    const float2 a = vnn, b = vnt, cc = add2(ctt, vtt);
    const float2 d = vnz, e = add2(ct[2], vtz), f = add2(c[pk(2, 2)], v[5]);
    const float2 i00 = fnma2(e, e, mul2(cc, f)), i10 = fnma2(b, f, mul2(d, e)), i11 = fnma2(d, d, mul2(a, f));
    const float2 i20 = fnma2(cc, d, mul2(b, e)), i21 = fnma2(a, e, mul2(b, d)), i22 = fnma2(b, b, mul2(a, cc));
    const float2 det = fma2(a, i00, fma2(b, i10, mul2(d, i20)));
    // which tracks take the single-track update (routing, as update() decides it)
    unsigned scalar = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        st[k] = -1;
        if (!(active >> k & 1u)) continue;
        const float ak = lane_of(a, k), ck = lane_of(cc, k), fk = lane_of(f, k), dk = lane_of(det, k);
        const bool pd = ak > 0.0f && lane_of(i22, k) > 0.0f && dk > 0.0f;
        bool slow = !pd;
        if (rt.mode == 1) {
            const float px = lane_of(x[3], k), py = lane_of(x[4], k);
            const float pt2 = px * px + py * py;
            slow = slow || dk <= rt.det_min * (ak * ck * fk) || pt2 < rt.pt_lo * rt.pt_lo || pt2 > rt.pt_hi * rt.pt_hi ||
                   (rt.gain_max > 0.0f && (lane_of(c[0], k) > rt.gain_max * lane_of(v[0], k) ||
                                           lane_of(c[2], k) > rt.gain_max * lane_of(v[2], k) ||
                                           lane_of(c[5], k) > rt.gain_max * lane_of(v[5], k)));
        }
        if (slow) scalar |= 1u << k;
        else st[k] = 0;
    }
    // the single-track update of those tracks, from their predicted state
    float xs[2][6], cs[2][21], ds[2] = {0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!(scalar >> k & 1u)) continue;
        float mk[3], vk[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) xs[k][i] = lane_of(x[i], k);
#pragma unroll
        for (int i = 0; i < 21; ++i) cs[k][i] = lane_of(c[i], k);
#pragma unroll
        for (int i = 0; i < 3; ++i) mk[i] = lane_of(m[i], k);
#pragma unroll
        for (int i = 0; i < 6; ++i) vk[i] = lane_of(v[i], k);
        st[k] = update(xs[k], cs[k], mk, vk, rt, &ds[k], slot, stride);
    }
    // a track without a hit keeps its prediction
    float xk[6], ck[21];
    const int keep = (active & 1u) ? ((active & 2u) ? -1 : 1) : 0;  // the track without a hit, if one
    if (keep >= 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) xk[i] = lane_of(x[i], keep);
#pragma unroll
        for (int i = 0; i < 21; ++i) ck[i] = lane_of(c[i], keep);
    }
    // the FP32 update of both
    const float2 id = rcp2(det);
    const float2 s00 = mul2(i00, id), s10 = mul2(i10, id), s11 = mul2(i11, id);
    const float2 s20 = mul2(i20, id), s21 = mul2(i21, id), s22 = mul2(i22, id);
    const float2 d0 = sub2(m[0], x[0]), d1 = sub2(m[1], x[1]);
    const float2 rn = fma2(nx, d0, mul2(ny, d1)), rt_ = fma2(nx, d1, mul2(nny, d0)), rz = sub2(m[2], x[2]);
    const float2 q0 = fma2(s00, rn, fma2(s10, rt_, mul2(s20, rz)));
    const float2 q1 = fma2(s10, rn, fma2(s11, rt_, mul2(s21, rz)));
    const float2 q2 = fma2(s20, rn, fma2(s21, rt_, mul2(s22, rz)));
    dchi2 = fma2(rn, q0, fma2(rt_, q1, mul2(rz, q2)));
    float2 col_t[6], col_z[6];
    col_t[1] = ctt;
    col_z[1] = ct[2];
    col_t[2] = ct[2];
    col_z[2] = c[pk(2, 2)];
#pragma unroll
    for (int u = 3; u < 6; ++u) {
        col_t[u] = ct[u];
        col_z[u] = c[pk(u, 2)];
    }
    float2 kt[6], kz[6];
#pragma unroll
    for (int u = 1; u < 6; ++u) {
        const float2 k0 = fma2(col_t[u], s10, mul2(col_z[u], s20));
        kt[u] = fma2(col_t[u], s11, mul2(col_z[u], s21));
        kz[u] = fma2(col_t[u], s21, mul2(col_z[u], s22));
        const float2 dxu = fma2(k0, rn, fma2(kt[u], rt_, mul2(kz[u], rz)));
        if (u == 1) {  // t: back to x/y
            x[0] = fma2(nny, dxu, x[0]);
            x[1] = fma2(nx, dxu, x[1]);
        } else {
            x[u] = add2(x[u], dxu);
        }
    }
    const float2 ntt = fnma2(kt[1], col_t[1], fnma2(kz[1], col_z[1], col_t[1]));
#pragma unroll
    for (int u = 2; u < 6; ++u) {
        const float2 nt = fnma2(kt[u], col_t[1], fnma2(kz[u], col_z[1], col_t[u]));
        const float2 nz = fnma2(kt[u], col_t[2], fnma2(kz[u], col_z[2], col_z[u]));
        c[pk(u, 0)] = mul2(nny, nt);
        c[pk(u, 1)] = mul2(nx, nt);
        if (u >= 3) c[pk(u, 2)] = nz;
        else c[pk(2, 2)] = nz;
#pragma unroll
        for (int w = 3; w <= u; ++w) c[pk(u, w)] = fnma2(kt[u], col_t[w], fnma2(kz[u], col_z[w], c[pk(u, w)]));
    }
    c[pk(0, 0)] = mul2(ny2, ntt);
    c[pk(1, 0)] = mul2(mul2(nxy, f2(-1.0f)), ntt);
    c[pk(1, 1)] = mul2(nx2, ntt);
    // the tracks the packed path did not update
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (scalar >> k & 1u) {
#pragma unroll
            for (int i = 0; i < 6; ++i) set_lane(x[i], k, xs[k][i]);
#pragma unroll
            for (int i = 0; i < 21; ++i) set_lane(c[i], k, cs[k][i]);
            set_lane(dchi2, k, ds[k]);
        }
    }
    if (keep >= 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) set_lane(x[i], keep, xk[i]);
#pragma unroll
        for (int i = 0; i < 21; ++i) set_lane(c[i], keep, ck[i]);
        set_lane(dchi2, keep, 0.0f);
    }
}

}  // namespace kf
