// Per-track Kalman-filter arithmetic in registers (Sections 2, 2.1 and 4.2 of
// arXiv:1705.02876): one thread owns one track's state x[6] and its packed
// covariance c[21]; every function below works on those registers.
//
// Packed symmetric storage: lower triangle row by row, index(i,j) = i(i+1)/2+j.
#pragma once

#include <stdint.h>

namespace kf {

constexpr float kField = 0.00299792458f;  // GeV / (cm T)

__host__ __device__ constexpr int pk(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// Divisions on the FP32 path use __fdividef (reciprocal approximation and a
// multiply, within 2 ulp for divisors of magnitude 2^-126..2^126, which every
// divisor here is) in place of the IEEE-rounded sequence.
//
// Propagation result and the non-trivial part of its Jacobian.  With
// P = {x, y, px, py} (state indices 0, 1, 3, 4), J has the block structure
//   J[P][P] = T (4x4), J[z][P] = jz (4), J[z][z] = 1, J[z][pz] = jzpz,
//   J[P][z] = J[P][pz] = 0, J[pz] = e_pz,
// because the crossing of a z-parallel cylinder does not depend on z or pz.
struct Jac {
    float T[4][4];
    float jz[4];
    float jzpz;
};

// Helix propagation to the first forward crossing of radius r (uniform field
// along z; transverse path length s, omega = q k Bz / pT).  Writing
// tau = tan(omega s / 2), the crossing condition |P(s)|^2 = r^2 is the
// quadratic  B' tau^2 + omega u tau - omega^2 D / 4 = 0  with
// u = P.t, w = P x t, D = r^2 - |P|^2, B' = 1 + omega w - omega^2 D / 4.
// Its roots are omega (-u +- sqrt(Q)) / (2 B'), Q = u^2 + D B'.  The root
// rationalised to tau = omega sigma / 2, sigma = D / (u + sqrt(Q)), stays
// exact as omega -> 0 (sigma is then the straight-line path length) and is
// the first crossing whenever u + sqrt(Q) > 0: for B' > 0 the other root lies
// beyond half a turn, for B' < 0 (a start past the circle's closest approach
// to the axis, crossing towards its farthest point) both roots share a sign
// and this one is the smaller.  sin and cos of the turning angle are rational
// in tau, so only one atan (for z) is evaluated.  A start moving inwards with
// u + sqrt(Q) <= 0 takes the general two-root path.  Returns false if the
// cylinder is not reached.
__device__ __forceinline__ bool propagate(const float x[6], float qkb, float r, float xn[6],
                                          float &s_out, Jac *J)
{
    const float px = x[3], py = x[4], pz = x[5];
    const float pt2 = px * px + py * py;
    const float ipt = rsqrtf(pt2);
    const float tx = px * ipt, ty = py * ipt;
    const float om = qkb * ipt;
    const float u = x[0] * tx + x[1] * ty;
    const float w = x[0] * ty - x[1] * tx;
    const float D = r * r - (x[0] * x[0] + x[1] * x[1]);
    const float Bp = 1.0f + om * w - 0.25f * om * om * D;
    const float Qd = u * u + D * Bp;
    if (!(Qd >= 0.0f) || !(pt2 > 0.0f)) return false;
    const float sq = sqrtf(Qd);
    float s, tau, sigma;
    if (u + sq > 0.0f) {
        sigma = __fdividef(D, u + sq);
        tau = 0.5f * om * sigma;
        const float t2 = tau * tau;
        // atan(tau)/tau: its Taylor series sum_k (-t2)^k / (2k+1) to t2^6 for
        // |tau| < 1/4 (truncation below 3e-10), else the library atanf
        float ratio;
        if (t2 < 0.0625f) {
            ratio = fmaf(t2, -1.0f / 13.0f, 1.0f / 11.0f);
            ratio = fmaf(t2, -ratio, 1.0f / 9.0f);
            ratio = fmaf(t2, -ratio, 1.0f / 7.0f);
            ratio = fmaf(t2, -ratio, 1.0f / 5.0f);
            ratio = fmaf(t2, -ratio, 1.0f / 3.0f);
            ratio = fmaf(t2, -ratio, 1.0f);
        } else {
            ratio = atanf(tau) / tau;
        }
        s = sigma * ratio;
    } else {
        // A start moving inwards: both roots of the quadratic, each mapped to
        // its smallest positive path length.
        if (om == 0.0f) return false;
        const float period = 6.283185307179586f / fabsf(om);
        float best = INFINITY;
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            float phi;
            if (Bp != 0.0f) {
                const float tr = om * (-u + sgn * copysignf(sq, om)) / (2.0f * Bp);
                phi = 2.0f * atanf(tr);
            } else {
                phi = sgn < 0 ? 2.0f * atanf(om * D / (4.0f * u)) : copysignf(3.14159265358979f, om);
            }
            float sk = phi / om;
            if (sk <= 0.0f) sk += period;
            best = fminf(best, sk);
        }
        s = best;
        tau = tanf(0.5f * om * s);
        sigma = om != 0.0f ? 2.0f * tau / om : s;
        if (!(s < INFINITY)) return false;
    }
    const float g = __fdividef(1.0f, 1.0f + tau * tau);
    const float a = sigma * g;          // sin(phi) / omega
    const float b = sigma * tau * g;    // (1 - cos(phi)) / omega
    const float sn = 2.0f * tau * g;    // sin(phi)
    const float c = 1.0f - 2.0f * tau * tau * g;  // cos(phi)
    xn[0] = x[0] + tx * a + ty * b;
    xn[1] = x[1] + ty * a - tx * b;
    xn[2] = x[2] + pz * s * ipt;
    xn[3] = px * c + py * sn;
    xn[4] = py * c - px * sn;
    xn[5] = pz;
    s_out = s;
    if (J) {
        const float phi = om * s;
        const float txn = xn[3] * ipt, tyn = xn[4] * ipt;
        // D = dF/dx0 at fixed s (phi depends on pT through omega)
        const float d03 = (a - s * tx * txn) * ipt, d04 = (b - s * ty * txn) * ipt;
        const float d13 = (-b - s * tx * tyn) * ipt, d14 = (a - s * ty * tyn) * ipt;
        const float d33 = c - phi * tx * tyn, d34 = sn - phi * ty * tyn;
        const float d43 = -sn + phi * tx * txn, d44 = c + phi * ty * txn;
        const float lz = pz * ipt;  // dz/ds
        const float d23 = -s * lz * tx * ipt, d24 = -s * lz * ty * ipt;
        // ds/dx0 from the constraint x'^2 + y'^2 = r^2
        const float iden = __fdividef(-1.0f, xn[0] * txn + xn[1] * tyn);
        const float ds0 = xn[0] * iden, ds1 = xn[1] * iden;
        const float ds3 = (xn[0] * d03 + xn[1] * d13) * iden;
        const float ds4 = (xn[0] * d04 + xn[1] * d14) * iden;
        const float f0 = txn, f1 = tyn, f3 = om * xn[4], f4 = -om * xn[3];  // dF/ds on P
        J->T[0][0] = 1.0f + f0 * ds0; J->T[0][1] = f0 * ds1; J->T[0][2] = d03 + f0 * ds3; J->T[0][3] = d04 + f0 * ds4;
        J->T[1][0] = f1 * ds0; J->T[1][1] = 1.0f + f1 * ds1; J->T[1][2] = d13 + f1 * ds3; J->T[1][3] = d14 + f1 * ds4;
        J->T[2][0] = f3 * ds0; J->T[2][1] = f3 * ds1; J->T[2][2] = d33 + f3 * ds3; J->T[2][3] = d34 + f3 * ds4;
        J->T[3][0] = f4 * ds0; J->T[3][1] = f4 * ds1; J->T[3][2] = d43 + f4 * ds3; J->T[3][3] = d44 + f4 * ds4;
        J->jz[0] = lz * ds0; J->jz[1] = lz * ds1; J->jz[2] = d23 + lz * ds3; J->jz[3] = d24 + lz * ds4;
        J->jzpz = s * ipt;
    }
    return true;
}

// C <- J C J^T using the block structure of J (178 FMA instead of 432 for a
// dense 6x6 triple product on the packed lower triangle).
__device__ __forceinline__ void transport(const Jac &J, float c[21])
{
    constexpr int P[4] = {0, 1, 3, 4};
    float A[4][4];  // A = T C[P][P]
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float acc = 0.0f;
#pragma unroll
            for (int n = 0; n < 4; ++n) acc = fmaf(J.T[k][n], c[pk(P[n], P[m])], acc);
            A[k][m] = acc;
        }
    float w[4], w2 = c[pk(2, 2)], w5 = c[pk(5, 2)];  // W = row z of J times C
    w2 = fmaf(J.jzpz, c[pk(5, 2)], w2);
    w5 = fmaf(J.jzpz, c[pk(5, 5)], c[pk(5, 2)]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float acc = fmaf(J.jzpz, c[pk(5, P[m])], c[pk(2, P[m])]);
#pragma unroll
        for (int n = 0; n < 4; ++n) acc = fmaf(J.jz[n], c[pk(P[n], P[m])], acc);
        w[m] = acc;
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        w2 = fmaf(J.jz[n], c[pk(P[n], 2)], w2);
        w5 = fmaf(J.jz[n], c[pk(P[n], 5)], w5);
    }
    float c5[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float acc = 0.0f;
#pragma unroll
        for (int n = 0; n < 4; ++n) acc = fmaf(c[pk(5, P[n])], J.T[m][n], acc);
        c5[m] = acc;
    }
    float nc[21];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m <= k; ++m) {
            float acc = 0.0f;
#pragma unroll
            for (int n = 0; n < 4; ++n) acc = fmaf(A[k][n], J.T[m][n], acc);
            nc[pk(P[k], P[m])] = acc;
        }
    float c22 = w2;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float acc = 0.0f;
#pragma unroll
        for (int n = 0; n < 4; ++n) acc = fmaf(w[n], J.T[m][n], acc);
        nc[pk(2, P[m])] = acc;
        c22 = fmaf(J.jz[m], w[m], c22);
    }
    nc[pk(2, 2)] = fmaf(J.jzpz, w5, c22);
#pragma unroll
    for (int m = 0; m < 4; ++m) nc[pk(5, P[m])] = c5[m];
    nc[pk(5, 2)] = w5;
    nc[pk(5, 5)] = c[pk(5, 5)];
#pragma unroll
    for (int i = 0; i < 21; ++i) c[i] = nc[i];
}

// theta0^2 of the Highland formula (beta = 1) for a thin layer of x_over_x0
// radiation lengths crossed at xn on radius 1/inv_r (path x_over_x0 /
// |cos(incidence)|); p2 receives |p|^2.
__device__ __forceinline__ float scattering_theta2(const float xn[6], float inv_r, float x_over_x0, float &p2)
{
    const float px = xn[3], py = xn[4], pz = xn[5];
    p2 = px * px + py * py + pz * pz;
    const float ip = rsqrtf(p2);
    const float cosi = fabsf(px * xn[0] + py * xn[1]) * ip * inv_r;
    const float xx0 = __fdividef(x_over_x0, cosi);
    const float th = 0.0136f * ip * sqrtf(xx0) * (1.0f + 0.038f * __logf(xx0));
    return th * th;
}

// Multiple scattering of a thin layer: Q = theta0^2 (|p|^2 I3 - p p^T) added
// to the momentum block.
__device__ __forceinline__ void add_scattering(const float xn[6], float inv_r, float x_over_x0, float c[21])
{
    if (!(x_over_x0 > 0.0f)) return;
    const float px = xn[3], py = xn[4], pz = xn[5];
    float p2;
    const float t2 = scattering_theta2(xn, inv_r, x_over_x0, p2);
    c[pk(3, 3)] = fmaf(t2, p2 - px * px, c[pk(3, 3)]);
    c[pk(4, 3)] = fmaf(-t2, px * py, c[pk(4, 3)]);
    c[pk(4, 4)] = fmaf(t2, p2 - py * py, c[pk(4, 4)]);
    c[pk(5, 3)] = fmaf(-t2, pz * px, c[pk(5, 3)]);
    c[pk(5, 4)] = fmaf(-t2, pz * py, c[pk(5, 4)]);
    c[pk(5, 5)] = fmaf(t2, p2 - pz * pz, c[pk(5, 5)]);
}

// The extended-precision paths are out of line and rare.  A non-inlined
// function's registers count towards the kernel's allocation, so these work
// from a per-thread slot of shared memory ([kSlotSize][stride] floats,
// thread-major so that a warp's accesses hit distinct banks), reading and
// writing the covariance one row at a time: the kernel keeps the register
// budget of the FP32 main path.
constexpr int kSlotX = 0, kSlotC = 6, kSlotM = 27, kSlotV = 30, kSlotChi2 = 36, kSlotSize = 37;

__device__ __forceinline__ void slot_write(float *slot, int stride, const float x[6], const float c[21], const float m[3],
                                           const float v[6])
{
#pragma unroll
    for (int i = 0; i < 6; ++i) slot[(kSlotX + i) * stride] = x[i];
#pragma unroll
    for (int i = 0; i < 21; ++i) slot[(kSlotC + i) * stride] = c[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) slot[(kSlotM + i) * stride] = m[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) slot[(kSlotV + i) * stride] = v[i];
}

struct SlotRef {
    float *p;
    int stride;
    __device__ __forceinline__ float &x(int i) const { return p[(kSlotX + i) * stride]; }
    __device__ __forceinline__ float &c(int i, int j) const { return p[(kSlotC + pk(i, j)) * stride]; }
    __device__ __forceinline__ float &m(int i) const { return p[(kSlotM + i) * stride]; }
    __device__ __forceinline__ float &v(int i) const { return p[(kSlotV + i) * stride]; }
    __device__ __forceinline__ float &chi2() const { return p[kSlotChi2 * stride]; }
};

// The slow paths work in the same local frame as the FP32 update (below):
// n = (x, y)/|(x, y)| at the predicted position, t = z x n.  The slot holds
// the Cartesian covariance, whose radial row is the FP32 rounding residue of
// an exact zero; the local block over (t, z, px, py, pz) drops it, exactly as
// the FP32 path does (in Cartesian form that residue, of order 1e-7 C_tt, can
// rival a fine hit's V_nn and bias the update).  The slot's 21 covariance
// floats are rewritten in place as the 15 of the local block (packed, local
// index u = 0 t, 1 z, 2 px, 3 py, 4 pz) and back: every value is streamed
// through the slot so that these out-of-line paths keep the register budget
// of the FP32 main path.  After the update the Cartesian covariance is
// rebuilt from the local block (x = -n_y t, y = n_x t), so its radial row is
// exactly zero again.
template <class R>
__device__ __forceinline__ void slot_to_local(const SlotRef &sl, R nx, R ny)
{
    float *c = sl.p + kSlotC * sl.stride;
    auto C = [&](int i, int j) -> float & { return c[pk(i, j) * sl.stride]; };
    const float ltt = (float)(ny * ny * (R)C(0, 0) - 2 * nx * ny * (R)C(1, 0) + nx * nx * (R)C(1, 1));
    float lkt[4];
#pragma unroll
    for (int k = 2; k < 6; ++k) lkt[k - 2] = (float)(nx * (R)C(k, 1) - ny * (R)C(k, 0));
    // increasing local position: every source lies above its destination and
    // is read before it is overwritten
#pragma unroll 1
    for (int u = 1; u < 5; ++u)
#pragma unroll 1
        for (int w = 1; w <= u; ++w) C(u, w) = C(u + 1, w + 1);
    C(0, 0) = ltt;
#pragma unroll
    for (int u = 1; u < 5; ++u) C(u, 0) = lkt[u - 1];
}

template <class R>
__device__ __forceinline__ void slot_to_cartesian(const SlotRef &sl, R nx, R ny)
{
    float *c = sl.p + kSlotC * sl.stride;
    auto C = [&](int i, int j) -> float & { return c[pk(i, j) * sl.stride]; };
    // decreasing Cartesian position: every source lies below its destination
#pragma unroll 1
    for (int i = 5; i >= 2; --i) {
#pragma unroll 1
        for (int j = i; j >= 2; --j) C(i, j) = C(i - 1, j - 1);
        const R lt = (R)C(i - 1, 0);
        C(i, 1) = (float)(nx * lt);
        C(i, 0) = (float)(-ny * lt);
    }
    const R ltt = (R)C(0, 0);
    C(1, 1) = (float)(nx * nx * ltt);
    C(1, 0) = (float)(-nx * ny * ltt);
    C(0, 0) = (float)(ny * ny * ltt);
}

// C_l -= K C_l[{t, z}, :] in place on the slot's local block, row u's gain
// (kt[u], kz[u]) against the original t and z columns: rows and, within a
// row, columns descending read only entries not yet rewritten, except the
// original (z, t) entry, kept for row t.
template <class R>
__device__ __forceinline__ void slot_local_downdate(const SlotRef &sl, const R kt[5], const R kz[5])
{
    float *c = sl.p + kSlotC * sl.stride;
    auto C = [&](int i, int j) -> float & { return c[pk(i, j) * sl.stride]; };
    const R zt = (R)C(1, 0);
#pragma unroll 1
    for (int u = 4; u >= 0; --u)
#pragma unroll 1
        for (int w = u; w >= 0; --w) {
            const R ctw = (R)C(w, 0);
            const R czw = w > 0 ? (R)C(w, 1) : u > 0 ? (R)C(1, 0) : zt;
            C(u, w) = (float)((R)C(u, w) - (kt[u] * ctw + kz[u] * czw));
        }
}

// Update in FP64 on the slot, in the local frame: S (n, t, z) and S^-1 by
// adjugate, the gain's five non-radial rows, x += K r, C -= K C[{t, z}, :]
// on the local block, chi2 = r^T S^-1 r; then the PSD repair: a local
// variance that cancellation drove to zero or below is clamped to 1e-12 of
// the local trace (correlations are left alone).  Returns 2, 3 (repaired) or
// 1 (S not positive definite).
static __device__ __noinline__ int update_fp64(float *slot_p, int stride)
{
    const SlotRef sl{slot_p, stride};
    const double X0 = sl.x(0), X1 = sl.x(1);
    const double ir = 1.0 / sqrt(X0 * X0 + X1 * X1);
    const double nx = X0 * ir, ny = X1 * ir;
    slot_to_local<double>(sl, nx, ny);
    auto L = [&](int i, int j) -> float & { return sl.c(i, j); };  // the slot's local block
    const double v0 = sl.v(0), v1 = sl.v(1), v2 = sl.v(2), v3 = sl.v(3), v4 = sl.v(4), v5 = sl.v(5);
    const double a = nx * nx * v0 + 2.0 * nx * ny * v1 + ny * ny * v2;
    const double b = nx * ny * (v2 - v0) + (nx * nx - ny * ny) * v1;
    const double cc = (double)L(0, 0) + (ny * ny * v0 - 2.0 * nx * ny * v1 + nx * nx * v2);
    const double d = nx * v3 + ny * v4, e = (double)L(1, 0) + (nx * v4 - ny * v3), f = (double)L(1, 1) + v5;
    const double i00 = cc * f - e * e, i10 = d * e - b * f, i11 = a * f - d * d;
    const double i20 = b * e - cc * d, i21 = b * d - a * e, i22 = a * cc - b * b;
    const double det = a * i00 + b * i10 + d * i20;
    if (!(a > 0.0) || !(i22 > 0.0) || !(det > 0.0)) {
        slot_to_cartesian<double>(sl, nx, ny);
        return 1;
    }
    const double id = 1.0 / det;
    const double s00 = i00 * id, s10 = i10 * id, s11 = i11 * id, s20 = i20 * id, s21 = i21 * id, s22 = i22 * id;
    const double d0 = (double)sl.m(0) - X0, d1 = (double)sl.m(1) - X1;
    const double rn = nx * d0 + ny * d1, rt = nx * d1 - ny * d0, rz = (double)sl.m(2) - sl.x(2);
    const double q0 = s00 * rn + s10 * rt + s20 * rz, q1 = s10 * rn + s11 * rt + s21 * rz;
    const double q2 = s20 * rn + s21 * rt + s22 * rz;
    sl.chi2() = (float)(rn * q0 + rt * q1 + rz * q2);
    double kt[5], kz[5];
#pragma unroll 1
    for (int u = 0; u < 5; ++u) {
        const double ct = L(u, 0), cz = L(u, 1);
        kt[u] = ct * s11 + cz * s21;
        kz[u] = ct * s21 + cz * s22;
        const double dx = (ct * s10 + cz * s20) * rn + kt[u] * rt + kz[u] * rz;
        if (u == 0) {
            sl.x(0) = (float)(X0 - ny * dx);
            sl.x(1) = (float)(X1 + nx * dx);
        } else {
            sl.x(u + 1) = (float)((double)sl.x(u + 1) + dx);
        }
    }
    slot_local_downdate<double>(sl, kt, kz);
    double tr = 0.0;
#pragma unroll 1
    for (int u = 0; u < 5; ++u) tr += fabs((double)L(u, u));
    bool rep = false;
#pragma unroll 1
    for (int u = 0; u < 5; ++u)
        if (!(L(u, u) > 0.0f)) {
            L(u, u) = (float)(1e-12 * tr);
            rep = true;
        }
    slot_to_cartesian<double>(sl, nx, ny);
    return rep ? 3 : 2;
}

// Float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, about 48
// significant bits carried on the FP32 pipe.  Error-free transformations
// (Knuth's two-sum, Dekker's fast two-sum, the FMA two-product) use the _rn
// intrinsics, which the compiler never contracts or reassociates.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const ff p = two_prod(x.hi, y.hi);
    return fast_two_sum(p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo)));
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
// a*b - c*d for float-float operands
__device__ __forceinline__ ff ff_det2(ff a, ff b, ff c, ff d) { return ff_add(ff_mul(a, b), ff_neg(ff_mul(c, d))); }
// sum_k s_k * c_k with float-float s and plain float c, accurate to float-float
__device__ __forceinline__ ff ff_dot3(ff s0, ff s1, ff s2, float c0, float c1, float c2)
{
    const ff p0 = two_prod(s0.hi, c0), p1 = two_prod(s1.hi, c1), p2 = two_prod(s2.hi, c2);
    const ff t0 = two_sum(p0.hi, p1.hi);
    const ff t1 = two_sum(t0.hi, p2.hi);
    float err = __fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, __fadd_rn(t0.lo, t1.lo)));
    err = __fmaf_rn(s0.lo, c0, __fmaf_rn(s1.lo, c1, __fmaf_rn(s2.lo, c2, err)));
    return fast_two_sum(t1.hi, err);
}

// Update on the slot with the gain formed in float-float, in the local frame
// of update_fp64: S (n, t, z) from the FP32 local entries (the entries that
// add C and V exact two-sums), S^-1 by adjugate / determinant, the gain's rows
// (C_ut, C_uz) S^-1 rounded to FP32, x += K r and C -= K C[{t, z}, :] in FP32;
// chi2 = r^T S^-1 r.  Returns 2, or 1 if S is not positive definite.
static __device__ __noinline__ int update_ff(float *slot_p, int stride)
{
    const SlotRef sl{slot_p, stride};
    const float X0 = sl.x(0), X1 = sl.x(1);
    const float ir = rsqrtf(X0 * X0 + X1 * X1);
    const float nx = X0 * ir, ny = X1 * ir;
    slot_to_local<float>(sl, nx, ny);
    auto L = [&](int i, int j) -> float & { return sl.c(i, j); };
    const float v0 = sl.v(0), v1 = sl.v(1), v2 = sl.v(2), v3 = sl.v(3), v4 = sl.v(4);
    const ff a{fmaf(nx * nx, v0, fmaf(2.0f * nx * ny, v1, ny * ny * v2)), 0.0f};
    const ff b{fmaf(nx * ny, v2 - v0, (nx * nx - ny * ny) * v1), 0.0f};
    const ff d{fmaf(nx, v3, ny * v4), 0.0f};
    const ff cc = two_sum(L(0, 0), fmaf(ny * ny, v0, fmaf(-2.0f * nx * ny, v1, nx * nx * v2)));
    const ff e = two_sum(L(1, 0), fmaf(nx, v4, -ny * v3)), f = two_sum(L(1, 1), sl.v(5));
    const ff i00 = ff_det2(cc, f, e, e), i10 = ff_det2(d, e, b, f), i11 = ff_det2(a, f, d, d);
    const ff i20 = ff_det2(b, e, cc, d), i21 = ff_det2(b, d, a, e), i22 = ff_det2(a, cc, b, b);
    const ff det = ff_add(ff_mul(a, i00), ff_add(ff_mul(b, i10), ff_mul(d, i20)));
    if (!(a.hi > 0.0f) || !(i22.hi > 0.0f) || !(det.hi > 0.0f)) {
        slot_to_cartesian<float>(sl, nx, ny);
        return 1;
    }
    // 1/det: one Newton step on the FP32 reciprocal, r + r (1 - det r)
    const float rc = 1.0f / det.hi;
    const ff one_minus = ff_add(ff{1.0f, 0.0f}, ff_neg(ff_mul(det, ff{rc, 0.0f})));
    const ff id = ff_add(ff{rc, 0.0f}, ff_mul(one_minus, ff{rc, 0.0f}));
    const ff s00 = ff_mul(i00, id), s10 = ff_mul(i10, id), s11 = ff_mul(i11, id);
    const ff s20 = ff_mul(i20, id), s21 = ff_mul(i21, id), s22 = ff_mul(i22, id);
    const float d0 = sl.m(0) - X0, d1 = sl.m(1) - X1;
    const ff rn = two_sum(nx * d0, ny * d1), rt = two_sum(nx * d1, -ny * d0), rz = two_sum(sl.m(2), -sl.x(2));
    const ff q0 = ff_add(ff_mul(s00, rn), ff_add(ff_mul(s10, rt), ff_mul(s20, rz)));
    const ff q1 = ff_add(ff_mul(s10, rn), ff_add(ff_mul(s11, rt), ff_mul(s21, rz)));
    const ff q2 = ff_add(ff_mul(s20, rn), ff_add(ff_mul(s21, rt), ff_mul(s22, rz)));
    const ff chi = ff_add(ff_mul(rn, q0), ff_add(ff_mul(rt, q1), ff_mul(rz, q2)));
    sl.chi2() = __fadd_rn(chi.hi, chi.lo);
    const float rrn = __fadd_rn(rn.hi, rn.lo), rrt = __fadd_rn(rt.hi, rt.lo), rrz = __fadd_rn(rz.hi, rz.lo);
    const ff zero{0.0f, 0.0f};
    float kt[5], kz[5];
    for (int u = 0; u < 5; ++u) {
        const float ct = L(u, 0), cz = L(u, 1);
        const ff knf = ff_dot3(s10, s20, zero, ct, cz, 0.0f);
        const ff ktf = ff_dot3(s11, s21, zero, ct, cz, 0.0f);
        const ff kzf = ff_dot3(s21, s22, zero, ct, cz, 0.0f);
        kt[u] = __fadd_rn(ktf.hi, ktf.lo);
        kz[u] = __fadd_rn(kzf.hi, kzf.lo);
        const float dx = fmaf(__fadd_rn(knf.hi, knf.lo), rrn, fmaf(kt[u], rrt, kz[u] * rrz));
        if (u == 0) {
            sl.x(0) = fmaf(-ny, dx, X0);
            sl.x(1) = fmaf(nx, dx, X1);
        } else {
            sl.x(u + 1) += dx;
        }
    }
    slot_local_downdate<float>(sl, kt, kz);
    slot_to_cartesian<float>(sl, nx, ny);
    return 2;
}

static __device__ __noinline__ int update_ext(float *slot, int stride, int kind)
{
    return kind == 2 ? update_fp64(slot, stride) : update_ff(slot, stride);
}

struct Routing {
    int mode;        // 0 FP32, 1 routed
    float det_min;   // 27 / (4 cond_max): the least det of S's correlation matrix done in FP32
    float pt_lo, pt_hi;
    float gain_max;  // information-gain threshold: C_ii / V_ii above it routes the gain
};

// Update with a 3-D hit (Section 2.1: 3x3 measurement covariance V).
//   S = C_xx + V, K = C[:, 0:3] S^-1, x += K r, C -= K C[0:3, :],
//   dchi2 = r^T S^-1 r.
//
// The FP32 path works in the local frame of the layer at the predicted
// position: n = (x, y, 0)/|(x, y)|, t = z x n, z.  Transport onto the cylinder
// leaves the covariance the exact null vector n (the crossing cannot move off
// the surface), so in x/y the exactly known radial direction and the
// uncertain tangential one share every entry and FP32 cannot resolve the gain
// of an update that shrinks the covariance by orders of magnitude (a hit
// after a diffuse seed).  In (n, t, z) they decouple: C's radial row is zero
// (its rounding residue is dropped), S = [[V_nn, V_nt, V_nz], [V_nt, C_tt +
// V_tt, C_tz + V_tz], [V_nz, C_tz + V_tz, C_zz + V_zz]], the gain's radial
// row is zero, and only the five non-radial rows (t, z, px, py, pz) are
// updated, each from the t and z columns.  dx and C are rotated back to x/y.
// Routing (mode 1):
//   * the whole update is redone in FP64 with a PSD repair (update_fp64) when
//     S is not positive definite in FP32, when the determinant of its
//     correlation matrix R = D^-1/2 S D^-1/2 (D = diag S) is below
//     27 / (4 cond_max), which keeps cond_2(R) <= cond_max on the FP32 path,
//     or when pT lies outside [pt_lo, pt_hi];
//   * with gain_max > 0, the gain is formed in float-float (update_ff) when
//     C_ii > gain_max V_ii for some i.  Float-float runs on the FP32 pipe,
//     which on this part is 64 times wider than the FP64 one.
// Returns 0 updated in FP32, 2 updated with extended-precision arithmetic,
// 3 updated in FP64 with a PSD repair, 1 failed (S not positive definite).
__device__ __forceinline__ int update(float x[6], float c[21], const float m[3], const float v[6],
                                      const Routing &rt, float *dchi2, float *slot, int stride)
{
    const float ir = rsqrtf(x[0] * x[0] + x[1] * x[1]);
    const float nx = x[0] * ir, ny = x[1] * ir;
    // t column of C in the local frame: C_it = -ny C_i0 + nx C_i1 (i >= 2),
    // C_tt = t^T C_xy t; the z column is C's own
    const float ctt = fmaf(ny * ny, c[pk(0, 0)], fmaf(-2.0f * nx * ny, c[pk(1, 0)], nx * nx * c[pk(1, 1)]));
    float ct[6];  // ct[i] = C_l[i][t] for i = 2..5
#pragma unroll
    for (int i = 2; i < 6; ++i) ct[i] = fmaf(nx, c[pk(i, 1)], -ny * c[pk(i, 0)]);
    const float vnn = fmaf(nx * nx, v[0], fmaf(2.0f * nx * ny, v[1], ny * ny * v[2]));
    const float vnt = fmaf(nx * ny, v[2] - v[0], (nx * nx - ny * ny) * v[1]);
    const float vtt = fmaf(ny * ny, v[0], fmaf(-2.0f * nx * ny, v[1], nx * nx * v[2]));
    const float vnz = fmaf(nx, v[3], ny * v[4]), vtz = fmaf(nx, v[4], -ny * v[3]);
    const float a = vnn, b = vnt, cc = ctt + vtt;
    const float d = vnz, e = ct[2] + vtz, f = c[pk(2, 2)] + v[5];
    const float i00 = cc * f - e * e, i10 = d * e - b * f, i11 = a * f - d * d;
    const float i20 = b * e - cc * d, i21 = b * d - a * e, i22 = a * cc - b * b;
    const float det = fmaf(a, i00, fmaf(b, i10, d * i20));
    const bool pd = a > 0.0f && i22 > 0.0f && det > 0.0f;
    int kind = 0;
    if (rt.mode == 1) {
        // S's correlation matrix R = D^-1/2 S D^-1/2 (D = diag S): the rounding
        // of the adjugate's cofactors grows with its condition, not with the
        // spread of S's diagonal (V_nn << C_zz is harmless).  With eigenvalues
        // summing to 3, det R >= 27 / (4 cond_max) bounds cond_2(R) by cond_max.
        const bool ill = !pd || det <= rt.det_min * (a * cc * f);
        const float pt2 = x[3] * x[3] + x[4] * x[4];
        if (ill || pt2 < rt.pt_lo * rt.pt_lo || pt2 > rt.pt_hi * rt.pt_hi)
            kind = 2;
        else if (rt.gain_max > 0.0f &&
                 (c[0] > rt.gain_max * v[0] || c[2] > rt.gain_max * v[2] || c[5] > rt.gain_max * v[5]))
            kind = 1;
    } else if (!pd) {
        return 1;
    }
    if (kind) {
        slot_write(slot, stride, x, c, m, v);
        const int st = update_ext(slot, stride, kind);
        if (st == 1) return 1;
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = slot[(kSlotX + i) * stride];
#pragma unroll
        for (int i = 0; i < 21; ++i) c[i] = slot[(kSlotC + i) * stride];
        *dchi2 = slot[kSlotChi2 * stride];
        return st;
    }
    const float id = __fdividef(1.0f, det);
    const float s00 = i00 * id, s10 = i10 * id, s11 = i11 * id, s20 = i20 * id, s21 = i21 * id, s22 = i22 * id;
    const float d0 = m[0] - x[0], d1 = m[1] - x[1];
    const float rn = fmaf(nx, d0, ny * d1), rt_ = fmaf(nx, d1, -ny * d0), rz = m[2] - x[2];
    const float q0 = fmaf(s00, rn, fmaf(s10, rt_, s20 * rz));
    const float q1 = fmaf(s10, rn, fmaf(s11, rt_, s21 * rz));
    const float q2 = fmaf(s20, rn, fmaf(s21, rt_, s22 * rz));
    *dchi2 = fmaf(rn, q0, fmaf(rt_, q1, rz * q2));
    // rows u = t, z, px, py, pz (state indices 1..5 of the local frame):
    // col_t[u] = C_l[u][t], col_z[u] = C_l[u][z], both before the update
    float col_t[6], col_z[6];
    col_t[1] = ctt;
    col_z[1] = ct[2];
    col_t[2] = ct[2];
    col_z[2] = c[pk(2, 2)];
#pragma unroll
    for (int u = 3; u < 6; ++u) {
        col_t[u] = ct[u];
        col_z[u] = c[pk(u, 2)];
    }
    // K_u = (C_ut, C_uz) S^-1[{t, z}, :]; the radial row of K is zero
    float kt[6], kz[6];
#pragma unroll
    for (int u = 1; u < 6; ++u) {
        const float k0 = fmaf(col_t[u], s10, col_z[u] * s20);
        kt[u] = fmaf(col_t[u], s11, col_z[u] * s21);
        kz[u] = fmaf(col_t[u], s21, col_z[u] * s22);
        const float dxu = fmaf(k0, rn, fmaf(kt[u], rt_, kz[u] * rz));
        if (u == 1) {  // t: back to x/y
            x[0] = fmaf(-ny, dxu, x[0]);
            x[1] = fmaf(nx, dxu, x[1]);
        } else {
            x[u] += dxu;
        }
    }
    // C'_uw = C_uw - K_ut C_tw - K_uz C_zw over the non-radial 5x5 block
    const float ntt = fmaf(-kt[1], col_t[1], fmaf(-kz[1], col_z[1], col_t[1]));
#pragma unroll
    for (int u = 2; u < 6; ++u) {
        const float nt = fmaf(-kt[u], col_t[1], fmaf(-kz[u], col_z[1], col_t[u]));  // C'_u t
        const float nz = fmaf(-kt[u], col_t[2], fmaf(-kz[u], col_z[2], col_z[u]));  // C'_u z
        c[pk(u, 0)] = -ny * nt;
        c[pk(u, 1)] = nx * nt;
        if (u >= 3) c[pk(u, 2)] = nz;
        else c[pk(2, 2)] = nz;
#pragma unroll
        for (int w = 3; w <= u; ++w) c[pk(u, w)] = fmaf(-kt[u], col_t[w], fmaf(-kz[u], col_z[w], c[pk(u, w)]));
    }
    c[pk(0, 0)] = ny * ny * ntt;
    c[pk(1, 0)] = -nx * ny * ntt;
    c[pk(1, 1)] = nx * nx * ntt;
    return 0;
}

}  // namespace kf
