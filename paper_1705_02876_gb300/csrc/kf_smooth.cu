// The Kalman smoother on sm_103a: the forward fit (Sections 2, 2.1 and 4.2)
// followed, in the same thread, by the backward Rauch-Tung-Striebel pass that
// gives at every layer the estimate using all of the track's hits (Section 2
// names a final fit with a smoother as the step after building).
//
// On a cylinder the predicted and filtered covariances are singular (the
// crossing cannot leave the surface: the radial direction n of the predicted
// crossing carries no variance), so the backward pass works in each layer's
// local coordinates (t, z, px, py, pz), t = z x n, where they are 5x5 and
// positive definite.  With G the Jacobian from layer l's local coordinates to
// layer l+1's and Q the scattering noise added at layer l+1:
//   A_l  = Cf_l G^T Cp_{l+1}^-1 = G^-1 (I - Q Cp_{l+1}^-1)  (Cp = G Cf G^T + Q),
//   xs_l = xf_l + R_l A_l (xs_{l+1} - xp_{l+1}),
//   Cs_l = Cf_l + A_l (Cs_{l+1} - Cp_{l+1}) A_l^T.
// The second form is the one computed: G^-1 is a 3x3 inverse of the
// transport's transverse block (well conditioned), and Cp^-1 (a Cholesky
// factorisation of Cp scaled to unit diagonal) only multiplies the scattering
// noise, so the FP32 rounding that Cp's correlations amplify enters A scaled
// by |Q| / |Cp|; the other factor is never formed.  The forward pass writes
// the filtered state and local covariance (with the frame) of every layer to
// the output arrays; the backward pass reads them, recomputes the prediction
// of layer l+1 from the filtered estimate of layer l (the same propagation,
// transport and scattering as the forward pass, on the same state bits: xp, G
// and Q come out identical, Cp differs by the rounding of the stored local
// covariance), and overwrites them with the smoothed ones.  Nothing else is
// stored: a track's filtered estimates (108 B per layer) are read back while
// still in L2, and each output line reaches DRAM once, smoothed.
#include "kf.h"
#include "kf_api_internal.h"
#include "kf_fit.cuh"

namespace kf {

struct SmoothState {};  // the smoother keeps no scratch

void destroy_smooth_state(SmoothState *s) { delete s; }

namespace {

struct SmoothIO {
    int64_t T;
    const float *seed_state, *seed_cov;
    const int8_t *charge;
    const float *hit_pos, *hit_cov;
    const uint32_t *hit_mask;
    float *out_state, *out_cov;  // [L][6][T], [L][21][T]
    int16_t *out_reached;
    uint32_t *out_flags;
};

__device__ __forceinline__ void local_of(const float c[21], float nx, float ny, float cl[15])
{
    cl[0] = fmaf(ny * ny, c[pk(0, 0)], fmaf(-2.0f * nx * ny, c[pk(1, 0)], nx * nx * c[pk(1, 1)]));
#pragma unroll
    for (int k = 2; k < 6; ++k) cl[pk(k - 1, 0)] = fmaf(nx, c[pk(k, 1)], -ny * c[pk(k, 0)]);
#pragma unroll
    for (int i = 2; i < 6; ++i)
#pragma unroll
        for (int j = 2; j <= i; ++j) cl[pk(i - 1, j - 1)] = c[pk(i, j)];
}

__device__ __forceinline__ float cart_of(const float cl[15], float nx, float ny, int i, int j)
{
    const float wi = i == 0 ? -ny : nx, wj = j == 0 ? -ny : nx;
    if (i < 2 && j < 2) return wi * wj * cl[0];
    if (i < 2) return wi * cl[pk(j - 1, 0)];
    if (j < 2) return wj * cl[pk(i - 1, 0)];
    return cl[pk(i - 1, j - 1)];
}

// The 13 non-trivial entries of the local Jacobian from frame n0 to frame n1
// (rows t, z, px, py, pz; columns the same):
//   t'  = M00 t + M01 px + M02 py,  px' = M10 t + M11 px + M12 py,
//   py' = M20 t + M21 px + M22 py,  z' = z + mz0 t + mz1 px + mz2 py + jp pz,
//   pz' = pz;  stored as M (9, row-major), mz (3), jp.
__device__ __forceinline__ void local_jacobian(const Jac &J, float nx0, float ny0, float nx1, float ny1, float g[13])
{
    float a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = fmaf(nx1, J.T[1][k], -ny1 * J.T[0][k]);
    g[0] = fmaf(nx0, a[1], -ny0 * a[0]);
    g[1] = a[2];
    g[2] = a[3];
#pragma unroll
    for (int r = 1; r < 3; ++r) {
        g[3 * r] = fmaf(nx0, J.T[r + 1][1], -ny0 * J.T[r + 1][0]);
        g[3 * r + 1] = J.T[r + 1][2];
        g[3 * r + 2] = J.T[r + 1][3];
    }
    g[9] = fmaf(nx0, J.jz[1], -ny0 * J.jz[0]);
    g[10] = J.jz[2];
    g[11] = J.jz[3];
    g[12] = J.jzpz;
}

// The scattering noise of layer l on the momentum block, packed (px,px)
// (py,px) (py,py) (pz,px) (pz,py) (pz,pz): theta0^2 (|p|^2 I3 - p p^T).
__device__ __forceinline__ void scattering_q6(const float xn[6], float inv_r, float x_over_x0, float q6[6])
{
#pragma unroll
    for (int i = 0; i < 6; ++i) q6[i] = 0.0f;
    if (!(x_over_x0 > 0.0f)) return;
    float p2;
    const float t2 = scattering_theta2(xn, inv_r, x_over_x0, p2);
    const float px = xn[3], py = xn[4], pz = xn[5];
    q6[0] = t2 * (p2 - px * px);
    q6[1] = -t2 * px * py;
    q6[2] = t2 * (p2 - py * py);
    q6[3] = -t2 * pz * px;
    q6[4] = -t2 * pz * py;
    q6[5] = t2 * (p2 - pz * pz);
}

// Registers capped at 128 (four blocks, 16 warps per SM) with a small spill:
// 2.23 ms on the fit workload against 2.46 ms uncapped (237 registers, eight
// warps); caps of 102 and 85 registers spill more and are slower.
__global__ void __launch_bounds__(128, 4) smooth_kernel(const FitGeom g, const Routing rt, const SmoothIO io)
{
    extern __shared__ float slots[];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= io.T) return;
    const int64_t T = io.T;
    const int L = g.L;
    float *slot = slots + threadIdx.x;
    const int stride = blockDim.x;
    auto ost = [&](int l, int i) -> float & { return io.out_state[((int64_t)l * 6 + i) * T + t]; };
    auto ocv = [&](int l, int i) -> float & { return io.out_cov[((int64_t)l * 21 + i) * T + t]; };

    // ---- forward: the fit, keeping every layer
    float x[6], c[21];
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        x[i] = __ldcs(io.seed_state + i * T + t);
        finite = finite && isfinite(x[i]);
    }
#pragma unroll
    for (int i = 0; i < 21; ++i) {
        c[i] = __ldcs(io.seed_cov + i * T + t);
        finite = finite && isfinite(c[i]);
    }
    const float qkb = (float)io.charge[t] * g.qk;
    const uint32_t mask = io.hit_mask[t];
    uint32_t flags = finite ? 0u : (uint32_t)KF_FLAG_NAN_INPUT;
    int K = 0;
    for (int l = 0; l < L && finite; ++l) {
        float xn[6], s;
        Jac J;
        if (!propagate(x, qkb, g.r[l], xn, s, &J)) {
            flags |= KF_FLAG_UNREACHABLE;
            break;
        }
        if (fabsf(xn[2]) > g.z_half) {
            flags |= KF_FLAG_LEFT_BARREL;
            break;
        }
        const float nx1 = xn[0] * g.inv_r[l], ny1 = xn[1] * g.inv_r[l];
        transport(J, c);
        {
            float q6[6];
            scattering_q6(xn, g.inv_r[l], g.xx0[l], q6);
            c[pk(3, 3)] += q6[0];
            c[pk(4, 3)] += q6[1];
            c[pk(4, 4)] += q6[2];
            c[pk(5, 3)] += q6[3];
            c[pk(5, 4)] += q6[4];
            c[pk(5, 5)] += q6[5];
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = xn[i];
        if ((mask >> l) & 1u) {
            float m[3], v[6], d = 0.0f;
#pragma unroll
            for (int i = 0; i < 3; ++i) m[i] = __ldcs(io.hit_pos + ((int64_t)l * 3 + i) * T + t);
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = __ldcs(io.hit_cov + ((int64_t)l * 6 + i) * T + t);
            bool hit_ok = true;
#pragma unroll
            for (int i = 0; i < 3; ++i) hit_ok = hit_ok && isfinite(m[i]);
#pragma unroll
            for (int i = 0; i < 6; ++i) hit_ok = hit_ok && isfinite(v[i]);
            if (!hit_ok) {
                flags |= KF_FLAG_NAN_INPUT;
                finite = false;
                break;
            }
            const int st = update(x, c, m, v, rt, &d, slot, stride);
            if (st == 1) flags |= KF_FLAG_INVERSION_FAILED;
            if (st >= 2) flags |= KF_FLAG_FP64_PATH;
            if (st == 3) flags |= KF_FLAG_PSD_REPAIRED;
        }
        // filtered: state, local covariance and its frame into the outputs
        {
            float cl[15];
            local_of(c, nx1, ny1, cl);
#pragma unroll
            for (int i = 0; i < 6; ++i) ost(l, i) = x[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) ocv(l, i) = cl[i];
            ocv(l, 15) = nx1;
            ocv(l, 16) = ny1;
        }
        K = l + 1;
    }
    if (!finite) K = 0;
    io.out_reached[t] = (int16_t)K;

    // ---- backward
    float xs[6], cs[15], nx = 1.0f, ny = 0.0f;  // smoothed at layer l+1 and its frame
    if (K > 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) xs[i] = ost(K - 1, i);
#pragma unroll
        for (int i = 0; i < 15; ++i) cs[i] = ocv(K - 1, i);
        nx = ocv(K - 1, 15);
        ny = ocv(K - 1, 16);
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) ocv(K - 1, pk(i, j)) = cart_of(cs, nx, ny, i, j);
    }
    for (int l = K - 2; l >= 0; --l) {
        float xf[6], cf[15], cp[15], xp[6], gj[13], q6[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) xf[i] = __ldlu(&ost(l, i));  // the filtered estimate's last read
#pragma unroll
        for (int i = 0; i < 15; ++i) cf[i] = __ldlu(&ocv(l, i));
        const float nxl = __ldlu(&ocv(l, 15)), nyl = __ldlu(&ocv(l, 16));
        {
            // the prediction of layer l+1 from the filtered estimate of layer
            // l, as the forward pass made it (the track reached layer l+1 there)
            float c21[21];
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) c21[pk(i, j)] = cart_of(cf, nxl, nyl, i, j);
            float sd;
            Jac J;
            propagate(xf, qkb, g.r[l + 1], xp, sd, &J);
            const float nx1 = xp[0] * g.inv_r[l + 1], ny1 = xp[1] * g.inv_r[l + 1];
            local_jacobian(J, nxl, nyl, nx1, ny1, gj);
            transport(J, c21);
            scattering_q6(xp, g.inv_r[l + 1], g.xx0[l + 1], q6);
            c21[pk(3, 3)] += q6[0];
            c21[pk(4, 3)] += q6[1];
            c21[pk(4, 4)] += q6[2];
            c21[pk(5, 3)] += q6[3];
            c21[pk(5, 4)] += q6[4];
            c21[pk(5, 5)] += q6[5];
            local_of(c21, nx1, ny1, cp);
        }
        // Cholesky of Cp scaled to unit diagonal: S = D Cp D, D = diag(Cp)^-1/2
        float dsc[5], Lc[15];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            ok = ok && cp[pk(i, i)] > 0.0f;
            dsc[i] = rsqrtf(cp[pk(i, i)]);
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            float djj = cp[pk(j, j)] * dsc[j] * dsc[j];
#pragma unroll
            for (int k = 0; k < j; ++k) djj = fmaf(-Lc[pk(j, k)], Lc[pk(j, k)], djj);
            ok = ok && djj > 0.0f;
            const float ljj = sqrtf(fmaxf(djj, 1e-30f)), il = 1.0f / ljj;
            Lc[pk(j, j)] = ljj;
#pragma unroll
            for (int i = j + 1; i < 5; ++i) {
                float sij = cp[pk(i, j)] * dsc[i] * dsc[j];
#pragma unroll
                for (int k = 0; k < j; ++k) sij = fmaf(-Lc[pk(i, k)], Lc[pk(j, k)], sij);
                Lc[pk(i, j)] = sij * il;
            }
        }
        // M^-1 of the transverse block (t, px, py) by adjugate
        const float m00 = gj[0], m01 = gj[1], m02 = gj[2], m10 = gj[3], m11 = gj[4], m12 = gj[5];
        const float m20 = gj[6], m21 = gj[7], m22 = gj[8];
        const float a00 = m11 * m22 - m12 * m21, a01 = m02 * m21 - m01 * m22, a02 = m01 * m12 - m02 * m11;
        const float a10 = m12 * m20 - m10 * m22, a11 = m00 * m22 - m02 * m20, a12 = m02 * m10 - m00 * m12;
        const float a20 = m10 * m21 - m11 * m20, a21 = m01 * m20 - m00 * m21, a22 = m00 * m11 - m01 * m10;
        const float detm = m00 * a00 + m01 * a10 + m02 * a20;
        ok = ok && fabsf(detm) > 1e-6f;
        if (!ok) {  // no smoothing across this layer: keep the filtered estimate
            flags |= KF_FLAG_INVERSION_FAILED;
#pragma unroll
            for (int i = 0; i < 6; ++i) xs[i] = xf[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) cs[i] = cf[i];
        } else {
            const float idet = 1.0f / detm;
            // G^-1 (5x5): (t, px, py) = Mi (t', px', py'); pz = pz';
            // z = z' - (mz Mi) . (t', px', py') - jp pz'
            float Gi[5][5];
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) Gi[i][j] = 0.0f;
            const float Mi[3][3] = {{a00 * idet, a01 * idet, a02 * idet},
                                    {a10 * idet, a11 * idet, a12 * idet},
                                    {a20 * idet, a21 * idet, a22 * idet}};
            constexpr int Q3[3] = {0, 2, 3};
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) Gi[Q3[r]][Q3[c3]] = Mi[r][c3];
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3)
                Gi[1][Q3[c3]] = -fmaf(gj[9], Mi[0][c3], fmaf(gj[10], Mi[1][c3], gj[11] * Mi[2][c3]));
            Gi[1][1] = 1.0f;
            Gi[1][4] = -gj[12];
            Gi[4][4] = 1.0f;
            // W = Cp^-1 Q (only Q's momentum columns are non-zero): three
            // solves with the scaled factor, Cp^-1 b = D S^-1 D b
            float W[5][3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // column 2 + k of the local Q (rows px, py, pz; packed q6 is
                // (px,px) (py,px) (py,py) (pz,px) (pz,py) (pz,pz))
                const float b5[5] = {0.0f, 0.0f, q6[k == 0 ? 0 : k == 1 ? 1 : 3], q6[k == 0 ? 1 : k == 1 ? 2 : 4],
                                     q6[k == 0 ? 3 : k == 1 ? 4 : 5]};
                float y[5];
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    float acc = dsc[i] * b5[i];
#pragma unroll
                    for (int j = 0; j < i; ++j) acc = fmaf(-Lc[pk(i, j)], y[j], acc);
                    y[i] = acc / Lc[pk(i, i)];
                }
#pragma unroll
                for (int i = 4; i >= 0; --i) {
                    float acc = y[i];
#pragma unroll
                    for (int j = i + 1; j < 5; ++j) acc = fmaf(-Lc[pk(j, i)], y[j], acc);
                    y[i] = acc / Lc[pk(i, i)];
                }
#pragma unroll
                for (int i = 0; i < 5; ++i) W[i][k] = dsc[i] * y[i];
            }
            // A = G^-1 (I - Q Cp^-1), (Q Cp^-1)[2 + k][j] = W[j][k]; kept as At = A^T
            float At[5][5];
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    float acc = Gi[i][j];
#pragma unroll
                    for (int k = 0; k < 3; ++k) acc = fmaf(-Gi[i][2 + k], W[j][k], acc);
                    At[j][i] = acc;
                }
            // state: delta = local(n_{l+1}) of (xs - xp)
            const float d0 = xs[0] - xp[0], d1 = xs[1] - xp[1];
            const float dl[5] = {fmaf(nx, d1, -ny * d0), xs[2] - xp[2], xs[3] - xp[3], xs[4] - xp[4],
                                 xs[5] - xp[5]};
            float e[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < 5; ++k) acc = fmaf(At[k][i], dl[k], acc);
                e[i] = acc;
            }
            xs[0] = fmaf(-nyl, e[0], xf[0]);
            xs[1] = fmaf(nxl, e[0], xf[1]);
#pragma unroll
            for (int i = 1; i < 5; ++i) xs[i + 1] = xf[i + 1] + e[i];
            // covariance: Cs = Cf + A (Cs' - Cp) A^T
            float D5[15];
#pragma unroll
            for (int i = 0; i < 15; ++i) D5[i] = cs[i] - cp[i];
            float AD[5][5];  // A D
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < 5; ++k) acc = fmaf(At[k][i], D5[pk(k, j)], acc);
                    AD[i][j] = acc;
                }
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) {
                    float acc = cf[pk(i, j)];
#pragma unroll
                    for (int k = 0; k < 5; ++k) acc = fmaf(AD[i][k], At[k][j], acc);
                    cs[pk(i, j)] = acc;
                }
        }
        nx = nxl;
        ny = nyl;
#pragma unroll
        for (int i = 0; i < 6; ++i) __stcs(&ost(l, i), xs[i]);  // final: streamed out
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) __stcs(&ocv(l, pk(i, j)), cart_of(cs, nx, ny, i, j));
    }
    // layers not reached (and every layer of a track with a non-finite input)
    for (int l = K; l < L; ++l) {
#pragma unroll
        for (int i = 0; i < 6; ++i) ost(l, i) = NAN;
#pragma unroll
        for (int i = 0; i < 21; ++i) ocv(l, i) = NAN;
    }
    io.out_flags[t] = flags;
}

}  // namespace
}  // namespace kf

using namespace kf;

extern "C" int kf_smooth_tracks(kf_context *ctx, const kf_geometry *geom, int64_t n_tracks, const float *seed_state,
                                const float *seed_cov, const int8_t *charge, const float *hit_pos, const float *hit_cov,
                                const uint32_t *hit_mask, float *out_state, float *out_cov, int16_t *out_reached,
                                uint32_t *out_flags, const kf_options *opt, kf_stream stream_)
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
    if (n_tracks == 0) return KF_OK;
    if ((rc = check_ptr(ctx, seed_state, 4, "seed_state")) || (rc = check_ptr(ctx, seed_cov, 4, "seed_cov")) ||
        (rc = check_ptr(ctx, charge, 1, "charge")) || (rc = check_ptr(ctx, hit_pos, 4, "hit_pos")) ||
        (rc = check_ptr(ctx, hit_cov, 4, "hit_cov")) || (rc = check_ptr(ctx, hit_mask, 4, "hit_mask")) ||
        (rc = check_ptr(ctx, out_state, 4, "out_state")) || (rc = check_ptr(ctx, out_cov, 4, "out_cov")) ||
        (rc = check_ptr(ctx, out_reached, 2, "out_reached")) || (rc = check_ptr(ctx, out_flags, 4, "out_flags")))
        return rc;
    DeviceGuard dg(context_device(ctx));
    SmoothIO io{n_tracks, seed_state, seed_cov, charge, hit_pos, hit_cov, hit_mask,
                out_state, out_cov, out_reached, out_flags};
    const unsigned blocks = (unsigned)((n_tracks + 127) / 128);
    smooth_kernel<<<blocks, 128, kSlotSize * 128 * sizeof(float), reinterpret_cast<cudaStream_t>(stream_)>>>(
        g, make_routing(o), io);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : cuda_error(ctx, e, "smoother launch");
}
