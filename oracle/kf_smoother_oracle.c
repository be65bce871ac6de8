/*
 * Plain FP64 CPU oracle for the Kalman smoother: after the forward fit of a
 * track (Sections 2 and 2.1 of arXiv:1705.02876), the backward
 * Rauch-Tung-Striebel pass gives at every layer the estimate that uses all of
 * the track's hits (Section 2 of the paper names a final Kalman fit with a
 * smoother, after building, as the step that gives each track's best
 * parameters).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite; shares no code with the
 * CUDA library.
 *
 * Pins (the CPU tests): the last layer equals the forward fit; without
 * scattering the smoothed states are one helix and equal a least-squares fit
 * of all hits at every layer; smoothing never increases a variance; smoothed
 * pulls have unit width.
 *
 * Forward: the oracle's own propagation, transport, scattering and update
 * (kf_oracle.c), keeping at every layer reached the predicted state x_p and
 * covariance C_p, the filtered x_f and C_f, and the transport Jacobian F from
 * the previous layer.  On a cylinder both covariances are singular (the
 * crossing cannot leave the surface, so the radial direction n = (x, y, 0)/r
 * of the predicted crossing carries no variance); the backward pass therefore
 * works in each layer's local coordinates (t, z, px, py, pz), t = z x n:
 * P_k projects a Cartesian vector onto them, R_k embeds them back (x = -n_y t,
 * y = n_x t).  With G = P_{k+1} F R_k (5x5):
 *   A_k    = Cf_k G^T Cp_{k+1}^-1,
 *   xs_k   = xf_k + R_k A_k P_{k+1} (xs_{k+1} - xp_{k+1}),
 *   Cs_k   = Cf_k + A_k (Cs_{k+1} - Cp_{k+1}) A_k^T  (local, then R_k . R_k^T),
 * starting from xs = xf, Cs = Cf at the last layer reached.  Dense 5x5
 * algebra; Cp^-1 by Gauss-Jordan elimination with partial pivoting.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define MAXL 64

int orc_propagate(const double *st, int q, double bz, double r, double *out, double *J, double *s_out);
void orc_ms_noise(const double *st, double x_over_x0, double *Q);
void orc_transport(const double *J, double *C, const double *Q);
int orc_update(double *x, double *C, const double *m, const double *Vp, double *dchi2);
void orc_unpack_sym(const double *packed, int n, double *full);

/* Cartesian <-> local (t, z, px, py, pz) at the radial direction (nx, ny) */
static void proj(double nx, double ny, double P[5][6])
{
    memset(P, 0, sizeof(double) * 30);
    P[0][0] = -ny;
    P[0][1] = nx;
    for (int i = 1; i < 5; ++i) P[i][i + 1] = 1.0;
}

static void embed(double nx, double ny, double R[6][5])
{
    memset(R, 0, sizeof(double) * 30);
    R[0][0] = -ny;
    R[1][0] = nx;
    for (int i = 1; i < 5; ++i) R[i + 1][i] = 1.0;
}

/* local 5x5 of a Cartesian 6x6: P C P^T */
static void to_local(const double *C6, double nx, double ny, double L5[5][5])
{
    double P[5][6];
    proj(nx, ny, P);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double s = 0.0;
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) s += P[i][a] * C6[a * 6 + b] * P[j][b];
            L5[i][j] = s;
        }
}

/* Gauss-Jordan inverse of a 5x5; returns 0 if singular */
static int inv5(double A[5][5], double Ai[5][5])
{
    double M[5][10];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 10; ++j) M[i][j] = j < 5 ? A[i][j] : (j - 5 == i);
    for (int c = 0; c < 5; ++c) {
        int p = c;
        for (int r = c + 1; r < 5; ++r)
            if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (M[p][c] == 0.0) return 0;
        if (p != c)
            for (int j = 0; j < 10; ++j) {
                const double t = M[p][j];
                M[p][j] = M[c][j];
                M[c][j] = t;
            }
        const double d = M[c][c];
        for (int j = 0; j < 10; ++j) M[c][j] /= d;
        for (int r = 0; r < 5; ++r)
            if (r != c) {
                const double f = M[r][c];
                for (int j = 0; j < 10; ++j) M[r][j] -= f * M[c][j];
            }
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Ai[i][j] = M[i][j + 5];
    return 1;
}

typedef struct {
    double xp[6], Cp[36], xf[6], Cf[36], F[36]; /* F: Jacobian from the previous layer */
    double nx, ny;                              /* radial direction of the predicted crossing */
} layer_t;

/*
 * Smooth tracks [t_begin, t_end) of a batch in the library's layout (float
 * inputs, promoted): seed_state [6][T], seed_cov [21][T], charge [T], hit_pos
 * [L][3][T], hit_cov [L][6][T], hit_mask [T].  Outputs: out_state [L][6][T]
 * and out_cov [L][21][T] packed, the smoothed estimate after every layer the
 * forward fit reached (NaN elsewhere, and everywhere for a track with a
 * non-finite input); out_filt_state [L][6][T] (may be NULL) the forward
 * filter's; out_reached [T] the number of layers reached.  A layer without a
 * hit, or whose update failed, has xf = xp, Cf = Cp.  Returns 0, or -1 if
 * n_layers is out of range.
 */
int orc_smooth_tracks(int n_layers, const double *radii, const double *x_over_x0, double z_half, double bz,
                      int64_t t_begin, int64_t t_end, int64_t n_tracks, const float *seed_state,
                      const float *seed_cov, const int8_t *charge, const float *hit_pos, const float *hit_cov,
                      const uint32_t *hit_mask, double *out_state, double *out_cov, double *out_filt_state,
                      int32_t *out_reached)
{
    const int64_t T = n_tracks;
    const int L = n_layers;
    if (L < 0 || L > MAXL) return -1;
    layer_t lay[MAXL];
    for (int64_t t = t_begin; t < t_end; ++t) {
        for (int l = 0; l < L; ++l) {
            for (int i = 0; i < 6; ++i) {
                out_state[((int64_t)l * 6 + i) * T + t] = NAN;
                if (out_filt_state) out_filt_state[((int64_t)l * 6 + i) * T + t] = NAN;
            }
            for (int i = 0; i < 21; ++i) out_cov[((int64_t)l * 21 + i) * T + t] = NAN;
        }
        double x[6], c0[21], C[36];
        int finite = 1;
        for (int i = 0; i < 6; ++i) {
            x[i] = seed_state[i * T + t];
            finite &= isfinite(x[i]) != 0;
        }
        for (int i = 0; i < 21; ++i) {
            c0[i] = seed_cov[i * T + t];
            finite &= isfinite(c0[i]) != 0;
        }
        orc_unpack_sym(c0, 6, C);
        const int q = charge[t];
        int K = 0;
        for (int l = 0; l < L && finite; ++l) {
            layer_t *k = &lay[l];
            double Q[36], s;
            if (orc_propagate(x, q, bz, radii[l], k->xp, k->F, &s) || fabs(k->xp[2]) > z_half) break;
            orc_ms_noise(k->xp, x_over_x0[l], Q);
            orc_transport(k->F, C, Q);
            memcpy(k->Cp, C, sizeof C);
            memcpy(x, k->xp, sizeof x);
            const double r = hypot(x[0], x[1]);
            k->nx = x[0] / r;
            k->ny = x[1] / r;
            if (hit_mask[t] >> l & 1u) {
                double m[3], v[6], d;
                for (int i = 0; i < 3; ++i) m[i] = hit_pos[((int64_t)l * 3 + i) * T + t];
                for (int i = 0; i < 6; ++i) v[i] = hit_cov[((int64_t)l * 6 + i) * T + t];
                int ok = 1;
                for (int i = 0; i < 3; ++i) ok &= isfinite(m[i]) != 0;
                for (int i = 0; i < 6; ++i) ok &= isfinite(v[i]) != 0;
                if (!ok) {
                    finite = 0;
                    break;
                }
                double xu[6], Cu[36];
                memcpy(xu, x, sizeof x);
                memcpy(Cu, C, sizeof C);
                if (orc_update(xu, Cu, m, v, &d) == 0) {
                    memcpy(x, xu, sizeof x);
                    memcpy(C, Cu, sizeof C);
                }
            }
            memcpy(k->xf, x, sizeof x);
            memcpy(k->Cf, C, sizeof C);
            K = l + 1;
        }
        out_reached[t] = finite ? K : 0;
        if (!finite) continue;
        /* backward pass */
        double xs[6], Cs5[5][5];
        if (K > 0) {
            memcpy(xs, lay[K - 1].xf, sizeof xs);
            to_local(lay[K - 1].Cf, lay[K - 1].nx, lay[K - 1].ny, Cs5);
        }
        for (int l = K - 1; l >= 0; --l) {
            layer_t *k = &lay[l];
            if (l < K - 1) {
                const layer_t *n1 = &lay[l + 1];
                double P1[5][6], R0[6][5], G[5][5], Cf5[5][5], Cp5[5][5], Cpi[5][5], A[5][5], D5[5][5];
                proj(n1->nx, n1->ny, P1);
                embed(k->nx, k->ny, R0);
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j < 5; ++j) {
                        double s = 0.0;
                        for (int a = 0; a < 6; ++a)
                            for (int b = 0; b < 6; ++b) s += P1[i][a] * n1->F[a * 6 + b] * R0[b][j];
                        G[i][j] = s;
                    }
                to_local(k->Cf, k->nx, k->ny, Cf5);
                to_local(n1->Cp, n1->nx, n1->ny, Cp5);
                if (!inv5(Cp5, Cpi)) break;
                /* A = Cf G^T Cp^-1 */
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j < 5; ++j) {
                        double s = 0.0;
                        for (int a = 0; a < 5; ++a)
                            for (int b = 0; b < 5; ++b) s += Cf5[i][a] * G[b][a] * Cpi[b][j];
                        A[i][j] = s;
                    }
                /* state: xs_l = xf + R0 A P1 (xs_{l+1} - xp_{l+1}) */
                double d6[6], d5[5], e5[5];
                for (int i = 0; i < 6; ++i) d6[i] = xs[i] - n1->xp[i];
                for (int i = 0; i < 5; ++i) {
                    double s = 0.0;
                    for (int a = 0; a < 6; ++a) s += P1[i][a] * d6[a];
                    d5[i] = s;
                }
                for (int i = 0; i < 5; ++i) {
                    double s = 0.0;
                    for (int a = 0; a < 5; ++a) s += A[i][a] * d5[a];
                    e5[i] = s;
                }
                for (int i = 0; i < 6; ++i) {
                    double s = 0.0;
                    for (int a = 0; a < 5; ++a) s += R0[i][a] * e5[a];
                    xs[i] = k->xf[i] + s;
                }
                /* covariance: Cs_l = Cf + A (Cs_{l+1} - Cp_{l+1}) A^T */
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j < 5; ++j) D5[i][j] = Cs5[i][j] - Cp5[i][j];
                double N5[5][5];
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j < 5; ++j) {
                        double s = 0.0;
                        for (int a = 0; a < 5; ++a)
                            for (int b = 0; b < 5; ++b) s += A[i][a] * D5[a][b] * A[j][b];
                        N5[i][j] = Cf5[i][j] + s;
                    }
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j < 5; ++j) Cs5[i][j] = 0.5 * (N5[i][j] + N5[j][i]);
            }
            double R[6][5];
            embed(k->nx, k->ny, R);
            for (int i = 0; i < 6; ++i) {
                out_state[((int64_t)l * 6 + i) * T + t] = xs[i];
                if (out_filt_state) out_filt_state[((int64_t)l * 6 + i) * T + t] = k->xf[i];
            }
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j <= i; ++j) {
                    double s = 0.0;
                    for (int a = 0; a < 5; ++a)
                        for (int b = 0; b < 5; ++b) s += R[i][a] * Cs5[a][b] * R[j][b];
                    out_cov[((int64_t)l * 21 + i * (i + 1) / 2 + j) * T + t] = s;
                }
        }
    }
    return 0;
}

/* The crossing of radius r going backwards along the helix from st (charge
 * q): the momentum and charge reversed, propagated forward, the momentum
 * reversed again.  Returns what orc_propagate returns. */
int orc_propagate_back(const double *st, int q, double bz, double r, double *out)
{
    double rev[6], J[36], s;
    memcpy(rev, st, sizeof rev);
    for (int i = 3; i < 6; ++i) rev[i] = -rev[i];
    const int rc = orc_propagate(rev, -q, bz, r, out, J, &s);
    for (int i = 3; i < 6; ++i) out[i] = -out[i];
    return rc;
}
