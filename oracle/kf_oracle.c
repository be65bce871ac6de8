/*
 * Plain FP64 CPU oracle for the Kalman-filter track fit (Sections 2, 2.1 and
 * 4.2 of arXiv:1705.02876).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is loaded by the test suite, by the
 * package smoke check and by the CPU-baseline leg of the benchmark, nothing
 * else.  It shares no code, header, table or constant generator with the CUDA
 * library; the two meet only in the arrays the seeded generator produces.
 *
 * The paper states no equations: it fixes the parametrisation (a 6-parameter
 * global state (x, y, z, px, py, pz) with a 6x6 covariance, a 3-D measurement
 * with a 3x3 covariance; Section 2.1) and says that the filter folds
 * multiple-scattering estimates into the trajectory (Section 2).  The steps
 * below are the textbook extended Kalman filter (the paper's reference for the
 * method, Fruhwirth 1987) in that parametrisation:
 *
 *   propagate  the state to the next cylinder along the helix of a uniform
 *              field Bz (smallest positive transverse path length s);
 *   transport  C' = J C J^T + Q, J = dF/dx0 at fixed s + dF/ds (x) ds/dx0;
 *   scatter    Q = theta0^2 (|p|^2 I3 - p p^T) on the momentum block, theta0
 *              from the Highland formula for beta = 1 and an effective
 *              thickness x/X0 / |cos(incidence)|;
 *   update     S = H C H^T + V, K = C H^T S^-1, x += K r, C -= K H C,
 *              C <- (C + C^T)/2, chi2 += r^T S^-1 r, with H = [I3 0].
 *
 * All linear algebra is dense and unblocked: full 6x6 products, a Cholesky
 * factorisation for S^-1.  Every function works in double precision on inputs
 * promoted from the float32 arrays the library sees.
 *
 * Pins (the CPU tests): the crossing against an RK4 integration of the
 * equation of motion and against the line-cylinder root at Bz = 0; J against
 * central differences; S^-1 against LU inversion; the update against the
 * information form; the fit against exact hits, against a Gauss-Newton least
 * squares fit when scattering is off, and against unit pulls and flat chi2
 * p-values on simulated tracks.  The Highland constants (0.0136 GeV, 0.038)
 * are a convention the generator and both implementations share: parity
 * unpinned for those two constants.  Q's structure (no component along p,
 * isotropic across it) and its size relative to the generator's kicks (the
 * pull widths) are pinned.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORC_K 0.00299792458 /* GeV / (cm T) */
#define ORC_PI 3.14159265358979323846

/* per-track result flags (values fixed by the library's C interface) */
#define ORC_FLAG_UNREACHABLE 1u
#define ORC_FLAG_LEFT_BARREL 2u
#define ORC_FLAG_INVERSION_FAILED 4u
#define ORC_FLAG_NAN_INPUT 8u

/* ------------------------------------------------------------------------ */
/* small dense helpers                                                       */

static void mat6_mul(const double *A, const double *B, double *out)
{
    double t[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k) acc += A[i * 6 + k] * B[k * 6 + j];
            t[i * 6 + j] = acc;
        }
    memcpy(out, t, sizeof t);
}

static void mat6_transpose(const double *A, double *out)
{
    double t[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) t[j * 6 + i] = A[i * 6 + j];
    memcpy(out, t, sizeof t);
}

/* packed lower triangle, row by row: (0,0),(1,0),(1,1),(2,0),... */
static int pidx(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

void orc_unpack_sym(const double *packed, int n, double *full)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) full[i * n + j] = packed[pidx(i, j)];
}

static void pack_sym6(const double *full, double *packed)
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) packed[pidx(i, j)] = full[i * 6 + j];
}

/* ------------------------------------------------------------------------ */
/* propagation to a cylinder                                                 */

/*
 * Move state st (charge q) to its first forward crossing of radius r in the
 * field bz.  Equations of motion in the transverse path length s, with
 * omega = q k Bz / pT:
 *   px(s) = px cos(omega s) + py sin(omega s),  py(s) = py cos - px sin,
 *   x(s) = x + (px sin + py (1 - cos)) / (q k Bz),
 *   y(s) = y + (py sin - px (1 - cos)) / (q k Bz),
 *   z(s) = z + pz s / pT,  pz(s) = pz.
 * The crossing is the circle-circle intersection of the helix projection with
 * the cylinder, taking the smallest positive s; a straight line (omega = 0)
 * uses the line-cylinder quadratic.  J (row-major 6x6, may be NULL) is the
 * Jacobian of the crossing state with respect to st.
 * Returns 0, or 1 if the cylinder is not reached.
 */
int orc_propagate(const double *st, int q, double bz, double r, double *out, double *J,
                  double *s_out)
{
    const double x = st[0], y = st[1], z = st[2], px = st[3], py = st[4], pz = st[5];
    const double pt = hypot(px, py);
    const double tx = px / pt, ty = py / pt;
    const double qk = (double)q * ORC_K * bz;
    const double omega = qk / pt;
    double s;

    if (!(pt > 0.0)) return 1;
    if (omega == 0.0) {
        const double u = x * tx + y * ty;
        const double disc = u * u - (x * x + y * y - r * r);
        if (disc < 0.0) return 1;
        const double s1 = -u - sqrt(disc), s2 = -u + sqrt(disc);
        s = s1 > 0.0 ? s1 : s2;
        if (!(s > 0.0)) return 1;
    } else {
        const double cx = x + ty / omega, cy = y - tx / omega;
        const double rho = 1.0 / fabs(omega);
        const double d = hypot(cx, cy);
        if (d == 0.0 || d + rho < r || fabs(d - rho) > r) return 1;
        const double a = (r * r - rho * rho + d * d) / (2.0 * d);
        const double h2 = r * r - a * a;
        const double h = h2 > 0.0 ? sqrt(h2) : 0.0;
        const double ux = cx / d, uy = cy / d;
        const double period = 2.0 * ORC_PI * rho;
        double best = INFINITY;
        for (int side = -1; side <= 1; side += 2) {
            const double X = a * ux - side * h * uy, Y = a * uy + side * h * ux;
            const double e0x = x - cx, e0y = y - cy, e1x = X - cx, e1y = Y - cy;
            /* the radius vector from the centre turns by -omega*s (counter-clockwise angle) */
            const double alpha = atan2(e0x * e1y - e0y * e1x, e0x * e1x + e0y * e1y);
            double sk = fmod(-alpha / omega, period);
            if (sk <= 0.0) sk += period;
            if (sk < best) best = sk;
        }
        s = best;
    }

    double c = 1.0, sn = 0.0, omc = 0.0, phi = 0.0;
    if (omega != 0.0) {
        phi = omega * s;
        c = cos(phi);
        sn = sin(phi);
        omc = 2.0 * sin(0.5 * phi) * sin(0.5 * phi); /* 1 - cos(phi) */
        out[0] = x + (px * sn + py * omc) / qk;
        out[1] = y + (py * sn - px * omc) / qk;
        out[3] = px * c + py * sn;
        out[4] = py * c - px * sn;
    } else {
        out[0] = x + s * tx;
        out[1] = y + s * ty;
        out[3] = px;
        out[4] = py;
    }
    out[2] = z + pz * s / pt;
    out[5] = pz;
    if (s_out) *s_out = s;
    if (!J) return 0;

    /* D = dF/dx0 at fixed s */
    double D[36];
    memset(D, 0, sizeof D);
    D[0 * 6 + 0] = 1.0;
    D[1 * 6 + 1] = 1.0;
    D[2 * 6 + 2] = 1.0;
    D[5 * 6 + 5] = 1.0;
    D[2 * 6 + 3] = -pz * s * px / (pt * pt * pt);
    D[2 * 6 + 4] = -pz * s * py / (pt * pt * pt);
    D[2 * 6 + 5] = s / pt;
    if (omega != 0.0) {
        /* phi = omega s depends on pT: dphi/dpx = -phi px / pT^2 */
        const double dphx = -phi * px / (pt * pt), dphy = -phi * py / (pt * pt);
        D[0 * 6 + 3] = (sn + out[3] * dphx) / qk;
        D[0 * 6 + 4] = (omc + out[3] * dphy) / qk;
        D[1 * 6 + 3] = (-omc + out[4] * dphx) / qk;
        D[1 * 6 + 4] = (sn + out[4] * dphy) / qk;
        D[3 * 6 + 3] = c + out[4] * dphx;
        D[3 * 6 + 4] = sn + out[4] * dphy;
        D[4 * 6 + 3] = -sn - out[3] * dphx;
        D[4 * 6 + 4] = c - out[3] * dphy;
    } else {
        D[0 * 6 + 3] = s * ty * ty / pt;
        D[0 * 6 + 4] = -s * tx * ty / pt;
        D[1 * 6 + 3] = -s * tx * ty / pt;
        D[1 * 6 + 4] = s * tx * tx / pt;
        D[3 * 6 + 3] = 1.0;
        D[4 * 6 + 4] = 1.0;
    }
    /* dF/ds and ds/dx0 from the constraint x'^2 + y'^2 = r^2 */
    const double dFds[6] = {out[3] / pt, out[4] / pt, pz / pt, omega * out[4], -omega * out[3], 0.0};
    const double den = out[0] * dFds[0] + out[1] * dFds[1];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            const double dsdj = -(out[0] * D[0 * 6 + j] + out[1] * D[1 * 6 + j]) / den;
            J[i * 6 + j] = D[i * 6 + j] + dFds[i] * dsdj;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* multiple scattering                                                       */

/* Q (row-major 6x6) for a thin layer of x_over_x0 at the state st, which sits on
 * the cylinder; the layer normal is n = (x, y, 0)/r. */
void orc_ms_noise(const double *st, double x_over_x0, double *Q)
{
    memset(Q, 0, 36 * sizeof(double));
    if (!(x_over_x0 > 0.0)) return;
    const double r = hypot(st[0], st[1]);
    const double nx = st[0] / r, ny = st[1] / r;
    const double p2 = st[3] * st[3] + st[4] * st[4] + st[5] * st[5];
    const double p = sqrt(p2);
    const double cosi = fabs(st[3] * nx + st[4] * ny) / p;
    const double xx0 = x_over_x0 / cosi;
    const double th0 = 0.0136 / p * sqrt(xx0) * (1.0 + 0.038 * log(xx0));
    const double t2 = th0 * th0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Q[(3 + i) * 6 + 3 + j] = t2 * ((i == j ? p2 : 0.0) - st[3 + i] * st[3 + j]);
}

/* ------------------------------------------------------------------------ */
/* 3x3 inverse by Cholesky                                                   */

/* S row-major 3x3 symmetric; returns 0 and Sinv, or 1 if S is not positive definite */
int orc_inv3_cholesky(const double *S, double *Sinv)
{
    double L[9] = {0}, Li[9] = {0};
    double d0 = S[0];
    if (!(d0 > 0.0)) return 1;
    L[0] = sqrt(d0);
    L[3] = S[3] / L[0];
    double d1 = S[4] - L[3] * L[3];
    if (!(d1 > 0.0)) return 1;
    L[4] = sqrt(d1);
    L[6] = S[6] / L[0];
    L[7] = (S[7] - L[6] * L[3]) / L[4];
    double d2 = S[8] - L[6] * L[6] - L[7] * L[7];
    if (!(d2 > 0.0)) return 1;
    L[8] = sqrt(d2);
    /* Li = L^-1 by forward substitution */
    Li[0] = 1.0 / L[0];
    Li[4] = 1.0 / L[4];
    Li[8] = 1.0 / L[8];
    Li[3] = -L[3] * Li[0] / L[4];
    Li[7] = -L[7] * Li[4] / L[8];
    Li[6] = -(L[6] * Li[0] + L[7] * Li[3]) / L[8];
    /* S^-1 = Li^T Li */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += Li[k * 3 + i] * Li[k * 3 + j];
            Sinv[i * 3 + j] = acc;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Kalman update with a 3-D hit                                              */

/* x[6], C row-major 6x6 (updated in place); m[3]; V packed 3x3.
 * Returns 0 and adds the chi2 increment, or 1 (S not positive definite; the
 * state is left unchanged). */
int orc_update(double *x, double *C, const double *m, const double *Vp, double *dchi2)
{
    double S[9], Si[9], K[18], r[3], Cn[36];
    double V[9];
    orc_unpack_sym(Vp, 3, V);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i * 3 + j] = C[i * 6 + j] + V[i * 3 + j];
    if (orc_inv3_cholesky(S, Si)) return 1;
    for (int i = 0; i < 3; ++i) r[i] = m[i] - x[i];
    /* K = C H^T S^-1 : 6x3 */
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += C[i * 6 + k] * Si[k * 3 + j];
            K[i * 3 + j] = acc;
        }
    double chi2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) chi2 += r[i] * Si[i * 3 + j] * r[j];
    for (int i = 0; i < 6; ++i)
        for (int k = 0; k < 3; ++k) x[i] += K[i * 3 + k] * r[k];
    /* C - K H C */
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += K[i * 3 + k] * C[k * 6 + j];
            Cn[i * 6 + j] = C[i * 6 + j] - acc;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) C[i * 6 + j] = 0.5 * (Cn[i * 6 + j] + Cn[j * 6 + i]);
    *dchi2 = chi2;
    return 0;
}

/* C <- J C J^T + Q (all row-major 6x6) */
void orc_transport(const double *J, double *C, const double *Q)
{
    double Jt[36];
    mat6_mul(J, C, C);
    mat6_transpose(J, Jt);
    mat6_mul(C, Jt, C);
    for (int i = 0; i < 36; ++i) C[i] += Q[i];
}

/* ------------------------------------------------------------------------ */
/* the fit                                                                   */

static int finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

/*
 * Fit one track (Section 4.2: all layers in order, no branching on the hit
 * content).  Inputs in double precision: x0[6], c0[21] packed, charge q,
 * hits m[L][3], V[L][6] packed, mask (bit l set = a hit on layer l).
 *
 * For each layer in order: propagate; stop (flag) if the cylinder is not
 * reached or the crossing lies beyond |z| = z_half; otherwise transport the
 * covariance, add the layer's scattering and, if the hit is present, update.
 * A non-finite seed, or a non-finite value in a hit the fit reaches and uses,
 * stops the fit and returns the seed unchanged (flag NAN_INPUT).
 * ls[L][6] and lc[L][21] (may be NULL) receive the state after each layer
 * (NaN where the track did not reach it).
 */
static void fit_one(int n_layers, const double *radii, const double *x_over_x0, double z_half,
                    double bz, const double *x0, const double *c0, int q, const double *m,
                    const double *V, uint32_t mask, double *x_out, double *c_out, double *chi2_out,
                    int32_t *ndof_out, uint32_t *flags_out, double *ls, double *lc)
{
    double x[6], C[36];
    uint32_t flags = 0;
    int nhits = 0;
    double chi2 = 0.0;
    memcpy(x, x0, sizeof x);
    orc_unpack_sym(c0, 6, C);
    if (!finite_all(x0, 6) || !finite_all(c0, 21)) flags |= ORC_FLAG_NAN_INPUT;
    if (ls)
        for (int i = 0; i < 6 * n_layers; ++i) ls[i] = NAN;
    if (lc)
        for (int i = 0; i < 21 * n_layers; ++i) lc[i] = NAN;

    for (int l = 0; l < n_layers && !(flags & ORC_FLAG_NAN_INPUT); ++l) {
        double xn[6], J[36], Q[36], s;
        if (orc_propagate(x, q, bz, radii[l], xn, J, &s)) {
            flags |= ORC_FLAG_UNREACHABLE;
            break;
        }
        if (fabs(xn[2]) > z_half) {
            flags |= ORC_FLAG_LEFT_BARREL;
            break;
        }
        orc_ms_noise(xn, x_over_x0[l], Q);
        orc_transport(J, C, Q);
        memcpy(x, xn, sizeof x);
        if (mask >> l & 1u) {
            double d;
            if (!finite_all(m + 3 * l, 3) || !finite_all(V + 6 * l, 6)) {
                flags |= ORC_FLAG_NAN_INPUT;
                break;
            }
            if (orc_update(x, C, m + 3 * l, V + 6 * l, &d)) {
                flags |= ORC_FLAG_INVERSION_FAILED;
            } else {
                chi2 += d;
                ++nhits;
            }
        }
        if (ls) memcpy(ls + 6 * l, x, sizeof x);
        if (lc) pack_sym6(C, lc + 21 * l);
    }
    if (flags & ORC_FLAG_NAN_INPUT) { /* a track with a non-finite input returns its seed */
        memcpy(x, x0, sizeof x);
        orc_unpack_sym(c0, 6, C);
        chi2 = 0.0;
        nhits = 0;
    }
    memcpy(x_out, x, sizeof x);
    pack_sym6(C, c_out);
    *chi2_out = chi2;
    *ndof_out = 3 * nhits - 6;
    *flags_out = flags;
}

#define MAXL 64

/*
 * Fit tracks [t_begin, t_end) of a batch of n_tracks stored in the library's
 * layout: seed_state [6][T], seed_cov [21][T] packed, charge [T],
 * hit_pos [L][3][T], hit_cov [L][6][T] packed, hit_mask [T].  Inputs are
 * float32 (the library's inputs, promoted) or, in orc_fit_tracks_f64, double.
 * Outputs: state [6][T], cov [21][T], chi2 [T], ndof [T] = 3 n_hits - 6,
 * flags [T]; layer_state [L][6][T] and layer_cov [L][21][T] may be NULL.
 * Returns 0, or -1 if n_layers is out of range.
 */
#define DEFINE_FIT_TRACKS(NAME, REAL)                                                          \
    int NAME(int n_layers, const double *radii, const double *x_over_x0, double z_half,       \
             double bz, int64_t t_begin, int64_t t_end, int64_t n_tracks,                      \
             const REAL *seed_state, const REAL *seed_cov, const int8_t *charge,               \
             const REAL *hit_pos, const REAL *hit_cov, const uint32_t *hit_mask,               \
             double *out_state, double *out_cov, double *out_chi2, int32_t *out_ndof,          \
             uint32_t *out_flags, double *layer_state, double *layer_cov)                      \
    {                                                                                          \
        const int64_t T = n_tracks;                                                            \
        if (n_layers < 0 || n_layers > MAXL) return -1;                                        \
        for (int64_t t = t_begin; t < t_end; ++t) {                                            \
            double x0[6], c0[21], m[3 * MAXL], V[6 * MAXL], xo[6], co[21];                     \
            double ls[6 * MAXL], lc[21 * MAXL];                                                \
            for (int i = 0; i < 6; ++i) x0[i] = seed_state[i * T + t];                         \
            for (int i = 0; i < 21; ++i) c0[i] = seed_cov[i * T + t];                          \
            for (int l = 0; l < n_layers; ++l) {                                               \
                for (int i = 0; i < 3; ++i) m[3 * l + i] = hit_pos[((int64_t)l * 3 + i) * T + t]; \
                for (int i = 0; i < 6; ++i) V[6 * l + i] = hit_cov[((int64_t)l * 6 + i) * T + t]; \
            }                                                                                  \
            fit_one(n_layers, radii, x_over_x0, z_half, bz, x0, c0, charge[t], m, V,           \
                    hit_mask[t], xo, co, &out_chi2[t], &out_ndof[t], &out_flags[t],            \
                    layer_state ? ls : NULL, layer_cov ? lc : NULL);                           \
            for (int i = 0; i < 6; ++i) out_state[i * T + t] = xo[i];                          \
            for (int i = 0; i < 21; ++i) out_cov[i * T + t] = co[i];                           \
            for (int l = 0; l < n_layers; ++l) {                                               \
                if (layer_state)                                                               \
                    for (int i = 0; i < 6; ++i)                                                \
                        layer_state[((int64_t)l * 6 + i) * T + t] = ls[6 * l + i];             \
                if (layer_cov)                                                                 \
                    for (int i = 0; i < 21; ++i)                                               \
                        layer_cov[((int64_t)l * 21 + i) * T + t] = lc[21 * l + i];             \
            }                                                                                  \
        }                                                                                      \
        return 0;                                                                              \
    }

DEFINE_FIT_TRACKS(orc_fit_tracks, float)
DEFINE_FIT_TRACKS(orc_fit_tracks_f64, double)
