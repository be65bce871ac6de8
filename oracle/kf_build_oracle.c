/*
 * Plain FP64 CPU oracle for the per-layer step of combinatorial track
 * building (Sections 3, 3.1 and 4.3 of arXiv:1705.02876).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark.  Shares no code with the CUDA
 * library.
 *
 * Pins (the CPU tests): on tiny events the kept candidates equal the best N
 * of fits of every hit sequence, enumerated by brute force; N = 1 is the
 * best-hit search; the capped windows hold exactly the hits of a brute-force
 * box; noise-free events give every seed its own track's hits; efficiency and
 * fake rate land where the paper reports them for its toy detector.  For the
 * proposal: BF16 rounding against hand-worked ties; the logit against the
 * perceptron's definition in mlp_oracle.py; the training log against the
 * plain build it records (build unchanged, labels on the surviving hits, rows
 * inside the windows); a proposal wider than every window is the exhaustive
 * build.
 *
 * The clone engine (Section 3.1): at each layer every candidate of a seed
 * yields one child per compatible hit plus one child without a hit (a hole);
 * the children are ranked by number of hits (more first) and chi2 (less
 * first) (Section 4.3), and only the best N survive, each updated with its
 * hit.  With N = 1 this is the best-hit approach (Section 3: the hit with the
 * lowest chi2 increment).  Readings taken here (the paper gives no
 * numbers): a hit is compatible if it lies in the window
 *   |dphi| <= nsigma sqrt(sigma_rphi,pred^2 + sigma_rphi,hit^2) / r,
 *   |dz|   <= nsigma sqrt(sigma_z,pred^2 + sigma_z,hit^2)
 * around the predicted crossing (half-widths capped at dphi_max and dz_max:
 * a candidate whose prediction has lost its precision, as near a tangential
 * crossing, does not search the whole layer) and its chi2 increment is at
 * most chi2_cut;
 * ties in (hits, chi2) go to the lower candidate index, then the lower hit
 * index within the layer (the hole first); a candidate that cannot reach a
 * layer or crosses it beyond |z| = z_half stops and yields only its hole child
 * from then on, with its state unchanged.
 *
 * Hits of one (event, layer) are found through an index sorted by phi: the
 * in-window set is exactly that of a scan over all of the layer's hits.
 *
 * Not in the paper: the learned hit proposal.  Optionally the build logs, for
 * every (candidate, hit) pair with the hit in the window, the proposal's 12
 * inputs and a label (1 if the pair became a surviving child at that layer);
 * and optionally a perceptron 12 -> 64 -> 64 -> 1 (ReLU) scores the in-window
 * hits of a candidate whose window holds more than topk of them, and only the
 * topk best by logit (ties to the lower hit index within the layer) are
 * tested against the chi2 cut.  The inputs, in the layer's local frame
 * (n = radial unit vector at the predicted crossing, t = z x n):
 *   0..2  (n.d, t.d, d_z) / sqrt(S_nn, S_tt, S_zz), d = hit - prediction,
 *         S = C_pos + V;
 *   3..8  log10 of the predicted covariance diagonal (floor 1e-30);
 *   9     q / pT of the prediction, signed by q B;
 *   10    the layer's index among the build layers / their number;
 *   11    the candidate's holes so far (layer index - hits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define MAXL 64
#define MAXN 16

int orc_propagate(const double *st, int q, double bz, double r, double *out, double *J, double *s_out);
void orc_ms_noise(const double *st, double x_over_x0, double *Q);
void orc_transport(const double *J, double *C, const double *Q);
int orc_update(double *x, double *C, const double *m, const double *Vp, double *dchi2);
int orc_inv3_cholesky(const double *S, double *Sinv);
void orc_unpack_sym(const double *packed, int n, double *full);

/* ------------------------------------------------------------------------ */
/* phi index of every (event, layer) segment                                 */

static const double *g_sort_phi;
static int cmp_phi(const void *a, const void *b)
{
    const double pa = g_sort_phi[*(const int64_t *)a], pb = g_sort_phi[*(const int64_t *)b];
    if (pa < pb) return -1;
    if (pa > pb) return 1;
    return (*(const int64_t *)a > *(const int64_t *)b) - (*(const int64_t *)a < *(const int64_t *)b);
}

/* phi[H] = atan2(y, x) of every hit; order[H] = within each segment
 * [offsets[k], offsets[k+1]) the hit indices sorted by phi.  Not thread-safe
 * (uses a file-scope comparator pointer); called once before the build. */
void orc_build_prepare(int64_t n_segments, const int64_t *offsets, const float *hit_pos, int64_t H, double *phi,
                       int64_t *order)
{
    for (int64_t h = 0; h < H; ++h) phi[h] = atan2((double)hit_pos[1 * H + h], (double)hit_pos[0 * H + h]);
    for (int64_t k = 0; k < n_segments; ++k) {
        for (int64_t h = offsets[k]; h < offsets[k + 1]; ++h) order[h] = h;
        g_sort_phi = phi;
        qsort(order + offsets[k], (size_t)(offsets[k + 1] - offsets[k]), sizeof(int64_t), cmp_phi);
    }
}

/* ------------------------------------------------------------------------ */

typedef struct {
    double x[6], C[36];  /* current state */
    double xp[6], Cp[36]; /* predicted at this layer */
    double chi2;
    int nhits, stopped, reached;
    int32_t hits[MAXL];
} cand_t;

typedef struct {
    int cand, nhits;
    int64_t hit_local; /* -1 for the hole */
    int64_t hit_global;
    double chi2;       /* candidate chi2 + increment */
    double dchi2;
    int64_t row;       /* row of the training log, -1 if none */
} child_t;

/* (hits desc, chi2 asc, candidate asc, hit asc) */
static int child_before(const child_t *a, const child_t *b)
{
    if (a->nhits != b->nhits) return a->nhits > b->nhits;
    if (a->chi2 != b->chi2) return a->chi2 < b->chi2;
    if (a->cand != b->cand) return a->cand < b->cand;
    return a->hit_local < b->hit_local;
}
static int cmp_child(const void *a, const void *b)
{
    const child_t *x = a, *y = b;
    if (child_before(x, y)) return -1;
    if (child_before(y, x)) return 1;
    return 0;
}

static double wrap_phi(double d)
{
    while (d > ORC_PI) d -= 2.0 * ORC_PI;
    while (d <= -ORC_PI) d += 2.0 * ORC_PI;
    return d;
}

/* first position p in order[lo, hi) with phi[order[p]] >= v */
static int64_t lower_phi(const double *phi, const int64_t *order, int64_t lo, int64_t hi, double v)
{
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (phi[order[mid]] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Chi2 increment of hit h against the predicted state; returns 0 if S is
 * not positive definite. */
static int hit_chi2(const double *xp, const double *Cp, const float *hit_pos, const float *hit_cov, int64_t H,
                    int64_t h, double *out)
{
    double V[9], S[9], Si[9], r[3], vp[6];
    for (int i = 0; i < 6; ++i) vp[i] = hit_cov[(int64_t)i * H + h];
    orc_unpack_sym(vp, 3, V);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i * 3 + j] = Cp[i * 6 + j] + V[i * 3 + j];
    if (orc_inv3_cholesky(S, Si)) return 0;
    for (int i = 0; i < 3; ++i) r[i] = (double)hit_pos[(int64_t)i * H + h] - xp[i];
    double c = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c += r[i] * Si[i * 3 + j] * r[j];
    *out = c;
    return 1;
}

/* keep the n best hit children of one candidate, sorted by key */
static void insert_child(child_t *list, int *count, int n, const child_t *c)
{
    int k = *count;
    if (k == n && !child_before(c, &list[n - 1])) return;
    if (k < n) ++k;
    int p = k - 1;
    while (p > 0 && child_before(c, &list[p - 1])) {
        list[p] = list[p - 1];
        --p;
    }
    list[p] = *c;
    *count = k;
}

/* The proposal's inputs for hit h against the predicted candidate. */
static void pair_features(const double *xp, const double *Cp, int q, double bz, int l, int L, int nhits,
                          const float *hit_pos, const float *hit_cov, int64_t H, int64_t h, double *f)
{
    double V[9], vp[6], d[3];
    for (int i = 0; i < 6; ++i) vp[i] = hit_cov[(int64_t)i * H + h];
    orc_unpack_sym(vp, 3, V);
    for (int i = 0; i < 3; ++i) d[i] = (double)hit_pos[(int64_t)i * H + h] - xp[i];
    const double rc = hypot(xp[0], xp[1]);
    const double n[2] = {xp[0] / rc, xp[1] / rc}, t[2] = {-xp[1] / rc, xp[0] / rc};
    double snn = 0.0, stt = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const double sij = Cp[i * 6 + j] + V[i * 3 + j];
            snn += n[i] * sij * n[j];
            stt += t[i] * sij * t[j];
        }
    const double szz = Cp[2 * 6 + 2] + V[2 * 3 + 2];
    f[0] = (n[0] * d[0] + n[1] * d[1]) / sqrt(snn > 1e-30 ? snn : 1e-30);
    f[1] = (t[0] * d[0] + t[1] * d[1]) / sqrt(stt > 1e-30 ? stt : 1e-30);
    f[2] = d[2] / sqrt(szz > 1e-30 ? szz : 1e-30);
    for (int i = 0; i < 6; ++i) {
        const double c = Cp[i * 6 + i];
        f[3 + i] = log10(c > 1e-30 ? c : 1e-30);
    }
    const double pt = hypot(xp[3], xp[4]);
    f[9] = ((double)q * bz < 0.0 ? -1.0 : 1.0) / pt;
    f[10] = (double)l / (double)L;
    f[11] = (double)(l - nhits);
}

/* v rounded to float32, then to bfloat16 (8-bit significand, round to
 * nearest, ties to even), returned as a double. */
double orc_bf16_round(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* Logit of the perceptron; w = W1 [12][64], b1 [64], W2 [64][64], b2 [64],
 * W3 [64], b3.  bf16 != 0 takes the top-k decision in the precision of the
 * tensor-core scoring: inputs, W1, W2 and the first hidden layer rounded to
 * bfloat16 (the biases, W3 and the sums stay wide). */
double orc_mlp_logit(const double *w, const double *f, int bf16)
{
    const double *W1 = w, *b1 = W1 + 12 * 64, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64, *b3 = W3 + 64;
    double h1[64], x[12], z = b3[0];
    for (int i = 0; i < 12; ++i) x[i] = bf16 ? orc_bf16_round(f[i]) : f[i];
    for (int j = 0; j < 64; ++j) {
        double a = 0.0;
        for (int i = 0; i < 12; ++i) a += x[i] * (bf16 ? orc_bf16_round(W1[i * 64 + j]) : W1[i * 64 + j]);
        a += b1[j];
        h1[j] = a > 0.0 ? a : 0.0;
        if (bf16) h1[j] = orc_bf16_round(h1[j]);
    }
    for (int j = 0; j < 64; ++j) {
        double a = 0.0;
        for (int i = 0; i < 64; ++i) a += h1[i] * (bf16 ? orc_bf16_round(W2[i * 64 + j]) : W2[i * 64 + j]);
        a += b2[j];
        z += W3[j] * (a > 0.0 ? a : 0.0);
    }
    return z;
}

typedef struct {
    int64_t h;
    double z;
} scored_t;

/* (logit desc, hit index asc) */
static int cmp_scored(const void *a, const void *b)
{
    const scored_t *x = a, *y = b;
    if (x->z != y->z) return x->z > y->z ? -1 : 1;
    return (x->h > y->h) - (x->h < y->h);
}

/* The phi intervals [lo, hi] of a window of half-width dphi around phic,
 * split at +-pi (one interval covering everything when dphi >= pi). */
static int window_intervals(double phic, double dphi, double lo_[3], double hi_[3])
{
    int nint = 0;
    const double a = phic - dphi, b = phic + dphi;
    if (dphi >= ORC_PI) {
        lo_[0] = -ORC_PI - 1.0;
        hi_[0] = ORC_PI + 1.0;
        return 1;
    }
    lo_[nint] = a < -ORC_PI ? -ORC_PI - 1.0 : a;
    hi_[nint] = b > ORC_PI ? ORC_PI + 1.0 : b;
    ++nint;
    if (a < -ORC_PI) {
        lo_[nint] = a + 2.0 * ORC_PI;
        hi_[nint] = ORC_PI + 1.0;
        ++nint;
    }
    if (b > ORC_PI) {
        lo_[nint] = -ORC_PI - 1.0;
        hi_[nint] = b - 2.0 * ORC_PI;
        ++nint;
    }
    return nint;
}

/*
 * Build seeds [s_begin, s_end).  Geometry: the build layers only.  Hits: all
 * layers of all events in hit_pos [3][H], hit_cov [6][H]; hit_offsets
 * [n_events][L+1]; phi and order from orc_build_prepare.  Seeds: seed_event
 * [S], state [6][S], cov [21][S] packed, charge [S] (float32).
 * Outputs (slot j of seed s = rank j after the last layer): out_hit
 * [S][N][L] global hit index or -1; out_chi2, out_nhits (-1 for an empty
 * slot) [S][N]; out_state [6][S*N]; out_cov [21][S*N] packed; out_ncand [S].
 * orc_build_tracks_ex adds the training log (log_f [cap][12], log_y [cap],
 * log_ref [cap][4] = seed, candidate, layer, hit; *log_n counts the pairs met,
 * rows past log_cap are dropped; log_n NULL = no log) and the proposal (mlp
 * the 5,057 weights, NULL = exhaustive search; topk >= 1; mlp_bf16 as in
 * mlp_logit).
 *
 * out_margin [S][4] (NULL = none) is a diagnostic for parity tests: for each
 * seed, over all its layers and candidates, how close each kind of decision
 * came to going the other way, as a relative distance (0 = on the edge):
 *   [0] a hit's window test, max(|dphi| / dphi_w, |dz| / dz_w) against 1 for
 *       the hits of a window 1.05 times wider, and a crossing's |z| against
 *       z_half;
 *   [1] a tested hit's chi2 increment against the cut, |dchi2 - cut| / cut;
 *   [2] the ranking: two children next to each other among a seed's first
 *       N + 1, or among a candidate's best N + 1 hit children (its list is
 *       cut at N), with the same number of hits, |chi2_a - chi2_b| /
 *       max(1, chi2_a);
 *   [3] the proposal's top-k: the logits at ranks topk and topk + 1,
 *       (z_k - z_k+1) / (1 + |z_k|).
 * Infinity where the seed met no such decision.  It takes no part in the
 * build.
 */
int orc_build_tracks_ex(int n_layers, const double *radii, const double *x_over_x0, double z_half, double bz,
                     const int64_t *hit_offsets, const float *hit_pos, const float *hit_cov, int64_t H,
                     const double *phi, const int64_t *order, int64_t s_begin, int64_t s_end, int64_t n_seeds,
                     const int32_t *seed_event, const float *seed_state, const float *seed_cov,
                     const int8_t *seed_charge, int max_cands, double chi2_cut, double nsigma,
                     double sigma_rphi_hit, double sigma_z_hit, int32_t *out_hit, double *out_chi2,
                     int32_t *out_nhits, double *out_state, double *out_cov, int32_t *out_ncand, double *log_f,
                     double *log_y, int32_t *log_ref, int64_t log_cap, int64_t *log_n, const double *mlp,
                     int topk, int mlp_bf16, double dphi_max, double dz_max, double *out_margin)
{
    const int N = max_cands, L = n_layers;
    const int64_t S = n_seeds;
    if (N < 1 || N > MAXN || L < 1 || L > MAXL || (mlp && topk < 1)) return -1;
    int64_t win_cap = 256;
    scored_t *win = malloc((size_t)win_cap * sizeof(scored_t));
    if (!win) return -2;
    cand_t cand[MAXN], next[MAXN];
    child_t hits_of[MAXN][MAXN], all[MAXN * (MAXN + 1)];
    child_t hits_m[MAXN + 1]; /* margins: a candidate's best N + 1 hit children */
    int nh[MAXN];
    for (int64_t s = s_begin; s < s_end; ++s) {
        double mg[4] = {HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL};
        const int q = seed_charge[s];
        const int64_t *off = hit_offsets + (int64_t)seed_event[s] * (L + 1);
        int nc = 1;
        memset(&cand[0], 0, sizeof(cand_t));
        for (int i = 0; i < 6; ++i) cand[0].x[i] = seed_state[(int64_t)i * S + s];
        {
            double cp[21];
            for (int i = 0; i < 21; ++i) cp[i] = seed_cov[(int64_t)i * S + s];
            orc_unpack_sym(cp, 6, cand[0].C);
        }
        for (int l = 0; l < L; ++l) cand[0].hits[l] = -1;

        for (int l = 0; l < L; ++l) {
            int n_all = 0;
            const int64_t seg_lo = off[l], seg_hi = off[l + 1];
            for (int c = 0; c < nc; ++c) {
                cand_t *k = &cand[c];
                nh[c] = 0;
                int nhm = 0;
                k->reached = 0;
                if (!k->stopped) {
                    double J[36], Q[36], sd;
                    const int unreachable = orc_propagate(k->x, q, bz, radii[l], k->xp, J, &sd);
                    if (!unreachable) mg[0] = fmin(mg[0], fabs(fabs(k->xp[2]) - z_half) / z_half);
                    if (unreachable || fabs(k->xp[2]) > z_half) {
                        k->stopped = 1;
                    } else {
                        memcpy(k->Cp, k->C, sizeof k->C);
                        orc_ms_noise(k->xp, x_over_x0[l], Q);
                        orc_transport(J, k->Cp, Q);
                        k->reached = 1;
                    }
                }
                if (k->reached) {
                    const double xp = k->xp[0], yp = k->xp[1], zp = k->xp[2];
                    const double rc = hypot(xp, yp);
                    const double tx = -yp / rc, ty = xp / rc;
                    const double var_rphi = tx * tx * k->Cp[0] + 2.0 * tx * ty * k->Cp[1] + ty * ty * k->Cp[7];
                    const double dphi =
                        fmin(nsigma * sqrt(var_rphi + sigma_rphi_hit * sigma_rphi_hit) / radii[l], dphi_max);
                    const double dz = fmin(nsigma * sqrt(k->Cp[14] + sigma_z_hit * sigma_z_hit), dz_max);
                    const double phic = atan2(yp, xp);
                    /* phi intervals of the window, split at +-pi */
                    double lo_[3], hi_[3];
                    const int nint = window_intervals(phic, dphi, lo_, hi_);
                    if (out_margin) {
                        /* window edges: every hit of the window 1.05 times wider */
                        double mlo[3], mhi[3];
                        const int mint = window_intervals(phic, 1.05 * dphi, mlo, mhi);
                        for (int iv = 0; iv < mint; ++iv)
                            for (int64_t p = lower_phi(phi, order, seg_lo, seg_hi, mlo[iv]);
                                 p < seg_hi && phi[order[p]] <= mhi[iv]; ++p) {
                                const int64_t h = order[p];
                                const double ep = fabs(wrap_phi(phi[h] - phic)) / dphi;
                                const double ez = fabs((double)hit_pos[2 * H + h] - zp) / dz;
                                if (ep > 1.05 || ez > 1.05) continue;
                                mg[0] = fmin(mg[0], fabs((ep > ez ? ep : ez) - 1.0));
                            }
                    }
                    /* the in-window hits */
                    int64_t n_in = 0;
                    for (int iv = 0; iv < nint; ++iv) {
                        for (int64_t p = lower_phi(phi, order, seg_lo, seg_hi, lo_[iv]);
                             p < seg_hi && phi[order[p]] <= hi_[iv]; ++p) {
                            const int64_t h = order[p];
                            if (!(fabs(wrap_phi(phi[h] - phic)) <= dphi)) continue;
                            if (!(fabs((double)hit_pos[2 * H + h] - zp) <= dz)) continue;
                            if (n_in == win_cap) {
                                scored_t *w2 = realloc(win, (size_t)(2 * win_cap) * sizeof(scored_t));
                                if (!w2) {
                                    free(win);
                                    return -2;
                                }
                                win = w2;
                                win_cap *= 2;
                            }
                            win[n_in].h = h;
                            win[n_in].z = 0.0;
                            ++n_in;
                        }
                    }
                    int64_t n_test = n_in;
                    if (mlp && n_in > topk) {
                        for (int64_t i = 0; i < n_in; ++i) {
                            double f[12];
                            pair_features(k->xp, k->Cp, q, bz, l, L, k->nhits, hit_pos, hit_cov, H, win[i].h, f);
                            win[i].z = orc_mlp_logit(mlp, f, mlp_bf16);
                        }
                        qsort(win, (size_t)n_in, sizeof(scored_t), cmp_scored);
                        n_test = topk;
                        mg[3] = fmin(mg[3], (win[topk - 1].z - win[topk].z) / (1.0 + fabs(win[topk - 1].z)));
                    }
                    for (int64_t i = 0; i < n_test; ++i) {
                        const int64_t h = win[i].h;
                        int64_t row = -1;
                        if (log_n) {
                            row = (*log_n)++;
                            if (row < log_cap) {
                                pair_features(k->xp, k->Cp, q, bz, l, L, k->nhits, hit_pos, hit_cov, H, h,
                                              log_f + row * 12);
                                log_y[row] = 0.0;
                                log_ref[row * 4 + 0] = (int32_t)s;
                                log_ref[row * 4 + 1] = c;
                                log_ref[row * 4 + 2] = l;
                                log_ref[row * 4 + 3] = (int32_t)h;
                            } else {
                                row = -1;
                            }
                        }
                        double dc;
                        if (!hit_chi2(k->xp, k->Cp, hit_pos, hit_cov, H, h, &dc)) continue;
                        mg[1] = fmin(mg[1], fabs(dc - chi2_cut) / chi2_cut);
                        if (!(dc <= chi2_cut)) continue;
                        child_t ch = {c, k->nhits + 1, h - seg_lo, h, k->chi2 + dc, dc, row};
                        insert_child(hits_of[c], &nh[c], N, &ch);
                        if (out_margin) insert_child(hits_m, &nhm, N + 1, &ch);
                    }
                    /* the cap of a candidate's list at N children is a ranking too */
                    for (int j = 0; j + 1 < nhm; ++j)
                        mg[2] = fmin(mg[2], fabs(hits_m[j].chi2 - hits_m[j + 1].chi2) / fmax(1.0, hits_m[j].chi2));
                }
                for (int i = 0; i < nh[c]; ++i) all[n_all++] = hits_of[c][i];
                child_t hole = {c, k->nhits, -1, -1, k->chi2, 0.0, -1};
                all[n_all++] = hole;
            }
            qsort(all, (size_t)n_all, sizeof(child_t), cmp_child);
            const int nn = n_all < N ? n_all : N;
            for (int j = 0; j + 1 < n_all && j < N; ++j)
                if (all[j].nhits == all[j + 1].nhits)
                    mg[2] = fmin(mg[2], fabs(all[j].chi2 - all[j + 1].chi2) / fmax(1.0, all[j].chi2));
            for (int j = 0; j < nn; ++j) {
                const child_t *ch = &all[j];
                const cand_t *par = &cand[ch->cand];
                cand_t *o = &next[j];
                *o = *par;
                o->stopped = par->stopped;
                if (par->reached) {
                    memcpy(o->x, par->xp, sizeof o->x);
                    memcpy(o->C, par->Cp, sizeof o->C);
                }
                if (ch->hit_local >= 0) {
                    double m[3], vp[6], d;
                    if (ch->row >= 0) log_y[ch->row] = 1.0;
                    for (int i = 0; i < 3; ++i) m[i] = hit_pos[(int64_t)i * H + ch->hit_global];
                    for (int i = 0; i < 6; ++i) vp[i] = hit_cov[(int64_t)i * H + ch->hit_global];
                    orc_update(o->x, o->C, m, vp, &d);
                    o->nhits = ch->nhits;
                    o->chi2 = ch->chi2;
                    o->hits[l] = (int32_t)ch->hit_global;
                } else {
                    o->hits[l] = -1;
                }
            }
            memcpy(cand, next, (size_t)nn * sizeof(cand_t));
            nc = nn;
        }
        out_ncand[s] = nc;
        if (out_margin)
            for (int i = 0; i < 4; ++i) out_margin[s * 4 + i] = mg[i];
        for (int j = 0; j < N; ++j) {
            const int64_t sj = s * N + j;
            for (int l = 0; l < L; ++l) out_hit[sj * L + l] = j < nc ? cand[j].hits[l] : -1;
            out_chi2[sj] = j < nc ? cand[j].chi2 : 0.0;
            out_nhits[sj] = j < nc ? cand[j].nhits : -1;
            for (int i = 0; i < 6; ++i) out_state[(int64_t)i * S * N + sj] = j < nc ? cand[j].x[i] : 0.0;
            for (int i = 0; i < 6; ++i)
                for (int jj = 0; jj <= i; ++jj)
                    out_cov[(int64_t)(i * (i + 1) / 2 + jj) * S * N + sj] = j < nc ? cand[j].C[i * 6 + jj] : 0.0;
        }
    }
    free(win);
    return 0;
}

int orc_build_tracks(int n_layers, const double *radii, const double *x_over_x0, double z_half, double bz,
                     const int64_t *hit_offsets, const float *hit_pos, const float *hit_cov, int64_t H,
                     const double *phi, const int64_t *order, int64_t s_begin, int64_t s_end, int64_t n_seeds,
                     const int32_t *seed_event, const float *seed_state, const float *seed_cov,
                     const int8_t *seed_charge, int max_cands, double chi2_cut, double nsigma,
                     double sigma_rphi_hit, double sigma_z_hit, int32_t *out_hit, double *out_chi2,
                     int32_t *out_nhits, double *out_state, double *out_cov, int32_t *out_ncand)
{
    return orc_build_tracks_ex(n_layers, radii, x_over_x0, z_half, bz, hit_offsets, hit_pos, hit_cov, H, phi, order,
                               s_begin, s_end, n_seeds, seed_event, seed_state, seed_cov, seed_charge, max_cands,
                               chi2_cut, nsigma, sigma_rphi_hit, sigma_z_hit, out_hit, out_chi2, out_nhits,
                               out_state, out_cov, out_ncand, NULL, NULL, NULL, 0, NULL, NULL, 1, 0, HUGE_VAL,
                               HUGE_VAL, NULL);
}
