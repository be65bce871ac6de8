/*
 * Plain FP64 CPU oracle for seeding from hits: triplets of hits on the first
 * three layers of an event that a track from the beam line with pT above a
 * threshold could have made.  The paper seeds from the true hits of each
 * simulated track and says realistic seeding is under development (Section
 * 2); this is the seeding that replaces the truth.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite; shares no code with the
 * CUDA library.
 *
 * Pins (the CPU tests): the triplet circle against exact helices; the
 * triplets equal a brute force over every hit combination; every track that
 * passes the cuts is found with its charge; the seed start on exact helices
 * and on straight (two-charge) triplets.
 *
 * A triplet (h0, h1, h2), h_i a hit of seed layer i of one event, with hit
 * radii r_i = |(x_i, y_i)|, azimuths phi_i and z_i, is a seed when
 *   (a) |phi_1 - phi_0| <= dphi_01 and (e) |phi_2 - phi_1| <= dphi_12 (wrapped),
 *       dphi_ab = asin(R_b / 2 R_min) - asin(R_a / 2 R_min) + d0_max (1/R_a + 1/R_b)
 *       with R_a the layers' radii and R_min = pt_min / (k |Bz|);
 *   (b) the straight line through (r_0, z_0), (r_1, z_1) meets r = 0 within
 *       |z| <= z0_max;
 *   (d) that line predicts z at r_2 within dz_max;
 *   (c) the circle through the three (x, y) points has curvature
 *       |kappa| <= k |Bz| / pt_min (pT >= pt_min) and passes within d0_max of
 *       the origin.
 * kappa = 2 orient / (|P1 - P0| |P2 - P1| |P2 - P0|), orient =
 * (P1 - P0) x (P2 - P0); the origin's power with respect to the circle is
 * F = -incircle(P0, P1, P2, O) / orient, and its distance to the circle
 * d0 = |F| |kappa| / (1 + sqrt(max(0, 1 + F kappa^2))), which stays exact as
 * kappa -> 0.  Charge: a positive charge turns clockwise when Bz > 0, so
 * q = +1 when orient Bz < 0; below a curvature the hits cannot resolve (pT
 * above pt_both_charges) a triplet seeds both charges (the caller's choice,
 * from orc_triplet_circle).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORC_PI 3.14159265358979323846
#define ORC_K 0.00299792458

static double wrap(double d)
{
    while (d > ORC_PI) d -= 2.0 * ORC_PI;
    while (d <= -ORC_PI) d += 2.0 * ORC_PI;
    return d;
}

static double dphi_window(double ra, double rb, double rmin, double d0_max)
{
    const double sa = ra / (2.0 * rmin), sb = rb / (2.0 * rmin);
    return asin(sb < 1.0 ? sb : 1.0) - asin(sa < 1.0 ? sa : 1.0) + d0_max * (1.0 / ra + 1.0 / rb);
}

/* Curvature, distance of the origin to the circle and orientation of three
 * points; returns 0 if they are collinear. */
int orc_triplet_circle(const double *p0, const double *p1, const double *p2, double *kappa, double *d0,
                       double *orient_out)
{
    const double ax = p1[0] - p0[0], ay = p1[1] - p0[1];
    const double bx = p2[0] - p1[0], by = p2[1] - p1[1];
    const double cx = p2[0] - p0[0], cy = p2[1] - p0[1];
    const double orient = ax * cy - ay * cx;
    if (orient == 0.0) return 0;
    const double k = 2.0 * orient / (sqrt(ax * ax + ay * ay) * sqrt(bx * bx + by * by) * sqrt(cx * cx + cy * cy));
    /* incircle determinant of (P0, P1, P2) about the origin */
    const double s0 = p0[0] * p0[0] + p0[1] * p0[1], s1 = p1[0] * p1[0] + p1[1] * p1[1];
    const double s2 = p2[0] * p2[0] + p2[1] * p2[1];
    const double inc = p0[0] * (p1[1] * s2 - s1 * p2[1]) - p0[1] * (p1[0] * s2 - s1 * p2[0]) +
                       s0 * (p1[0] * p2[1] - p1[1] * p2[0]);
    const double F = -inc / orient;
    const double q = 1.0 + F * k * k;
    *kappa = k;
    *d0 = fabs(F) * fabs(k) / (1.0 + sqrt(q > 0.0 ? q : 0.0));
    *orient_out = orient;
    return 1;
}

/*
 * Triplets of events [e_begin, e_end): hit_pos [3][H] (all seed-layer hits),
 * offsets [E][4] (event e's hits of seed layer l are offsets[e][l] ..
 * offsets[e][l+1]-1), layer_r[3] the layers' radii.  Writes up to cap
 * triplets as out[n][4] = (event, h0, h1, h2) (global hit indices) in the
 * order event, h1, h0, h2; returns the number found (may exceed cap).
 */
int64_t orc_seed_triplets(const double *layer_r, double bz, double pt_min, double d0_max, double z0_max,
                          double dz_max, const float *hit_pos, int64_t H, const int64_t *offsets, int64_t e_begin,
                          int64_t e_end, int64_t *out, int64_t cap)
{
    const double rmin = pt_min / (ORC_K * fabs(bz)), kmax = ORC_K * fabs(bz) / pt_min;
    const double w01 = dphi_window(layer_r[0], layer_r[1], rmin, d0_max);
    const double w12 = dphi_window(layer_r[1], layer_r[2], rmin, d0_max);
    int64_t n = 0;
    double *phi = malloc((size_t)(H > 0 ? H : 1) * sizeof(double));
    if (!phi) return -1;
    for (int64_t e = e_begin; e < e_end; ++e)
        for (int64_t h = offsets[e * 4]; h < offsets[e * 4 + 3]; ++h) phi[h] = atan2(hit_pos[H + h], hit_pos[h]);
    for (int64_t e = e_begin; e < e_end; ++e) {
        const int64_t *off = offsets + e * 4;
        for (int64_t h1 = off[1]; h1 < off[2]; ++h1) {
            const double P1[2] = {hit_pos[h1], hit_pos[H + h1]}, z1 = hit_pos[2 * H + h1];
            const double r1 = hypot(P1[0], P1[1]);
            for (int64_t h0 = off[0]; h0 < off[1]; ++h0) {
                if (!(fabs(wrap(phi[h1] - phi[h0])) <= w01)) continue;
                const double P0[2] = {hit_pos[h0], hit_pos[H + h0]}, z0 = hit_pos[2 * H + h0];
                const double r0 = hypot(P0[0], P0[1]);
                const double zv = (z0 * r1 - z1 * r0) / (r1 - r0);
                if (!(fabs(zv) <= z0_max)) continue;
                for (int64_t h2 = off[2]; h2 < off[3]; ++h2) {
                    if (!(fabs(wrap(phi[h2] - phi[h1])) <= w12)) continue;
                    const double P2[2] = {hit_pos[h2], hit_pos[H + h2]}, z2 = hit_pos[2 * H + h2];
                    const double r2 = hypot(P2[0], P2[1]);
                    const double zp = z1 + (z1 - z0) * (r2 - r1) / (r1 - r0);
                    if (!(fabs(z2 - zp) <= dz_max)) continue;
                    double k, d0, orient;
                    if (!orc_triplet_circle(P0, P1, P2, &k, &d0, &orient)) continue;
                    if (!(fabs(k) <= kmax) || !(d0 <= d0_max)) continue;
                    if (n < cap) {
                        out[4 * n + 0] = e;
                        out[4 * n + 1] = h0;
                        out[4 * n + 2] = h1;
                        out[4 * n + 3] = h2;
                    }
                    ++n;
                }
            }
        }
    }
    free(phi);
    return n;
}
