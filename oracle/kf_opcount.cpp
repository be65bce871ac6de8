// Operation count of the FP64 oracle's track fit: the oracle's own source
// (kf_oracle.c), compiled as C++ with its floating-point type replaced by a
// scalar that counts every arithmetic operation it performs.
//
// TEST INFRASTRUCTURE ONLY: built and loaded by the test suite to measure the
// flops per track-layer of the oracle's dense formulation (6x6 matrix
// products, a Cholesky inverse); shares no code with the CUDA library.
//
// Counted: additions and subtractions, multiplications, divisions, square
// roots, and the other library calls (sin, cos, atan2, log, hypot, fmod), one
// each.
// Sign flips, comparisons, fabs and copies are not counted.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cmath>

typedef double plain_double;

namespace opcount {
unsigned long long n_add, n_mul, n_div, n_sqrt, n_fun;
}

struct CountedReal {
    plain_double v;
    CountedReal() = default;
    CountedReal(plain_double x) : v(x) {}
    explicit operator plain_double() const { return v; }
    explicit operator float() const { return (float)v; }
    explicit operator int() const { return (int)v; }
    CountedReal operator-() const { return CountedReal(-v); }
    CountedReal &operator+=(CountedReal b)
    {
        ++opcount::n_add;
        v += b.v;
        return *this;
    }
    CountedReal &operator-=(CountedReal b)
    {
        ++opcount::n_add;
        v -= b.v;
        return *this;
    }
    CountedReal &operator*=(CountedReal b)
    {
        ++opcount::n_mul;
        v *= b.v;
        return *this;
    }
    CountedReal &operator/=(CountedReal b)
    {
        ++opcount::n_div;
        v /= b.v;
        return *this;
    }
};

inline CountedReal operator+(CountedReal a, CountedReal b) { return a += b; }
inline CountedReal operator-(CountedReal a, CountedReal b) { return a -= b; }
inline CountedReal operator*(CountedReal a, CountedReal b) { return a *= b; }
inline CountedReal operator/(CountedReal a, CountedReal b) { return a /= b; }
inline bool operator<(CountedReal a, CountedReal b) { return a.v < b.v; }
inline bool operator>(CountedReal a, CountedReal b) { return a.v > b.v; }
inline bool operator<=(CountedReal a, CountedReal b) { return a.v <= b.v; }
inline bool operator>=(CountedReal a, CountedReal b) { return a.v >= b.v; }
inline bool operator==(CountedReal a, CountedReal b) { return a.v == b.v; }
inline bool operator!=(CountedReal a, CountedReal b) { return a.v != b.v; }
inline bool operator!(CountedReal a) { return !a.v; }
inline CountedReal sqrt(CountedReal a)
{
    ++opcount::n_sqrt;
    return CountedReal(std::sqrt(a.v));
}
inline CountedReal fabs(CountedReal a) { return CountedReal(std::fabs(a.v)); }
inline CountedReal sin(CountedReal a)
{
    ++opcount::n_fun;
    return CountedReal(std::sin(a.v));
}
inline CountedReal cos(CountedReal a)
{
    ++opcount::n_fun;
    return CountedReal(std::cos(a.v));
}
inline CountedReal log(CountedReal a)
{
    ++opcount::n_fun;
    return CountedReal(std::log(a.v));
}
inline CountedReal atan2(CountedReal a, CountedReal b)
{
    ++opcount::n_fun;
    return CountedReal(std::atan2(a.v, b.v));
}
inline CountedReal hypot(CountedReal a, CountedReal b)
{
    ++opcount::n_fun;
    return CountedReal(std::hypot(a.v, b.v));
}
inline CountedReal fmod(CountedReal a, CountedReal b)
{
    ++opcount::n_fun;
    return CountedReal(std::fmod(a.v, b.v));
}
inline bool isfinite(CountedReal a) { return std::isfinite(a.v); }

#define double CountedReal
#include "kf_oracle.c"
#undef double

// Fit tracks [0, n_tracks) exactly as orc_fit_tracks does and return the
// operations the fits performed: counts[0..4] = additions, multiplications,
// divisions, square roots, other library calls; counts[5] = their sum;
// counts[6] = the layers the fits processed (sum over tracks of the layers
// reached).
extern "C" int orc_count_fit(int n_layers, const plain_double *radii, const plain_double *x_over_x0,
                             plain_double z_half, plain_double bz, int64_t n_tracks, const float *seed_state,
                             const float *seed_cov, const int8_t *charge, const float *hit_pos,
                             const float *hit_cov, const uint32_t *hit_mask, unsigned long long *counts)
{
    if (n_layers < 0 || n_layers > MAXL) return -1;
    opcount::n_add = opcount::n_mul = opcount::n_div = opcount::n_sqrt = opcount::n_fun = 0;
    const int64_t T = n_tracks;
    CountedReal r[MAXL], xx0[MAXL];
    for (int l = 0; l < n_layers; ++l) {
        r[l] = radii[l];
        xx0[l] = x_over_x0[l];
    }
    unsigned long long layers = 0;
    for (int64_t t = 0; t < T; ++t) {
        CountedReal x0[6], c0[21], m[3 * MAXL], V[6 * MAXL], xo[6], co[21], chi2;
        CountedReal ls[6 * MAXL];
        for (int i = 0; i < 6; ++i) x0[i] = seed_state[i * T + t];
        for (int i = 0; i < 21; ++i) c0[i] = seed_cov[i * T + t];
        for (int l = 0; l < n_layers; ++l) {
            for (int i = 0; i < 3; ++i) m[3 * l + i] = hit_pos[((int64_t)l * 3 + i) * T + t];
            for (int i = 0; i < 6; ++i) V[6 * l + i] = hit_cov[((int64_t)l * 6 + i) * T + t];
        }
        int32_t ndof = 0;
        uint32_t flags = 0;
        // per-layer states mark the layers reached (NaN beyond the stop)
        fit_one(n_layers, r, xx0, CountedReal(z_half), CountedReal(bz), x0, c0, charge[t], m, V, hit_mask[t], xo,
                co, &chi2, &ndof, &flags, ls, nullptr);
        for (int l = 0; l < n_layers; ++l)
            if (std::isfinite(ls[6 * l].v)) ++layers;
    }
    counts[0] = opcount::n_add;
    counts[1] = opcount::n_mul;
    counts[2] = opcount::n_div;
    counts[3] = opcount::n_sqrt;
    counts[4] = opcount::n_fun;
    counts[5] = opcount::n_add + opcount::n_mul + opcount::n_div + opcount::n_sqrt + opcount::n_fun;
    counts[6] = layers;
    return 0;
}
