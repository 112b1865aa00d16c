/*
 * synth.c — seeded synthetic sparse-tensor inputs.
 *
 * This module draws random numbers only: coordinates, values and dense
 * factor entries.  It holds none of the MTTKRP / CP arithmetic, so both the
 * CPU oracle and the GPU library can be fed from it without sharing code.
 *
 * Random source: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: draw number `ctr` of stream `key` is the SplitMix64 output
 * function applied to key + (ctr + 1) * gamma.  Every draw is therefore a
 * pure function of (seed, stream, counter), which makes the multithreaded
 * fills below bit-for-bit reproducible for any thread count.
 *
 * Zipf sampling: rejection-inversion of Hörmann & Derflinger ("Rejection-
 * inversion to generate variates from monotone discrete distributions",
 * ACM TOMACS 1996), without the squeeze shortcut; O(1) per draw, no table.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* key of stream `stream` under `seed` */
uint64_t synth_key(uint64_t seed, uint64_t stream) {
    return mix64(seed + GAMMA * (2 * stream + 1)) ^ mix64(stream + 0x632BE59BD9B4E019ULL);
}

/* draw `ctr` of the stream keyed `key` */
uint64_t synth_u64(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * GAMMA); }

/* uniform double in (0, 1] */
static inline double u01(uint64_t x) { return ((double)(x >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) (multiply-shift, Lemire 2019) */
static inline uint64_t below(uint64_t x, uint64_t n) {
    return (uint64_t)(((unsigned __int128)x * (unsigned __int128)n) >> 64);
}

/* ---- Zipf(s) on {1..n}: P(k) proportional to k^-s ---------------------- */
typedef struct {
    double s, n, lo, hi;  /* u is drawn uniformly in [lo, hi] */
} zipf_t;

/* log1p(t)/t and expm1(t)/t with their limits at t = 0 */
static double helper1(double t) { return fabs(t) > 1e-8 ? log1p(t) / t : 1.0 - t * (0.5 - t / 3.0); }
static double helper2(double t) { return fabs(t) > 1e-8 ? expm1(t) / t : 1.0 + t * 0.5 * (1.0 + t / 3.0); }
/* H(x) = integral of x^-s, normalised so that it is smooth in s at s = 1 */
static double zH(const zipf_t* z, double x) { double lx = log(x); return helper2((1.0 - z->s) * lx) * lx; }
static double zHinv(const zipf_t* z, double u) { double t = u * (1.0 - z->s); return exp(helper1(t) * u); }
static double zh(const zipf_t* z, double x) { return exp(-z->s * log(x)); }

static void zipf_init(zipf_t* z, double s, int64_t n) {
    z->s = s;
    z->n = (double)n;
    z->lo = zH(z, 1.5) - 1.0; /* interval of k = 1 has length h(1) = 1 */
    z->hi = zH(z, z->n + 0.5);
}

/* one Zipf draw, rank in [1, n]; attempts use counters (ctr<<6)|a, re-keyed after 64 */
static int64_t zipf_draw(const zipf_t* z, uint64_t key, uint64_t ctr) {
    for (uint64_t a = 0;; ++a) {
        uint64_t k2 = a < 64 ? key : mix64(key ^ (a >> 6) * GAMMA);
        double u = z->lo + u01(synth_u64(k2, (ctr << 6) | (a & 63))) * (z->hi - z->lo);
        double x = zHinv(z, u);
        double kd = floor(x + 0.5);
        if (kd < 1.0) kd = 1.0;
        if (kd > z->n) kd = z->n;
        /* accept iff u lies in the length-h(k) interval ending at H(k+1/2) */
        if (u >= zH(z, kd + 0.5) - zh(z, kd)) return (int64_t)kd;
    }
}

/* ---- public fills ----------------------------------------------------- */

/* Fisher-Yates permutation of [0, n) */
void synth_permutation(uint64_t seed, uint64_t stream, int64_t n, int32_t* perm) {
    uint64_t key = synth_key(seed, stream);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)below(synth_u64(key, (uint64_t)i), (uint64_t)(i + 1));
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* out[k*stride] uniform in [0, dim) for k < n */
void synth_index_uniform(uint64_t seed, uint64_t stream, int64_t n, int64_t dim, int32_t* out, int64_t stride) {
    uint64_t key = synth_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) out[k * stride] = (int32_t)below(synth_u64(key, (uint64_t)k), (uint64_t)dim);
}

/* out[k*stride] = perm[rank-1], rank ~ Zipf(s) on {1..dim}; perm NULL = identity */
void synth_index_zipf(uint64_t seed, uint64_t stream, int64_t n, int64_t dim, double s, const int32_t* perm,
                      int32_t* out, int64_t stride) {
    uint64_t key = synth_key(seed, stream);
    zipf_t z;
    zipf_init(&z, s, dim);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        int64_t r = zipf_draw(&z, key, (uint64_t)k) - 1;
        out[k * stride] = perm ? perm[r] : (int32_t)r;
    }
}

/* kind 0: U(lo,hi) ; 1: lognormal(mu=lo, sigma=hi) ; 2: normal(mean=lo, sd=hi) */
void synth_values(uint64_t seed, uint64_t stream, int64_t n, int kind, double lo, double hi, float* out) {
    uint64_t key = synth_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        if (kind == 0) {
            /* 24 random bits -> [0,1) exactly representable in float */
            double u = (double)(synth_u64(key, (uint64_t)k) >> 40) * (1.0 / 16777216.0);
            out[k] = (float)(lo + (hi - lo) * u);
        } else {
            /* Box-Muller, one normal per draw pair */
            double u1 = u01(synth_u64(key, 2 * (uint64_t)k));
            double u2 = u01(synth_u64(key, 2 * (uint64_t)k + 1));
            double zn = sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
            double v = lo + hi * zn;
            out[k] = (float)(kind == 1 ? exp(v) : v);
        }
    }
}
