/*
 * Seeded synthetic inputs for the GAS superstep engine and its oracle.
 *
 * This file holds random-number and sampling code only: no step of the
 * superstep method (no message generation, merge or apply) lives here. The
 * CUDA path and the CPU oracle both consume what it writes.
 *
 * Random numbers: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator. Value i (i = 0, 1, ...) of the stream with seed S is the
 * SplitMix64 output after i+1 state increments:
 *     z  = S + (i + 1) * 0x9E3779B97F4A7C15          (mod 2^64)
 *     z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
 *     z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
 *     out = z ^ (z >> 31)
 * Because every value is a pure function of (S, i), the generators below are
 * order-free and parallel, and give the same bits on every host.
 *
 * Uniform doubles take the top 53 bits: u = (out >> 11) * 2^-53, in [0, 1).
 * Bounded integers in [0, k) take the high word of (out >> 32) * k, i.e.
 * ((out >> 32) * k) >> 32 (Lemire's multiply-shift), for k < 2^32.
 *
 * Build: plain C99, optional OpenMP. Built as its own shared library.
 */
#include <stdint.h>
#include <stddef.h>

#define GXS_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gxs_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Value i of the SplitMix64 stream seeded with `seed`. */
uint64_t gxs_u64(uint64_t seed, uint64_t i) {
    return gxs_mix(seed + (i + 1ULL) * GXS_GAMMA);
}

static inline double gxs_unit(uint64_t r) {
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

static inline uint32_t gxs_below(uint64_t r, uint32_t k) {
    return (uint32_t)(((r >> 32) * (uint64_t)k) >> 32);
}

/* Fill out[0..n) with values i0 .. i0+n-1 of stream `seed`. */
void gxs_fill_u64(uint64_t seed, uint64_t i0, uint64_t n, uint64_t* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = gxs_u64(seed, i0 + (uint64_t)i);
}

/* Fill out[0..n) with uniform doubles in [0,1) from values i0.. of stream `seed`. */
void gxs_fill_unit(uint64_t seed, uint64_t i0, uint64_t n, double* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = gxs_unit(gxs_u64(seed, i0 + (uint64_t)i));
}

/*
 * R-MAT edge list (D. Chakrabarti, Y. Zhan, C. Faloutsos, "R-MAT: A recursive
 * model for graph mining", SDM 2004): n = 2^scale vertices, n_edges directed
 * edges. Edge i descends `scale` levels, most significant bit first; at level
 * l it draws u = unit(value i*scale + l) and picks the quadrant
 *     u < a          -> (src bit 0, dst bit 0)
 *     u < a+b        -> (0, 1)
 *     u < a+b+c      -> (1, 0)
 *     otherwise      -> (1, 1)
 * No noise, no id permutation; duplicates and self-loops are kept.
 */
void gxs_rmat(uint32_t scale, uint64_t n_edges, double a, double b, double c,
              uint64_t seed, uint32_t* src, uint32_t* dst) {
    const double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n_edges; ++i) {
        uint32_t s = 0, d = 0;
        const uint64_t base = (uint64_t)i * scale;
        for (uint32_t l = 0; l < scale; ++l) {
            const double u = gxs_unit(gxs_u64(seed, base + l));
            uint32_t sb, db;
            if (u < a)        { sb = 0; db = 0; }
            else if (u < ab)  { sb = 0; db = 1; }
            else if (u < abc) { sb = 1; db = 0; }
            else              { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        src[i] = s;
        dst[i] = d;
    }
}

/*
 * Erdős–Rényi G(n, m) as m uniform unordered pairs {u, v}, u != v, duplicates
 * kept, each stored in both directions: edge 2i = (u -> v), edge 2i+1 =
 * (v -> u). Pair i tries attempts j = 0..15: u = below(value 2(16i+j), n),
 * v = below(value 2(16i+j)+1, n), and keeps the first attempt with u != v.
 * If all 16 fail (possible only for tiny n), v = (u + 1) mod n.
 * Requires n >= 2.
 */
void gxs_er(uint64_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        uint32_t u = 0, v = 0;
        int ok = 0;
        for (uint64_t j = 0; j < 16 && !ok; ++j) {
            const uint64_t k = 2ULL * (16ULL * (uint64_t)i + j);
            u = gxs_below(gxs_u64(seed, k), (uint32_t)n);
            v = gxs_below(gxs_u64(seed, k + 1), (uint32_t)n);
            ok = (u != v);
        }
        if (!ok) v = (uint32_t)((u + 1ULL) % n);
        src[2 * i] = u;     dst[2 * i] = v;
        src[2 * i + 1] = v; dst[2 * i + 1] = u;
    }
}

/*
 * Clustered graph (a planted-partition model): the n vertices are cut into k
 * contiguous blocks [n c / k, n (c+1) / k), the same cut as the default
 * partitioning into k partitions. Pair i draws, for attempts j = 0..15 (five
 * values 5(16i+j) .. 5(16i+j)+4): its block c = below(v0, k), whether it
 * crosses to another block (unit(v1) < p_cross; the other block is
 * (c + 1 + below(v2, k-1)) mod k), and its ends u = lo(c) + below(v3, size(c))
 * and v = lo(c') + below(v4, size(c')); it keeps the first attempt with
 * u != v (else v = (u + 1) mod n, as for gxs_er). Each pair is stored in both
 * directions. Requires n >= 2k.
 */
void gxs_clustered(uint64_t n, uint32_t k, uint64_t m, double p_cross, uint64_t seed, uint32_t* src,
                   uint32_t* dst) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        uint32_t u = 0, v = 0;
        int ok = 0;
        for (uint64_t j = 0; j < 16 && !ok; ++j) {
            const uint64_t b = 5ULL * (16ULL * (uint64_t)i + j);
            const uint32_t c = gxs_below(gxs_u64(seed, b), k);
            const double x = (double)(gxs_u64(seed, b + 1) >> 11) * (1.0 / 9007199254740992.0);
            const uint32_t c2 = (k > 1 && x < p_cross) ? (c + 1u + gxs_below(gxs_u64(seed, b + 2), k - 1u)) % k : c;
            const uint64_t lo = n * c / k, hi = n * (c + 1) / k;
            const uint64_t lo2 = n * c2 / k, hi2 = n * (c2 + 1) / k;
            u = (uint32_t)(lo + gxs_below(gxs_u64(seed, b + 3), (uint32_t)(hi - lo)));
            v = (uint32_t)(lo2 + gxs_below(gxs_u64(seed, b + 4), (uint32_t)(hi2 - lo2)));
            ok = (u != v);
        }
        if (!ok) v = (uint32_t)((u + 1ULL) % n);
        src[2 * i] = u;     dst[2 * i] = v;
        src[2 * i + 1] = v; dst[2 * i + 1] = u;
    }
}

/* Uniform integer weights in [lo, hi]: w[i] = lo + below(value i, hi-lo+1). */
void gxs_weights(uint64_t n, uint32_t lo, uint32_t hi, uint64_t seed, uint32_t* w) {
    const uint32_t k = hi - lo + 1u;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) w[i] = lo + gxs_below(gxs_u64(seed, (uint64_t)i), k);
}

/*
 * k distinct vertices drawn uniformly without replacement from those with
 * eligible[v] != 0, by rejection: candidate j = below(value j, n), taken in
 * order of j when eligible and not yet chosen. Returns the number written
 * (k unless fewer than k candidates appear within 64*n + 1024 draws).
 * `taken` is caller scratch of n bytes, zeroed by this function.
 */
uint32_t gxs_sample(uint64_t n, const uint8_t* eligible, uint32_t k, uint64_t seed,
                    uint8_t* taken, uint32_t* out) {
    for (uint64_t v = 0; v < n; ++v) taken[v] = 0;
    uint32_t got = 0;
    const uint64_t limit = 64ULL * n + 1024ULL;
    for (uint64_t j = 0; j < limit && got < k; ++j) {
        const uint32_t v = gxs_below(gxs_u64(seed, j), (uint32_t)n);
        if (eligible[v] && !taken[v]) { taken[v] = 1; out[got++] = v; }
    }
    return got;
}

int gxs_omp_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
