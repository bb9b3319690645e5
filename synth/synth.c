/*
 * Seeded synthetic inputs for the dynamic-graph store and its algorithms.
 *
 * This module only draws inputs: edge lists, weights, permutations and
 * request streams.  It holds none of the store's or the algorithms'
 * arithmetic, and both the CUDA path and the CPU oracle receive the arrays
 * it produces.  Every random number is counter-based SplitMix64 (Steele, Lea
 * and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
 * value i of stream `seed` is mix(seed + (i + 1) * golden_gamma), so any
 * element can be drawn independently and the output does not depend on how
 * the work is split.
 *
 * Graph shapes follow the paper's workloads (Section "Experimental
 * evaluation", Table 5): R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004)
 * for the power-law social and web graphs, a 2D grid with a few long-range
 * edges for the road network, and uniform random pairs for the random graph.
 *
 * Plain C99, no platform intrinsics: it builds and gives the same output on
 * x86_64 and aarch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Value i of the SplitMix64 stream that starts from state `seed`. */
static inline uint64_t at(uint64_t seed, uint64_t i)
{
    return sm_mix(seed + (i + 1) * GOLDEN_GAMMA);
}

uint64_t syn_splitmix_at(uint64_t seed, uint64_t i)
{
    return at(seed, i);
}

/* A seed for a named sub-stream, so that streams with different tags never
 * overlap in practice. */
uint64_t syn_substream(uint64_t seed, uint64_t tag)
{
    return sm_mix(seed ^ sm_mix(tag + GOLDEN_GAMMA));
}

/* Uniform integer in [0, n) from the high 32 bits of r (n <= 2^32). */
static inline uint32_t bounded32(uint64_t r, uint64_t n)
{
    return (uint32_t)(((r >> 32) * n) >> 32);
}

/* Uniform double in [0, 1) from the high 53 bits of r. */
static inline double unit53(uint64_t r)
{
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* n uniform (src, dst) pairs over [0, V). */
void syn_uniform_pairs(uint32_t V, uint64_t n, uint64_t seed, uint32_t *src, uint32_t *dst)
{
    for (uint64_t i = 0; i < n; ++i) {
        src[i] = bounded32(at(seed, 2 * i), V);
        dst[i] = bounded32(at(seed, 2 * i + 1), V);
    }
}

/* n uniform weights in [wmin, wmax]. */
void syn_weights(uint64_t n, uint64_t seed, uint32_t wmin, uint32_t wmax, uint32_t *w)
{
    uint64_t span = (uint64_t)wmax - (uint64_t)wmin + 1;
    for (uint64_t i = 0; i < n; ++i)
        w[i] = wmin + bounded32(at(seed, i), span);
}

/* n R-MAT pairs on 2^scale vertices with quadrant probabilities a, b, c and
 * d = 1 - a - b - c, no noise.  Level l picks bit (scale - 1 - l) of both
 * endpoints from one draw. */
void syn_rmat_pairs(uint32_t scale, uint64_t n, double a, double b, double c, uint64_t seed,
                    uint32_t *src, uint32_t *dst)
{
    double ab = a + b, abc = a + b + c;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t s = 0, d = 0;
        for (uint32_t l = 0; l < scale; ++l) {
            double u = unit53(at(seed, i * scale + l));
            uint32_t bit = 1u << (scale - 1 - l);
            /* quadrants in order a (0,0), b (0,1), c (1,0), d (1,1) */
            uint32_t row = (uint32_t)(u >= ab);
            uint32_t col = (uint32_t)((u >= a) & (u < ab)) | (uint32_t)(u >= abc);
            s |= bit & (0u - row);
            d |= bit & (0u - col);
        }
        src[i] = s;
        dst[i] = d;
    }
}

/* Preferential (degree-skewed) R-MAT variant used for growth streams: with
 * probability `skew` the source is replaced by the source of an earlier
 * pair of the stream chosen uniformly (so sources repeat in proportion to
 * how often they appeared before); otherwise the R-MAT draw is kept.
 * `prev_src`/`n_prev` is the history to copy from. */
void syn_skew_sources(uint64_t n, double skew, uint64_t seed, const uint32_t *prev_src,
                      uint64_t n_prev, uint32_t *src)
{
    if (n_prev == 0)
        return;
    for (uint64_t i = 0; i < n; ++i) {
        double u = unit53(at(seed, 2 * i));
        if (u < skew) {
            uint64_t r = at(seed, 2 * i + 1);
            uint64_t j = (uint64_t)(unit53(r) * (double)n_prev);
            if (j >= n_prev)
                j = n_prev - 1;
            src[i] = prev_src[j];
        }
    }
}

/* Uniform random permutation of [0, n) (Fisher-Yates, Knuth Vol. 2 3.4.2). */
void syn_permutation(uint64_t n, uint64_t seed, uint32_t *perm)
{
    for (uint64_t i = 0; i < n; ++i)
        perm[i] = (uint32_t)i;
    for (uint64_t i = n; i > 1; --i) {
        uint64_t r = at(seed, i);
        uint64_t j = (uint64_t)(unit53(r) * (double)i);
        if (j >= i)
            j = i - 1;
        uint32_t t = perm[i - 1];
        perm[i - 1] = perm[j];
        perm[j] = t;
    }
}

/* Directed 4-neighbour grid on rows x cols vertices (vertex r * cols + c),
 * both directions of every grid link.  Writes 2 * (rows*(cols-1) +
 * cols*(rows-1)) pairs in row-major order of the source and returns that
 * count. */
uint64_t syn_grid_pairs(uint32_t rows, uint32_t cols, uint32_t *src, uint32_t *dst)
{
    uint64_t k = 0;
    for (uint32_t r = 0; r < rows; ++r) {
        for (uint32_t c = 0; c < cols; ++c) {
            uint32_t v = r * cols + c;
            if (c + 1 < cols) { src[k] = v; dst[k] = v + 1; ++k; }
            if (c > 0) { src[k] = v; dst[k] = v - 1; ++k; }
            if (r + 1 < rows) { src[k] = v; dst[k] = v + cols; ++k; }
            if (r > 0) { src[k] = v; dst[k] = v - cols; ++k; }
        }
    }
    return k;
}

/* Stable LSD radix sort of (key, index) by key over the low `keybits`
 * bits, 11 bits per pass. */
static int radix_sort_kv(uint64_t *key, uint32_t *idx, uint64_t n, uint32_t keybits)
{
    uint64_t *k2 = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint32_t *i2 = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint64_t *cnt = (uint64_t *)malloc(2048 * sizeof(uint64_t));
    if (!k2 || !i2 || !cnt) {
        free(k2); free(i2); free(cnt);
        return -1;
    }
    uint64_t *ka = key, *kb = k2;
    uint32_t *ia = idx, *ib = i2;
    uint32_t passes = (keybits + 10) / 11;
    for (uint32_t p = 0; p < passes; ++p) {
        uint32_t sh = 11 * p;
        memset(cnt, 0, 2048 * sizeof(uint64_t));
        for (uint64_t i = 0; i < n; ++i)
            cnt[(ka[i] >> sh) & 0x7FF]++;
        uint64_t sum = 0;
        for (uint32_t d = 0; d < 2048; ++d) {
            uint64_t t = cnt[d];
            cnt[d] = sum;
            sum += t;
        }
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t o = cnt[(ka[i] >> sh) & 0x7FF]++;
            kb[o] = ka[i];
            ib[o] = ia[i];
        }
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *ti = ia; ia = ib; ib = ti;
    }
    if (ka != key) {
        memcpy(key, ka, n * sizeof(uint64_t));
        memcpy(idx, ia, n * sizeof(uint32_t));
    }
    free(k2); free(i2); free(cnt);
    return 0;
}

/* Workload recipe step "duplicates and self-loops dropped": keeps the first
 * occurrence of every (src, dst) pair, optionally drops src == dst, and
 * compacts in place preserving the order of the kept pairs.  `vbits` is the
 * number of bits of a vertex id.  Returns the kept count, or UINT64_MAX if
 * memory ran out. */
uint64_t syn_dedup_pairs(uint32_t *src, uint32_t *dst, uint64_t n, uint32_t vbits, int drop_self)
{
    if (n == 0)
        return 0;
    uint64_t *key = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint32_t *idx = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint8_t *keep = (uint8_t *)calloc(n, 1);
    if (!key || !idx || !keep) {
        free(key); free(idx); free(keep);
        return UINT64_MAX;
    }
    for (uint64_t i = 0; i < n; ++i) {
        key[i] = ((uint64_t)src[i] << vbits) | dst[i];
        idx[i] = (uint32_t)i;
    }
    if (radix_sort_kv(key, idx, n, 2 * vbits) != 0) {
        free(key); free(idx); free(keep);
        return UINT64_MAX;
    }
    for (uint64_t i = 0; i < n; ++i)
        if (i == 0 || key[i] != key[i - 1])
            keep[idx[i]] = 1;
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (!keep[i] || (drop_self && src[i] == dst[i]))
            continue;
        src[m] = src[i];
        dst[m] = dst[i];
        ++m;
    }
    free(key); free(idx); free(keep);
    return m;
}

/* Exponential inter-arrival gaps (Poisson process of rate `rate` per second)
 * in seconds, by inversion of the exponential CDF. */
void syn_exponential_gaps(uint64_t n, double rate, uint64_t seed, double *gap)
{
    for (uint64_t i = 0; i < n; ++i) {
        double u = unit53(at(seed, i));
        double one_minus = 1.0 - u; /* in (0, 1] */
        gap[i] = -log(one_minus) / rate;
    }
}

/* Log-uniform integers in [lo, hi]: exp of a uniform draw over
 * [ln lo, ln(hi + 1)), floored. */
void syn_log_uniform(uint64_t n, uint64_t lo, uint64_t hi, uint64_t seed, uint64_t *out)
{
    double a = log((double)lo), b = log((double)hi + 1.0);
    for (uint64_t i = 0; i < n; ++i) {
        double u = unit53(at(seed, i));
        uint64_t v = (uint64_t)exp(a + u * (b - a));
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        out[i] = v;
    }
}

/* ------------------------------------------------------------------ */
/* Live-edge set of a batch stream.  A recipe that must draw deletes and
 * "present" queries from the edges that are live when a batch runs keeps
 * the set of live (src, dst) pairs here: open addressing with linear
 * probing over 64-bit keys src << 32 | dst and deletion by backward shift
 * (Knuth Vol. 3, 6.4, Algorithm R), so no tombstones accumulate.  It only
 * decides which pairs a generator draws; nothing reads it to compute an
 * expected result. */
typedef struct {
    uint64_t *key;
    uint64_t mask;
    uint64_t count;
} syn_set;

#define SET_EMPTY UINT64_MAX

static inline uint64_t set_home(const syn_set *s, uint64_t k)
{
    return sm_mix(k) & s->mask;
}

/* A set with room for `capacity` keys (the table holds at least twice that
 * many slots).  Returns NULL if memory ran out. */
void *syn_set_create(uint64_t capacity)
{
    syn_set *s = (syn_set *)malloc(sizeof(syn_set));
    if (!s)
        return NULL;
    uint64_t slots = 1024;
    while (slots < 2 * capacity)
        slots <<= 1;
    s->key = (uint64_t *)malloc(slots * sizeof(uint64_t));
    if (!s->key) {
        free(s);
        return NULL;
    }
    memset(s->key, 0xFF, slots * sizeof(uint64_t));
    s->mask = slots - 1;
    s->count = 0;
    return s;
}

void syn_set_destroy(void *h)
{
    syn_set *s = (syn_set *)h;
    if (s) {
        free(s->key);
        free(s);
    }
}

uint64_t syn_set_count(void *h)
{
    return ((syn_set *)h)->count;
}

/* Adds the pairs in order; added[i] (nullable) = 1 iff pair i was absent
 * (so of repeated pairs only the first is 1).  Returns the number added, or
 * UINT64_MAX if the table would pass half full (nothing after that pair is
 * added). */
uint64_t syn_set_add(void *h, const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *added)
{
    syn_set *s = (syn_set *)h;
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t k = ((uint64_t)src[i] << 32) | dst[i];
        uint64_t at_ = set_home(s, k);
        while (s->key[at_] != SET_EMPTY && s->key[at_] != k)
            at_ = (at_ + 1) & s->mask;
        int fresh = s->key[at_] == SET_EMPTY;
        if (fresh) {
            if (2 * (s->count + 1) > s->mask + 1)
                return UINT64_MAX;
            s->key[at_] = k;
            s->count++;
            m++;
        }
        if (added)
            added[i] = (uint8_t)fresh;
    }
    return m;
}

/* Removes the pairs in order; removed[i] (nullable) = 1 iff pair i was
 * present.  Returns the number removed. */
uint64_t syn_set_remove(void *h, const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *removed)
{
    syn_set *s = (syn_set *)h;
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t k = ((uint64_t)src[i] << 32) | dst[i];
        uint64_t at_ = set_home(s, k);
        while (s->key[at_] != SET_EMPTY && s->key[at_] != k)
            at_ = (at_ + 1) & s->mask;
        int hit = s->key[at_] == k;
        if (hit) {
            /* backward shift: move later keys of the run into the hole
             * unless their home lies cyclically in (hole, their slot] */
            uint64_t hole = at_, j = at_;
            for (;;) {
                j = (j + 1) & s->mask;
                if (s->key[j] == SET_EMPTY)
                    break;
                uint64_t home = set_home(s, s->key[j]);
                int stays = (hole <= j) ? (hole < home && home <= j) : (hole < home || home <= j);
                if (!stays) {
                    s->key[hole] = s->key[j];
                    hole = j;
                }
            }
            s->key[hole] = SET_EMPTY;
            s->count--;
            m++;
        }
        if (removed)
            removed[i] = (uint8_t)hit;
    }
    return m;
}

/* present[i] = 1 iff pair i is in the set. */
void syn_set_contains(void *h, const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *present)
{
    syn_set *s = (syn_set *)h;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t k = ((uint64_t)src[i] << 32) | dst[i];
        uint64_t at_ = set_home(s, k);
        while (s->key[at_] != SET_EMPTY && s->key[at_] != k)
            at_ = (at_ + 1) & s->mask;
        present[i] = (uint8_t)(s->key[at_] == k);
    }
}
