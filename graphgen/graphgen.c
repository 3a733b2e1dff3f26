/*
 * graphgen.c -- seeded synthetic undirected graphs for the influence-maximisation
 * workloads (Erdos-Renyi, Chung-Lu power law, R-MAT).
 *
 * This module only synthesises inputs.  It holds none of the method's arithmetic
 * (no edge sampling, no connectivity, no gains): both the CPU oracle and the GPU
 * library consume its output, a canonical edge list.
 *
 * Output contract (all generators):
 *   - m distinct undirected edges, no self-loops, stored as u[e] < v[e];
 *   - sorted by (u, v) ascending, so the edge id e is the rank of (u, v);
 *   - the edge set is "the first m distinct pairs in draw order": draw j is a pure
 *     function of (seed, j) (a splitmix64 counter stream), self-loops are dropped,
 *     and a pair repeated later in the stream is a duplicate.
 *
 * Random numbers: the splitmix64 generator of Steele, Lea and Flood (OOPSLA 2014),
 * state_j = seed + (j+1)*0x9E3779B97F4A7C15, output = its 64-bit finaliser.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* j-th output of the splitmix64 stream started at `seed`. */
static inline uint64_t gg_rand(uint64_t seed, uint64_t j) {
    return gg_mix(seed + (j + 1) * GG_GAMMA);
}

/* uniform integer in [0, bound) from a 64-bit random word (multiply-high). */
static inline uint64_t gg_below(uint64_t r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

static int gg_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Stable LSD radix sort of (key, idx) pairs on the low `bits` bits of key.
 * --------------------------------------------------------------------------- */
#define RADIX_BITS 11
#define RADIX_SIZE (1u << RADIX_BITS)

static int radix_sort_pairs(uint64_t* key, uint32_t* idx, uint64_t cnt, int bits) {
    uint64_t* k2 = (uint64_t*)malloc(cnt * sizeof(uint64_t) + 8);
    uint32_t* i2 = (uint32_t*)malloc(cnt * sizeof(uint32_t) + 4);
    if (!k2 || !i2) { free(k2); free(i2); return -1; }
    int nt = gg_threads();
    uint64_t* hist = (uint64_t*)calloc((size_t)nt * RADIX_SIZE, sizeof(uint64_t));
    if (!hist) { free(k2); free(i2); return -1; }
    uint64_t *ks = key, *kd = k2;
    uint32_t *is = idx, *id = i2;
    int passes = (bits + RADIX_BITS - 1) / RADIX_BITS;
    for (int pass = 0; pass < passes; ++pass) {
        int shift = pass * RADIX_BITS;
        memset(hist, 0, (size_t)nt * RADIX_SIZE * sizeof(uint64_t));
#pragma omp parallel num_threads(nt)
        {
#ifdef _OPENMP
            int t = omp_get_thread_num();
#else
            int t = 0;
#endif
            uint64_t lo = cnt * (uint64_t)t / nt, hi = cnt * (uint64_t)(t + 1) / nt;
            uint64_t* h = hist + (size_t)t * RADIX_SIZE;
            for (uint64_t i = lo; i < hi; ++i) h[(ks[i] >> shift) & (RADIX_SIZE - 1)]++;
#pragma omp barrier
#pragma omp single
            {
                uint64_t run = 0;
                for (uint32_t b = 0; b < RADIX_SIZE; ++b)
                    for (int tt = 0; tt < nt; ++tt) {
                        uint64_t c = hist[(size_t)tt * RADIX_SIZE + b];
                        hist[(size_t)tt * RADIX_SIZE + b] = run;
                        run += c;
                    }
            }
            for (uint64_t i = lo; i < hi; ++i) {
                uint64_t pos = h[(ks[i] >> shift) & (RADIX_SIZE - 1)]++;
                kd[pos] = ks[i];
                id[pos] = is[i];
            }
        }
        uint64_t* tk = ks; ks = kd; kd = tk;
        uint32_t* ti = is; is = id; id = ti;
    }
    if (ks != key) {
        memcpy(key, ks, cnt * sizeof(uint64_t));
        memcpy(idx, is, cnt * sizeof(uint32_t));
    }
    free(hist); free(k2); free(i2);
    return 0;
}

static int bitlen(uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }

/* A draw function writes the canonical key of draw j (or `invalid`). */
typedef uint64_t (*gg_draw_fn)(const void* prm, uint64_t j);

/*
 * Keep the first m distinct valid keys in draw order, emit them sorted.
 * Returns m on success, -1 on allocation failure, -2 if the graph cannot hold m
 * distinct edges within the draw budget.
 */
static int64_t first_m_distinct(const void* prm, gg_draw_fn draw, uint64_t m, int s,
                                double oversample, uint32_t* u_out, uint32_t* v_out) {
    const uint64_t invalid = (s >= 32) ? UINT64_MAX : ((1ULL << (2 * s)) - 1);
    const int bits = 2 * s;
    if (m == 0) return 0;
    uint64_t D = (uint64_t)((double)m * oversample) + 64;
    for (int attempt = 0; attempt < 8; ++attempt) {
        if (D > 0xFFFFFFF0ULL) D = 0xFFFFFFF0ULL;
        uint64_t* key = (uint64_t*)malloc(D * sizeof(uint64_t));
        uint32_t* idx = (uint32_t*)malloc(D * sizeof(uint32_t));
        uint64_t* first = (uint64_t*)calloc((D + 63) / 64, sizeof(uint64_t));
        if (!key || !idx || !first) { free(key); free(idx); free(first); return -1; }
#pragma omp parallel for schedule(static)
        for (uint64_t j = 0; j < D; ++j) { key[j] = draw(prm, j); idx[j] = (uint32_t)j; }
        if (radix_sort_pairs(key, idx, D, bits) != 0) { free(key); free(idx); free(first); return -1; }
        /* mark the first occurrence (smallest draw index) of every valid key */
        uint64_t distinct = 0;
        for (uint64_t i = 0; i < D; ++i) {
            if (key[i] == invalid) continue;
            if (i == 0 || key[i] != key[i - 1]) {
                first[idx[i] >> 6] |= 1ULL << (idx[i] & 63);
                ++distinct;
            }
        }
        if (distinct >= m) {
            /* cutoff = 1 + draw index of the m-th first occurrence */
            uint64_t seen = 0, cutoff = D;
            for (uint64_t w = 0; w < (D + 63) / 64; ++w) {
                uint64_t word = first[w];
                int pc = __builtin_popcountll(word);
                if (seen + (uint64_t)pc < m) { seen += pc; continue; }
                for (int b = 0; b < 64; ++b)
                    if (word >> b & 1ULL) {
                        if (++seen == m) { cutoff = w * 64 + b + 1; break; }
                    }
                break;
            }
            uint64_t out = 0;
            for (uint64_t i = 0; i < D; ++i) {
                if (key[i] == invalid) continue;
                if (i == 0 || key[i] != key[i - 1]) {
                    if (idx[i] < cutoff) {
                        u_out[out] = (uint32_t)(key[i] >> s);
                        v_out[out] = (uint32_t)(key[i] & ((1ULL << s) - 1));
                        ++out;
                    }
                }
            }
            free(key); free(idx); free(first);
            return (out == m) ? (int64_t)m : -3;
        }
        free(key); free(idx); free(first);
        if (D == 0xFFFFFFF0ULL) break;
        D = D + D / 2 + (m - distinct) * 4;
    }
    return -2;
}

/* ------------------------------- Erdos-Renyi ------------------------------ */
typedef struct { uint64_t seed; uint32_t n; int s; uint64_t invalid; } er_prm;

static uint64_t er_draw(const void* p, uint64_t j) {
    const er_prm* q = (const er_prm*)p;
    uint64_t a = gg_below(gg_rand(q->seed, 2 * j), q->n);
    uint64_t b = gg_below(gg_rand(q->seed, 2 * j + 1), q->n);
    if (a == b) return q->invalid;
    if (a > b) { uint64_t t = a; a = b; b = t; }
    return (a << q->s) | b;
}

int64_t gg_erdos_renyi(uint32_t n, uint64_t m, uint64_t seed, uint32_t* u, uint32_t* v) {
    if (n < 2 && m > 0) return -2;
    if ((double)m > 0.5 * (double)n * (double)(n - 1)) return -2;
    er_prm q; q.seed = seed; q.n = n; q.s = bitlen(n - 1); if (q.s == 0) q.s = 1;
    q.invalid = (1ULL << (2 * q.s)) - 1;
    double full = 0.5 * (double)n * (double)(n - 1);
    double over = 1.1 + 4.0 * (double)m / full;
    return first_m_distinct(&q, er_draw, m, q.s, over, u, v);
}

/* -------------------------------- Chung-Lu -------------------------------- */
typedef struct { uint64_t seed; uint32_t n; int s; uint64_t invalid; const uint64_t* cum; uint64_t total; } cl_prm;

static inline uint32_t cl_pick(const cl_prm* q, uint64_t r) {
    uint64_t x = gg_below(r, q->total);       /* x in [0, total) */
    uint32_t lo = 0, hi = q->n - 1;           /* first i with cum[i] > x */
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (q->cum[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static uint64_t cl_draw(const void* p, uint64_t j) {
    const cl_prm* q = (const cl_prm*)p;
    uint64_t a = cl_pick(q, gg_rand(q->seed, 2 * j));
    uint64_t b = cl_pick(q, gg_rand(q->seed, 2 * j + 1));
    if (a == b) return q->invalid;
    if (a > b) { uint64_t t = a; a = b; b = t; }
    return (a << q->s) | b;
}

/*
 * Expected-degree power law: w_i = c (i+1)^(-1/(exponent-1)), c chosen so that
 * sum w = 2m, each w_i capped at max_deg; endpoints are drawn proportional to w
 * (weights quantised to integers with 2^10 resolution, at least 1).
 */
int64_t gg_chung_lu(uint32_t n, uint64_t m, double exponent, double max_deg, uint64_t seed,
                    uint32_t* u, uint32_t* v) {
    if (n < 2 && m > 0) return -2;
    if (!(exponent > 1.0)) return -4;
    double beta = 1.0 / (exponent - 1.0);
    double* w = (double*)malloc((size_t)n * sizeof(double));
    uint64_t* cum = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    if (!w || !cum) { free(w); free(cum); return -1; }
    double sum = 0.0;
    for (uint32_t i = 0; i < n; ++i) { w[i] = pow((double)i + 1.0, -beta); sum += w[i]; }
    double c = 2.0 * (double)m / sum;
    uint64_t run = 0;
    for (uint32_t i = 0; i < n; ++i) {
        double wi = c * w[i];
        if (max_deg > 0 && wi > max_deg) wi = max_deg;
        uint64_t qi = (uint64_t)(wi * 1024.0);
        if (qi == 0) qi = 1;
        run += qi;
        cum[i] = run;
    }
    free(w);
    cl_prm q; q.seed = seed; q.n = n; q.s = bitlen(n - 1); if (q.s == 0) q.s = 1;
    q.invalid = (1ULL << (2 * q.s)) - 1; q.cum = cum; q.total = run;
    int64_t r = first_m_distinct(&q, cl_draw, m, q.s, 1.35, u, v);
    free(cum);
    return r;
}

/* --------------------------------- R-MAT ---------------------------------- */
typedef struct { uint64_t seed; int scale; uint64_t invalid; uint32_t ta, tab, tabc; } rm_prm;

static uint64_t rm_draw(const void* p, uint64_t j) {
    const rm_prm* q = (const rm_prm*)p;
    const uint64_t words = (uint64_t)(q->scale + 1) / 2;  /* two levels per 64-bit word */
    uint64_t a = 0, b = 0;
    for (int lvl = 0; lvl < q->scale; ++lvl) {
        uint64_t rw = gg_rand(q->seed, j * words + (uint64_t)(lvl >> 1));
        uint32_t x = (lvl & 1) ? (uint32_t)(rw >> 32) : (uint32_t)rw;
        uint64_t bu, bv;
        if (x < q->ta)        { bu = 0; bv = 0; }
        else if (x < q->tab)  { bu = 0; bv = 1; }
        else if (x < q->tabc) { bu = 1; bv = 0; }
        else                  { bu = 1; bv = 1; }
        a = (a << 1) | bu;
        b = (b << 1) | bv;
    }
    if (a == b) return q->invalid;
    if (a > b) { uint64_t t = a; a = b; b = t; }
    return (a << q->scale) | b;
}

/* R-MAT without noise; quadrant probabilities a, b, c, d = 1-a-b-c (thresholds on 32-bit words). */
int64_t gg_rmat(uint32_t scale, uint64_t m, double a, double b, double c, uint64_t seed,
                uint32_t* u, uint32_t* v) {
    if (scale < 1 || scale > 31) return -4;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -4;
    rm_prm q; q.seed = seed; q.scale = (int)scale;
    q.invalid = (1ULL << (2 * scale)) - 1;
    double two32 = 4294967296.0;
    double ta = floor(a * two32), tab = floor((a + b) * two32), tabc = floor((a + b + c) * two32);
    q.ta = (uint32_t)(ta > 4294967295.0 ? 4294967295.0 : ta);
    q.tab = (uint32_t)(tab > 4294967295.0 ? 4294967295.0 : tab);
    q.tabc = (uint32_t)(tabc > 4294967295.0 ? 4294967295.0 : tabc);
    return first_m_distinct(&q, rm_draw, m, (int)scale, 1.6, u, v);
}

int gg_num_threads(void) { return gg_threads(); }
