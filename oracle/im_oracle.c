/*
 * im_oracle.c -- plain, slow, sequential-per-sketch CPU oracle for sketch-based
 * influence maximisation under the IC model on undirected graphs
 * (PaC-IM, "Fast and Space-Efficient Parallel Algorithms for Influence Maximization").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or constant table
 * with the GPU library; it re-states every rule from the paper on its own.
 *
 * Everything is integer arithmetic (hash, thresholds, ids, sizes, gains).
 *
 * What it computes, each with the passage it follows:
 *   - live-edge rule, Sec. 2 "fusion" sampling and Alg. 3 Sample(e, r):
 *       edge e is live in sketch r iff random(e, r) is below p_e; here random(e, r) is a
 *       64-bit splitmix64-derived word h(e, r) and the test is h < floor(p_e * 2^64), with
 *       one p for all edges or per-edge p_e (given, or the weighted cascade 2/(d_u+d_v)).
 *   - per-sketch connected components, Sec. 3 "Sketch Construction": a plain BFS per
 *     sketch over the CSR, re-hashing every arc; the label is the smallest vertex id.
 *   - component sizes (histogram) and the initial scores Delta[v] = sum_r |C_r(v)|,
 *     the memoised CC information of Sec. 2 (InfuserMG) and Alg. 2's initial scores.
 *   - centers and compact sketches <r, label[1..rho], size[1..rho]>, Sec. 3 / Alg. 3.
 *   - GetCenter / Marginal / MarkSeed exactly as Alg. 3 states them (BFS until a center).
 *   - plain non-lazy greedy (Sec. 2, the greedy of Kempe et al.), ties to the smallest id
 *     (Sec. 4: "break the tie by vertex id"), in two forms: recompute and exact decrement.
 *   - sequential CELF (Alg. 2), to count evaluations per round.
 *   - spread sum_r |union_{s in S} C_r(s)| (Alg. 1's estimate of sigma(S), times R).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_NONE 0xFFFFFFFFu

/* ------------------------------------------------------------------------
 * Hash.  Reading of the paper's random(e, r) (Sec. 2 fusion, Alg. 3 Sample):
 *   mix(x)  = splitmix64 output finaliser (Steele, Lea, Flood 2014):
 *             z = (x ^ x>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB;
 *             z ^ z>>31
 *   key(e)  = mix(mix(seed + GAMMA) ^ e)              (a per-edge splitmix64 state)
 *   h(e, r) = mix(key(e) + (r + 1) * GAMMA)           (the (r+1)-th draw of that stream)
 * with GAMMA = 0x9E3779B97F4A7C15 and all arithmetic mod 2^64.
 * ------------------------------------------------------------------------ */
static const uint64_t OR_GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t or_mix(uint64_t x) {
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return z;
}

uint64_t or_edge_key(uint64_t seed, uint64_t e) {
    return or_mix(or_mix(seed + OR_GAMMA) ^ e);
}

uint64_t or_edge_hash(uint64_t seed, uint64_t e, uint32_t r) {
    uint64_t state = or_edge_key(seed, e) + ((uint64_t)r + 1) * OR_GAMMA;
    return or_mix(state);
}

/* Threshold T = floor(p * 2^64).  p <= 0: nothing live.  p >= 1: everything live. */
void or_threshold(double p, uint64_t* T, int* all_live) {
    *all_live = 0;
    *T = 0;
    if (!(p > 0.0)) return;
    if (p >= 1.0) { *all_live = 1; return; }
    double scaled = ldexp(p, 64);          /* exact: scaling by a power of two */
    *T = (uint64_t)scaled;                 /* truncation toward zero = floor  */
}

/* ------------------------------------------------------------------------
 * Graph: an undirected edge list (u[e], v[e]) and its CSR, each arc tagged by the
 * id e of its edge (both directions share e: the sampling is direction-oblivious).
 * Optionally per-edge IC probabilities p_e (the IC model of Sec. 2 assigns one to every
 * edge), kept as thresholds floor(p_e * 2^64) and "always live" flags.
 * ------------------------------------------------------------------------ */
typedef struct {
    uint32_t n;
    uint64_t m;
    uint64_t* off;    /* n + 1 */
    uint32_t* adj;    /* 2m    */
    uint64_t* aeid;   /* 2m    */
    uint64_t* eT;     /* m, or NULL: per-edge thresholds */
    uint8_t* eall;    /* m, or NULL: p_e >= 1            */
} or_graph;

/* ------------------------------------------------------------------------
 * The sampler.  mode 0: the hash rule above with one p.  mode 1 ("worlds"): edge e is
 * live in sketch r iff bit e of r is set, so R = 2^m sketches enumerate every live-edge
 * world exactly once (used to pin the oracle against exact expectations).  mode 2: the
 * hash rule with edge e's own threshold (or_graph_set_probs / or_graph_set_wic).
 * ------------------------------------------------------------------------ */
typedef struct {
    int mode;
    uint64_t seed;
    uint64_t T;
    int all_live;
    const uint64_t* eT;
    const uint8_t* eall;
} or_sampler;

static int or_live(const or_sampler* s, uint64_t e, uint32_t r) {
    if (s->mode == 1) return (int)((r >> e) & 1u);
    if (s->mode == 2) {
        if (s->eall[e]) return 1;
        return or_edge_hash(s->seed, e, r) < s->eT[e];
    }
    if (s->all_live) return 1;
    return or_edge_hash(s->seed, e, r) < s->T;
}

static int or_make_sampler(or_sampler* s, int mode, uint64_t seed, double p, const or_graph* g) {
    s->mode = mode;
    s->seed = seed;
    or_threshold(p, &s->T, &s->all_live);
    s->eT = g ? g->eT : NULL;
    s->eall = g ? g->eall : NULL;
    if (mode == 2) return (s->eT && s->eall) ? OR_OK : OR_EINVAL;
    return (mode == 0 || mode == 1) ? OR_OK : OR_EINVAL;
}

or_graph* or_graph_new(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev) {
    for (uint64_t e = 0; e < m; ++e)
        if (eu[e] >= n || ev[e] >= n || eu[e] == ev[e]) return NULL;
    or_graph* g = (or_graph*)calloc(1, sizeof(or_graph));
    if (!g) return NULL;
    g->n = n;
    g->m = m;
    g->off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    g->adj = (uint32_t*)malloc((2 * m + 1) * sizeof(uint32_t));
    g->aeid = (uint64_t*)malloc((2 * m + 1) * sizeof(uint64_t));
    uint64_t* fill = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!g->off || !g->adj || !g->aeid || !fill) {
        free(fill); free(g->off); free(g->adj); free(g->aeid); free(g);
        return NULL;
    }
    for (uint64_t e = 0; e < m; ++e) { g->off[eu[e] + 1]++; g->off[ev[e] + 1]++; }
    for (uint32_t x = 0; x < n; ++x) g->off[x + 1] += g->off[x];
    for (uint64_t e = 0; e < m; ++e) {
        uint32_t a = eu[e], b = ev[e];
        uint64_t pa = g->off[a] + fill[a]++;
        g->adj[pa] = b; g->aeid[pa] = e;
        uint64_t pb = g->off[b] + fill[b]++;
        g->adj[pb] = a; g->aeid[pb] = e;
    }
    free(fill);
    return g;
}

void or_graph_free(or_graph* g) {
    if (!g) return;
    free(g->off); free(g->adj); free(g->aeid); free(g->eT); free(g->eall); free(g);
}

/* Per-edge probabilities p[e] (edge order of the input list). */
int or_graph_set_probs(or_graph* g, const double* p) {
    if (!g || (!p && g->m)) return OR_EINVAL;
    if (!g->eT) g->eT = (uint64_t*)malloc((g->m + 1) * sizeof(uint64_t));
    if (!g->eall) g->eall = (uint8_t*)malloc(g->m + 1);
    if (!g->eT || !g->eall) return OR_ENOMEM;
    for (uint64_t e = 0; e < g->m; ++e) {
        int all = 0;
        or_threshold(p[e], &g->eT[e], &all);
        g->eall[e] = (uint8_t)all;
    }
    return OR_OK;
}

/* The weighted cascade on an undirected graph: p_e = 2 / (d_u + d_v), the mean of the two
 * directions' 1 / d (degrees count every edge of the list, parallel edges included). */
int or_graph_set_wic(or_graph* g, double* p_out) {
    if (!g) return OR_EINVAL;
    double* p = (double*)malloc((g->m + 1) * sizeof(double));
    if (!p) return OR_ENOMEM;
    /* the endpoints of e are read back from the arcs tagged e */
    uint32_t* eu = (uint32_t*)malloc((g->m + 1) * sizeof(uint32_t));
    uint32_t* ev = (uint32_t*)malloc((g->m + 1) * sizeof(uint32_t));
    uint8_t* seen = (uint8_t*)calloc(g->m + 1, 1);
    if (!eu || !ev || !seen) { free(p); free(eu); free(ev); free(seen); return OR_ENOMEM; }
    for (uint32_t x = 0; x < g->n; ++x)
        for (uint64_t a = g->off[x]; a < g->off[x + 1]; ++a) {
            uint64_t e = g->aeid[a];
            if (!seen[e]) { eu[e] = x; ev[e] = g->adj[a]; seen[e] = 1; }
        }
    for (uint64_t e = 0; e < g->m; ++e) {
        double du = (double)(g->off[eu[e] + 1] - g->off[eu[e]]);
        double dv = (double)(g->off[ev[e] + 1] - g->off[ev[e]]);
        p[e] = 2.0 / (du + dv);
    }
    int rc = or_graph_set_probs(g, p);
    if (p_out) memcpy(p_out, p, g->m * sizeof(double));
    free(p); free(eu); free(ev); free(seen);
    return rc;
}

/* ------------------------------------------------------------------------
 * Labels of one sketch by BFS: scanning start vertices in increasing id, the start of
 * each new BFS is the smallest id of its component, and it labels the whole component.
 * L must hold n entries.  `queue` is scratch of n entries.
 * ------------------------------------------------------------------------ */
static void or_bfs_labels(const or_graph* g, const or_sampler* s, uint32_t r,
                          uint32_t* L, uint32_t* queue) {
    const uint32_t n = g->n;
    for (uint32_t x = 0; x < n; ++x) L[x] = OR_NONE;
    for (uint32_t start = 0; start < n; ++start) {
        if (L[start] != OR_NONE) continue;
        uint32_t head = 0, tail = 0;
        queue[tail++] = start;
        L[start] = start;
        while (head < tail) {
            uint32_t x = queue[head++];
            for (uint64_t a = g->off[x]; a < g->off[x + 1]; ++a) {
                uint32_t y = g->adj[a];
                if (L[y] != OR_NONE) continue;
                if (!or_live(s, g->aeid[a], r)) continue;
                L[y] = start;
                queue[tail++] = y;
            }
        }
    }
}

/* Labels of sketches r0 .. r0+count-1 into L[(r - r0) * n + v]. */
int or_labels(const or_graph* g, int mode, uint64_t seed, double p, uint32_t r0, uint32_t count,
              uint32_t* L, int nthreads) {
    or_sampler s;
    if (!g || or_make_sampler(&s, mode, seed, p, g) != OR_OK) return OR_EINVAL;
    int err = OR_OK;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        uint32_t* queue = (uint32_t*)malloc(((size_t)g->n + 1) * sizeof(uint32_t));
        if (!queue) {
#pragma omp atomic write
            err = OR_ENOMEM;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t i = 0; i < (int64_t)count; ++i)
                or_bfs_labels(g, &s, r0 + (uint32_t)i, L + (size_t)i * g->n, queue);
            free(queue);
        }
    }
    return err;
}

/* Component-size histogram of one sketch: size[x] = #{v : L[v] = x}. */
void or_histogram(uint32_t n, const uint32_t* L, uint32_t* size) {
    for (uint32_t x = 0; x < n; ++x) size[x] = 0;
    for (uint32_t v = 0; v < n; ++v) size[L[v]]++;
}

/* Initial scores from memoised components: gain[v] = sum_r |C_r(v)|. */
int or_gains(uint32_t n, uint32_t R, const uint32_t* L, uint64_t* gain) {
    uint32_t* size = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!size) return OR_ENOMEM;
    for (uint32_t v = 0; v < n; ++v) gain[v] = 0;
    for (uint32_t r = 0; r < R; ++r) {
        const uint32_t* Lr = L + (size_t)r * n;
        or_histogram(n, Lr, size);
        for (uint32_t v = 0; v < n; ++v) gain[v] += size[Lr[v]];
    }
    free(size);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Centers (Sec. 3: rho = alpha * n centers drawn uniformly at random, one global set).
 * Reading: rho = ceil(alpha * n) evaluated in IEEE double; the centers are the rho
 * vertices with the smallest ckey(v) = mix(v ^ mix(seed ^ 0xC3)) (a bijection of v, so
 * no ties); center index i orders the centers by increasing vertex id.
 * ------------------------------------------------------------------------ */
uint32_t or_num_centers(uint32_t n, double alpha) {
    if (!(alpha > 0.0) || alpha > 1.0) return 0;
    double x = ceil(alpha * (double)n);
    if (x > (double)n) x = (double)n;
    return (uint32_t)x;
}

typedef struct { uint64_t key; uint32_t v; } or_ck;

static int or_ck_cmp(const void* a, const void* b) {
    const or_ck* x = (const or_ck*)a;
    const or_ck* y = (const or_ck*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->v < y->v ? -1 : (x->v > y->v);
}

static int or_u32_cmp(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y);
}

uint64_t or_center_key(uint64_t seed, uint32_t v) {
    return or_mix((uint64_t)v ^ or_mix(seed ^ 0xC3ULL));
}

int or_centers(uint32_t n, uint64_t seed, double alpha, uint32_t* centers, uint32_t* rho_out) {
    uint32_t rho = or_num_centers(n, alpha);
    if (rho == 0 && n > 0) return OR_EINVAL;
    or_ck* all = (or_ck*)malloc(((size_t)n + 1) * sizeof(or_ck));
    if (!all) return OR_ENOMEM;
    for (uint32_t v = 0; v < n; ++v) { all[v].key = or_center_key(seed, v); all[v].v = v; }
    qsort(all, n, sizeof(or_ck), or_ck_cmp);
    for (uint32_t i = 0; i < rho; ++i) centers[i] = all[i].v;
    qsort(centers, rho, sizeof(uint32_t), or_u32_cmp);
    free(all);
    *rho_out = rho;
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Compact sketches (Sec. 3, Alg. 3 Sketch(r)):
 *   label[i] = the smallest center index j with c_j in the same component as c_i;
 *   size[i]  = |component of c_i| if label[i] = i, else 0.
 * Stored center-major: label[i * R + r], size[i * R + r].
 * ------------------------------------------------------------------------ */
int or_compact(uint32_t n, uint32_t R, const uint32_t* L, const uint32_t* centers, uint32_t rho,
               uint32_t* label, uint32_t* size) {
    uint32_t* hist = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t* first = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!hist || !first) { free(hist); free(first); return OR_ENOMEM; }
    for (uint32_t x = 0; x < n; ++x) first[x] = OR_NONE;
    for (uint32_t r = 0; r < R; ++r) {
        const uint32_t* Lr = L + (size_t)r * n;
        or_histogram(n, Lr, hist);
        for (uint32_t i = 0; i < rho; ++i) {
            uint32_t root = Lr[centers[i]];
            if (first[root] == OR_NONE) first[root] = i;
            label[(size_t)i * R + r] = first[root];
            size[(size_t)i * R + r] = (first[root] == i) ? hist[root] : 0;
        }
        for (uint32_t i = 0; i < rho; ++i) first[Lr[centers[i]]] = OR_NONE;
    }
    free(hist); free(first);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Plain greedy on memoised components.  Delta(v | S) = sum_r [C_r(v) has no seed] |C_r(v)|.
 * argmax over V \ S, ties to the smallest id; if every candidate scores 0 the smallest id
 * not in S is taken.
 *   variant 0: recompute every Delta from scratch in every round (definition, small inputs)
 *   variant 1: keep Delta exact by subtracting |C| from every member of each component
 *              that the new seed covers (same quantity, O(R n + k n) work)
 * ------------------------------------------------------------------------ */
typedef struct {
    uint32_t n, R;
    const uint32_t* L;
    uint32_t* size;       /* R * n : component sizes, indexed by root */
    uint8_t* covered;     /* R * n : component (root) already holds a seed */
} or_memo;

static int or_memo_init(or_memo* M, uint32_t n, uint32_t R, const uint32_t* L) {
    M->n = n; M->R = R; M->L = L;
    M->size = (uint32_t*)malloc((size_t)R * n * sizeof(uint32_t) + 4);
    M->covered = (uint8_t*)calloc((size_t)R * n + 1, 1);
    if (!M->size || !M->covered) { free(M->size); free(M->covered); return OR_ENOMEM; }
    for (uint32_t r = 0; r < R; ++r) or_histogram(n, L + (size_t)r * n, M->size + (size_t)r * n);
    return OR_OK;
}

static void or_memo_free(or_memo* M) { free(M->size); free(M->covered); }

static uint64_t or_memo_delta(const or_memo* M, uint32_t v) {
    uint64_t d = 0;
    for (uint32_t r = 0; r < M->R; ++r) {
        uint32_t root = M->L[(size_t)r * M->n + v];
        if (!M->covered[(size_t)r * M->n + root]) d += M->size[(size_t)r * M->n + root];
    }
    return d;
}

int or_greedy(uint32_t n, uint32_t R, const uint32_t* L, uint32_t k, int variant,
              uint32_t* seeds, uint64_t* gains) {
    if (k > n) return OR_EINVAL;
    or_memo M;
    if (or_memo_init(&M, n, R, L) != OR_OK) return OR_ENOMEM;
    uint8_t* in_s = (uint8_t*)calloc((size_t)n + 1, 1);
    uint64_t* delta = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t* moff = NULL;   /* variant 1: members of every component, per sketch */
    uint32_t* mem = NULL;
    if (!in_s || !delta) { free(in_s); free(delta); or_memo_free(&M); return OR_ENOMEM; }
    if (variant == 1) {
        moff = (uint32_t*)malloc(((size_t)n + 1) * R * sizeof(uint32_t));
        mem = (uint32_t*)malloc((size_t)n * R * sizeof(uint32_t) + 4);
        if (!moff || !mem) {
            free(moff); free(mem); free(in_s); free(delta); or_memo_free(&M);
            return OR_ENOMEM;
        }
        for (uint32_t r = 0; r < R; ++r) {
            const uint32_t* Lr = L + (size_t)r * n;
            uint32_t* o = moff + (size_t)r * (n + 1);
            uint32_t* mm = mem + (size_t)r * n;
            for (uint32_t x = 0; x <= n; ++x) o[x] = 0;
            for (uint32_t v = 0; v < n; ++v) o[Lr[v] + 1]++;
            for (uint32_t x = 0; x < n; ++x) o[x + 1] += o[x];
            for (uint32_t v = 0; v < n; ++v) mm[o[Lr[v]]++] = v;      /* o[x] now = end of x */
            for (uint32_t x = n; x > 0; --x) o[x] = o[x - 1];
            o[0] = 0;
        }
        for (uint32_t v = 0; v < n; ++v) delta[v] = or_memo_delta(&M, v);
    }
    for (uint32_t i = 0; i < k; ++i) {
        if (variant == 0)
            for (uint32_t v = 0; v < n; ++v) delta[v] = in_s[v] ? 0 : or_memo_delta(&M, v);
        int64_t best = -1;
        uint32_t s = OR_NONE;
        for (uint32_t v = 0; v < n; ++v) {
            if (in_s[v]) continue;
            if ((int64_t)delta[v] > best) { best = (int64_t)delta[v]; s = v; }
        }
        seeds[i] = s;
        if (gains) gains[i] = (uint64_t)best;
        in_s[s] = 1;
        for (uint32_t r = 0; r < R; ++r) {
            uint32_t root = L[(size_t)r * n + s];
            uint8_t* c = &M.covered[(size_t)r * n + root];
            if (*c) continue;
            *c = 1;
            if (variant == 1) {
                uint32_t sz = M.size[(size_t)r * n + root];
                const uint32_t* o = moff + (size_t)r * (n + 1);
                const uint32_t* mm = mem + (size_t)r * n;
                for (uint32_t t = o[root]; t < o[root + 1]; ++t) delta[mm[t]] -= sz;
            }
        }
    }
    free(moff); free(mem); free(in_s); free(delta); or_memo_free(&M);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Sequential CELF (Alg. 2) over memoised components: a binary max-heap of stale scores;
 * pop the top, re-evaluate, return it if its fresh score beats the new top, else push it
 * back.  Keys compare (score, then smaller id first), the same order as the greedy above.
 * evals[i] = number of evaluations in round i (the initial scores are not counted).
 * ------------------------------------------------------------------------ */
typedef struct { uint64_t g; uint32_t v; } or_hent;

static int or_hgt(or_hent a, or_hent b) { return a.g != b.g ? a.g > b.g : a.v < b.v; }

static void or_hpush(or_hent* h, uint32_t* sz, or_hent x) {
    uint32_t i = (*sz)++;
    h[i] = x;
    while (i > 0) {
        uint32_t p = (i - 1) / 2;
        if (!or_hgt(h[i], h[p])) break;
        or_hent t = h[i]; h[i] = h[p]; h[p] = t; i = p;
    }
}

static or_hent or_hpop(or_hent* h, uint32_t* sz) {
    or_hent top = h[0];
    h[0] = h[--(*sz)];
    uint32_t i = 0;
    for (;;) {
        uint32_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < *sz && or_hgt(h[l], h[b])) b = l;
        if (r < *sz && or_hgt(h[r], h[b])) b = r;
        if (b == i) break;
        or_hent t = h[i]; h[i] = h[b]; h[b] = t; i = b;
    }
    return top;
}

int or_celf(uint32_t n, uint32_t R, const uint32_t* L, uint32_t k, uint32_t* seeds,
            uint64_t* gains, uint64_t* evals) {
    if (k > n) return OR_EINVAL;
    or_memo M;
    if (or_memo_init(&M, n, R, L) != OR_OK) return OR_ENOMEM;
    or_hent* h = (or_hent*)malloc(((size_t)n + 1) * sizeof(or_hent));
    if (!h) { or_memo_free(&M); return OR_ENOMEM; }
    uint32_t hs = 0;
    for (uint32_t v = 0; v < n; ++v) { or_hent x = { or_memo_delta(&M, v), v }; or_hpush(h, &hs, x); }
    for (uint32_t i = 0; i < k; ++i) {
        uint64_t ev = 0;
        or_hent s;
        for (;;) {
            s = or_hpop(h, &hs);
            if (i > 0) { s.g = or_memo_delta(&M, s.v); ++ev; }
            if (hs == 0 || or_hgt(s, h[0])) break;
            or_hpush(h, &hs, s);
        }
        seeds[i] = s.v;
        if (gains) gains[i] = s.g;
        if (evals) evals[i] = ev;
        for (uint32_t r = 0; r < R; ++r)
            M.covered[(size_t)r * n + L[(size_t)r * n + s.v]] = 1;
    }
    free(h); or_memo_free(&M);
    return OR_OK;
}

/* Spread: sum_r |union_{s in S} C_r(s)| (duplicates in `seeds` count once). */
int or_spread(uint32_t n, uint32_t R, const uint32_t* L, const uint32_t* seeds, uint32_t k,
              uint64_t* out) {
    uint32_t* size = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint8_t* mark = (uint8_t*)calloc((size_t)n + 1, 1);
    if (!size || !mark) { free(size); free(mark); return OR_ENOMEM; }
    for (uint32_t i = 0; i < k; ++i) if (seeds[i] >= n) { free(size); free(mark); return OR_EINVAL; }
    uint64_t total = 0;
    for (uint32_t r = 0; r < R; ++r) {
        const uint32_t* Lr = L + (size_t)r * n;
        or_histogram(n, Lr, size);
        for (uint32_t i = 0; i < k; ++i) {
            uint32_t root = Lr[seeds[i]];
            if (!mark[root]) { mark[root] = 1; total += size[root]; }
        }
        for (uint32_t i = 0; i < k; ++i) mark[Lr[seeds[i]]] = 0;
    }
    free(size); free(mark);
    *out = total;
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * The paper's compact-sketch procedures, as Alg. 3 states them.
 *   GetCenter(Phi_r, v, S): BFS from v on G'_r.  If a center c_i is met, l = label[i] and
 *     the result is <size[l], l>.  Otherwise <0, -1> if a seed was visited, else
 *     <#visited, -1>.
 *   Marginal(S, v) = sum_r delta_r   (kept as an integer sum; the paper divides by R).
 *   MarkSeed(s): for every sketch, if GetCenter gives l != -1, size[l] <- 0.
 * cidx[x] = center index of x, or OR_NONE.  `size` is modified by MarkSeed.
 * ------------------------------------------------------------------------ */
typedef struct {
    const or_graph* g;
    or_sampler s;
    uint32_t R;
    const uint32_t* cidx;
    const uint32_t* label;   /* rho * R */
    uint32_t* size;          /* rho * R */
    const uint8_t* in_s;
    uint32_t* queue;         /* n */
    uint32_t* stamp;         /* n, visit marks */
    uint32_t epoch;
} or_compact_ctx;

static uint64_t or_get_center(or_compact_ctx* C, uint32_t v, uint32_t r, int64_t* l_out) {
    const or_graph* g = C->g;
    if (++C->epoch == 0) {                      /* stamp wrap-around: clear marks */
        memset(C->stamp, 0, (size_t)g->n * sizeof(uint32_t));
        C->epoch = 1;
    }
    uint32_t head = 0, tail = 0;
    int seen_seed = 0;
    C->queue[tail++] = v;
    C->stamp[v] = C->epoch;
    while (head < tail) {
        uint32_t x = C->queue[head++];
        if (C->cidx[x] != OR_NONE) {
            uint32_t l = C->label[(size_t)C->cidx[x] * C->R + r];
            *l_out = l;
            return C->size[(size_t)l * C->R + r];
        }
        if (C->in_s[x]) seen_seed = 1;
        for (uint64_t a = g->off[x]; a < g->off[x + 1]; ++a) {
            uint32_t y = g->adj[a];
            if (C->stamp[y] == C->epoch) continue;
            if (!or_live(&C->s, g->aeid[a], r)) continue;
            C->stamp[y] = C->epoch;
            C->queue[tail++] = y;
        }
    }
    *l_out = -1;
    return seen_seed ? 0 : tail;
}

/*
 * Plain greedy on compact sketches: every round evaluates Marginal for all v not in S
 * (ties to the smallest id), then MarkSeed.  `size` (rho * R) is copied, not modified.
 */
int or_compact_greedy(const or_graph* g, int mode, uint64_t seed, double p, uint32_t R,
                      const uint32_t* centers, uint32_t rho, const uint32_t* label,
                      const uint32_t* size, uint32_t k, uint32_t* seeds, uint64_t* gains) {
    if (!g || k > g->n) return OR_EINVAL;
    const uint32_t n = g->n;
    or_compact_ctx C;
    memset(&C, 0, sizeof C);
    if (or_make_sampler(&C.s, mode, seed, p, g) != OR_OK) return OR_EINVAL;
    C.g = g; C.R = R; C.label = label;
    uint32_t* cidx = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint8_t* in_s = (uint8_t*)calloc((size_t)n + 1, 1);
    C.size = (uint32_t*)malloc((size_t)rho * R * sizeof(uint32_t) + 4);
    C.queue = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    C.stamp = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
    int err = OR_OK;
    if (!cidx || !in_s || !C.size || !C.queue || !C.stamp) { err = OR_ENOMEM; goto done; }
    for (uint32_t x = 0; x < n; ++x) cidx[x] = OR_NONE;
    for (uint32_t i = 0; i < rho; ++i) cidx[centers[i]] = i;
    memcpy(C.size, size, (size_t)rho * R * sizeof(uint32_t));
    C.cidx = cidx; C.in_s = in_s;
    for (uint32_t i = 0; i < k; ++i) {
        int64_t best = -1;
        uint32_t s = OR_NONE;
        for (uint32_t v = 0; v < n; ++v) {
            if (in_s[v]) continue;
            uint64_t d = 0;
            int64_t l;
            for (uint32_t r = 0; r < R; ++r) d += or_get_center(&C, v, r, &l);
            if ((int64_t)d > best) { best = (int64_t)d; s = v; }
        }
        seeds[i] = s;
        if (gains) gains[i] = (uint64_t)best;
        for (uint32_t r = 0; r < R; ++r) {          /* MarkSeed(s) with S before adding s */
            int64_t l;
            or_get_center(&C, s, r, &l);
            if (l != -1) C.size[(size_t)l * R + r] = 0;
        }
        in_s[s] = 1;
    }
done:
    free(cidx); free(in_s); free(C.size); free(C.queue); free(C.stamp);
    return err;
}

/* Marginal(S, v) on compact sketches for an explicit S given as a flag array, with `size`
 * already reflecting MarkSeed of S (so callers can test single evaluations). */
int or_compact_marginal(const or_graph* g, int mode, uint64_t seed, double p, uint32_t R,
                        const uint32_t* cidx, const uint32_t* label, const uint32_t* size,
                        const uint8_t* in_s, uint32_t v, uint64_t* out) {
    if (!g || v >= g->n) return OR_EINVAL;
    or_compact_ctx C;
    memset(&C, 0, sizeof C);
    if (or_make_sampler(&C.s, mode, seed, p, g) != OR_OK) return OR_EINVAL;
    C.g = g; C.R = R; C.label = label; C.size = (uint32_t*)size; C.cidx = cidx; C.in_s = in_s;
    C.queue = (uint32_t*)malloc(((size_t)g->n + 1) * sizeof(uint32_t));
    C.stamp = (uint32_t*)calloc((size_t)g->n + 1, sizeof(uint32_t));
    if (!C.queue || !C.stamp) { free(C.queue); free(C.stamp); return OR_ENOMEM; }
    uint64_t d = 0;
    for (uint32_t r = 0; r < R; ++r) { int64_t l; d += or_get_center(&C, v, r, &l); }
    free(C.queue); free(C.stamp);
    *out = d;
    return OR_OK;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
