/*
 * im_gb300.h -- C ABI of the GB300 (sm_103a) sketch engine for influence maximisation
 * under the independent cascade (IC) model on undirected graphs, after
 * "Fast and Space-Efficient Parallel Algorithms for Influence Maximization" (PaC-IM).
 *
 * The calls follow the paper's problem statement (Sec. 2: given G = (V, E), k and IC
 * probabilities, find |S| = k maximising the expected spread sigma(S)) and its
 * sketch-based framework (Alg. 1: Step 1 builds R sketches, Step 2 selects k seeds).
 *
 * Conventions shared by every call
 *   - Return value: IM_OK (0) or a negative IM_E* code; no exception crosses the ABI.
 *     im_last_error() then describes the failure.
 *   - Every call is synchronous with respect to the host: when it returns, its device
 *     work on the context's stream has finished and outputs are written.
 *   - Output buffers are owned by the caller.  ptr_kind says whether a pointer is a host
 *     pointer (IM_PTR_HOST) or a device pointer on the context's device (IM_PTR_DEVICE).
 *   - Gains and spreads are integer sums over the R sketches (sigma(S) * R); the paper
 *     divides by R (Alg. 3, Marginal), which callers may do for display.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - Vertex ids are uint32 with n < 2^31; edge ids are uint32 positions in the input
 *     edge list (m < 2^32).
 */
#ifndef IM_GB300_H
#define IM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IM_OK        0
#define IM_EINVAL   (-1)   /* bad argument (sizes, ids, p, alpha, k, R, pointer kind) */
#define IM_ENOMEM   (-2)   /* device allocation failed                                */
#define IM_ECUDA    (-3)   /* a CUDA runtime call failed                              */
#define IM_ESTATE   (-4)   /* call out of order (e.g. selection before sketches)      */
#define IM_ETIMEOUT (-5)   /* a bounded device wait gave up                           */
#define IM_EDEVICE  (-6)   /* a kernel reported an internal error through its status */

#define IM_PTR_HOST   0
#define IM_PTR_DEVICE 1

typedef struct im_ctx im_ctx;

/*
 * im_create -- load the input graph G = (V, E) (Sec. 2) onto the device and build its CSR.
 *   n        number of vertices (1 <= n < 2^31).
 *   m        number of undirected edges (m < 2^32); m = 0 is allowed.
 *   u, v     m endpoints each: edge e = {u[e], v[e]}, e is its id for sampling
 *            (Alg. 3 Sample(e, r)); u[e] != v[e], both < n.  The list is copied; the
 *            caller keeps ownership.  Canonical inputs have u[e] < v[e] sorted by (u, v).
 *   ptr_kind IM_PTR_HOST or IM_PTR_DEVICE for u and v.
 *   stream   a cudaStream_t to run on (NULL: the context creates its own stream).
 *   out      receives the context; NULL on failure.
 * Errors: IM_EINVAL (n, ids, self-loops), IM_ENOMEM, IM_ECUDA.
 */
int im_create(im_ctx** out, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v,
              int ptr_kind, void* stream);

/*
 * im_load_graph -- replace the context's graph by another edge list (same conventions as
 * im_create; page-locked host lists that the device can address are read in place by the
 * packing kernel, other host lists are copied through a staging buffer the context keeps;
 * either way the call returns after the lists were read).  Device
 * buffers are reused while n and m are unchanged, and the sketch buffers and selection graph
 * of the next im_build_sketches too when its shapes are; a long-lived context thus serves one
 * graph after another without allocating.  The sketches and any selection are discarded:
 * im_build_sketches must run next.  On failure no graph is loaded (IM_ESTATE until a
 * successful load).
 * Errors: IM_EINVAL (n, m, ids, self-loops), IM_ENOMEM, IM_ECUDA.
 */
int im_load_graph(im_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v,
                  int ptr_kind);

/*
 * im_set_edge_probs -- the IC probability of every edge (Sec. 2: the IC model gives each edge
 * its own p_e; the paper's other workloads are uniform random and weighted-cascade ones).
 *   model  IM_PROBS_UNIFORM: one p for every edge, the p argument of im_build_sketches
 *                            (the default; p is ignored otherwise);
 *          IM_PROBS_ARRAY:   p[e] for edge e of the loaded list (m doubles, host or device
 *                            per ptr_kind; values >= 1 always live, <= 0 or NaN never);
 *          IM_PROBS_WIC:     weighted cascade p_e = 2 / (d_u + d_v), degrees counting every
 *                            edge of the list at both ends (p is ignored).
 * Edge e is live in sketch r iff h(e, r) < floor(p_e * 2^64) (h as in im_build_sketches).
 * Costs 24 m bytes of device memory.  Discards the sketches and any selection;
 * im_load_graph returns to IM_PROBS_UNIFORM.
 * Errors: IM_EINVAL, IM_ESTATE (no graph), IM_ENOMEM, IM_ECUDA.
 */
#define IM_PROBS_UNIFORM 0
#define IM_PROBS_ARRAY 1
#define IM_PROBS_WIC 2
int im_set_edge_probs(im_ctx* ctx, int model, const double* p, int ptr_kind);

/*
 * im_build_sketches -- Step 1 of Alg. 1: build R compact sketches (Sec. 3, Alg. 3).
 *   R      number of sketches (1 <= R <= 65536).  Sketch r in [0, R) is the sampled graph
 *          G'_r whose live edges are those with h(e, r) < floor(p * 2^64), where
 *          h(e, r) = mix(mix(mix(seed + G) ^ e) + (r + 1) G), G = 0x9E3779B97F4A7C15 and
 *          mix is the splitmix64 finaliser ("fusion" sampling, Sec. 2).  No sampled graph
 *          is stored.
 *   seed   hash seed; also seeds the choice of centers.
 *   p      uniform IC probability; p <= 0 makes no edge live, p >= 1 every edge.
 *   alpha  center fraction in (0, 1] (the paper's rate; rho = ceil(alpha * n) centers,
 *          the rho vertices with the smallest mix(v ^ mix(seed ^ 0xC3)), indexed by
 *          increasing vertex id).  alpha = 1 stores every vertex's component (full labels).
 * Produces, on the device: initial gains Delta[v] = sum_r |C_r(v)|, and per sketch the
 * compact arrays label[i] (smallest center index in the component of center i) and
 * size[i] (component size where label[i] = i, else 0).  Resets any seed selection.
 * Errors: IM_EINVAL (R, alpha, or R * n too large for the 64-bit packed keys),
 *         IM_ENOMEM, IM_ECUDA, IM_EDEVICE.
 */
int im_build_sketches(im_ctx* ctx, uint32_t R, uint64_t seed, double p, double alpha);

/*
 * im_select_seeds -- Step 2 of Alg. 1: greedy seeds by lazy evaluation on the device
 * (CELF, Alg. 2, with prefix-doubling batches of re-evaluations as in Alg. 4).
 *   k          total number of seeds wanted (1 <= k <= n).  Selection is prefix-consistent:
 *              a later call with a larger k continues from the seeds already chosen; a
 *              smaller k returns the prefix.
 *   seeds_out  host array of k vertex ids, in selection order.
 *   gains_out  host array of k marginal gains Delta(s_i | S_{i-1}) (sum over sketches),
 *              or NULL.
 * Ties between equal gains go to the smaller vertex id (Sec. 4); a vertex already in S is
 * never chosen again.  The result equals plain (non-lazy) greedy exactly.
 * Errors: IM_ESTATE (no sketches), IM_EINVAL (k), IM_ECUDA, IM_EDEVICE.
 */
int im_select_seeds(im_ctx* ctx, uint32_t k, uint32_t* seeds_out, uint64_t* gains_out);

/*
 * im_spread -- sum_r |union_{s in S} C_r(s)| for an arbitrary seed list (the sketch estimate
 * of sigma(S), Alg. 1, times R).  Duplicated seeds count once.
 *   seeds      host array of k vertex ids (each < n); 0 <= k <= 16384.
 *   spread_out host pointer to the result.
 * Independent of, and not changing, the selection state.
 * Errors: IM_ESTATE, IM_EINVAL, IM_ECUDA, IM_EDEVICE.
 */
int im_spread(im_ctx* ctx, const uint32_t* seeds, uint32_t k, uint64_t* spread_out);

/* im_reset_selection -- forget the chosen seeds; the sketches are kept. */
int im_reset_selection(im_ctx* ctx);

/*
 * im_get_labels -- connected-component labels of sketch r (Sec. 3 Sketch(r)): out[v] = the
 * smallest vertex id in the component of v in G'_r.  Recomputed on demand (n entries).
 * Errors: IM_ESTATE, IM_EINVAL (r >= R, ptr_kind), IM_ECUDA.
 */
int im_get_labels(im_ctx* ctx, uint32_t r, uint32_t* out, int ptr_kind);

/* im_get_gains -- initial gains Delta[v] = sum_r |C_r(v)| (n entries, uint64). */
int im_get_gains(im_ctx* ctx, uint64_t* out, int ptr_kind);

/* im_get_centers -- center vertex ids by center index (rho entries); *rho_out = rho. */
int im_get_centers(im_ctx* ctx, uint32_t* out, uint32_t* rho_out, int ptr_kind);

/*
 * im_get_compact -- the compact sketches of Alg. 3, center-major: label[i * R + r] and
 * size[i * R + r] for center index i < rho and sketch r < R.  size is the component size
 * as built (seed coverage from im_select_seeds is reported separately and not applied).
 */
int im_get_compact(im_ctx* ctx, uint32_t* label, uint32_t* size, int ptr_kind);

typedef struct {
    uint32_t n, R, rho, rounds;     /* rounds = seeds selected so far                    */
    uint64_t m;
    uint64_t evaluations;           /* re-evaluations (Marginal calls) during selection  */
    uint64_t batches;               /* prefix-doubling batches                           */
    uint64_t bfs_fallbacks;         /* (v, r) searches that spilled to the global queue  */
    uint64_t launches;              /* kernels launched by this context                  */
    uint32_t sketch_batch;          /* sketches processed per edge pass                  */
    uint64_t hop1_arcs;             /* arcs scanned by first-hop searches (32 sketches each) */
    uint64_t hop2_searches;         /* (vertex, sketch) searches that went past the 1st hop */
    uint64_t hop2_chunks;           /* 32-arc chunks scanned by those searches             */
    uint64_t refresh_batches;       /* batches evaluated by recomputing the sketches        */
    uint64_t live_pairs;            /* live (edge, sketch) pairs unioned since im_create    */
    uint64_t build_live_pairs;      /* of those, unioned by the last im_build_sketches      */
    uint64_t spec_batches;          /* batches evaluated from a candidate first seed's
                                       overlaps (see im_set_seed_speculation)             */
    uint64_t hubs;                  /* hubs of the last build (see im_set_hubs)            */
    uint32_t union_path;            /* union path of the last build (IM_UNION_AUTO resolved) */
} im_stats;

int im_get_stats(im_ctx* ctx, im_stats* out);

/* Per-round evaluation counts (Sec. 4, F_i): out[i] for i < min(count, rounds). */
int im_get_round_evals(im_ctx* ctx, uint64_t* out, uint32_t count);

/*
 * Profiling: when enabled, every kernel launch is bracketed by CUDA events on the context
 * stream and its device time accumulated per kernel kind.
 */
int im_profile_enable(im_ctx* ctx, int on);
int im_profile_reset(im_ctx* ctx);
int im_profile_get(im_ctx* ctx, int kernel_id, double* total_ms, uint64_t* launches);
int im_kernel_count(void);
const char* im_kernel_name(int kernel_id);

/* Tuning: sketches per edge pass (power of two, 1..32; 0 = automatic).  Takes effect at the
 * next im_build_sketches. */
int im_set_sketch_batch(im_ctx* ctx, uint32_t batch);

/* Failure injection for tests (no counterpart in the paper): after `after` more device
 * allocations of the library (any context, any thread) have succeeded, the next one fails as
 * if the device were out of memory -- nothing is allocated, the call that needed it returns
 * IM_ENOMEM and leaves its context usable (a later call allocates again) -- and the hook
 * disarms itself.  A negative `after` disarms it.  No GPU work is involved: the failure is
 * made on the host, before cudaMalloc would be called.  Returns IM_OK. */
int im_debug_fail_alloc(int64_t after);

/* Test hook (no counterpart in the paper): the sketch kernels of every later build use at most
 * `records` live-pair records per lane and batch (a negative value restores the allocated
 * capacity), so that a test can make the record buffer overflow: the union kernel then redoes
 * the batch with the fused sampling+union loop, with the same results.  Returns IM_OK. */
int im_debug_record_cap(int64_t records);

/*
 * im_sketch_static -- labels and component sizes of one sketch, for callers that cannot
 * allocate device memory.  The paper has no counterpart of this call.
 *
 * Who needs it: code that runs inside a host process which owns all device memory itself,
 * e.g. a serving or database process whose pool allocator hands out every buffer and caps
 * its footprint, or a latency-critical loop.  There a cudaMalloc would bypass the pool's
 * accounting, may fail under its cap, and (with cudaFree) synchronises the whole device.
 * Everything else in this ABI allocates through its context; this call allocates nothing:
 * no cudaMalloc, no cudaFree, no allocating library routine.
 *
 *   n         vertices, 1 <= n <= IM_STATIC_MAX_N.
 *   m, d_u, d_v  m undirected edges as two DEVICE arrays of vertex ids (edge id = index),
 *             u != v, both < n; not modified.
 *   seed, p, r   sketch r under the same live-edge rule as im_build_sketches.
 *   d_labels  DEVICE output, n entries: smallest vertex id of the component of v (or NULL).
 *   d_sizes   DEVICE output, n entries: |C_r(v)| (or NULL; not both NULL).
 *   stream    cudaStream_t to run on (NULL: the legacy default stream).  The call returns
 *             when its work on that stream has finished.
 *
 * Scratch: a file-scope static device array of 2 * IM_STATIC_MAX_N + 64 uint32 words
 * (8 MiB + 256 B), present on every device where the library is loaded, until the process
 * exits.  Its device address is looked up (cudaGetSymbolAddress, which allocates nothing) in
 * the calling thread's current context by every call made outside stream capture, so any
 * context works: the primary one, one created after a cudaDeviceReset, or a non-primary
 * context made current.  A call made while `stream` is being captured uses the address the
 * last uncaptured call found on that device: make one call on the device, in the context
 * that the capture uses, before capturing (without one the call fails with IM_ECUDA).  All calls
 * share the array; each call clears what it needs, but calls whose GPU work overlaps (two
 * streams, two threads) race on it and give wrong results: serialise them.
 * Errors: IM_EINVAL (n out of range, m >= 2^32, NULL arrays, an edge id >= n or a self-loop
 * found while sampling -- outputs are then undefined), IM_ECUDA.  im_last_error(NULL)
 * describes the failure.
 */
#define IM_STATIC_MAX_N (1u << 20)
int im_sketch_static(uint32_t n, uint64_t m, const uint32_t* d_u, const uint32_t* d_v,
                     uint64_t seed, double p, uint32_t r, uint32_t* d_labels, uint32_t* d_sizes,
                     void* stream);

/* Tuning: re-evaluation batches of at least `min_batch` candidates are evaluated by
 * recomputing every sketch's components (Sketch(r), Alg. 3) and looking each candidate up,
 * instead of one GetCenter search per (candidate, sketch); the values are identical.
 * 0 = automatic (max(16384, n / 4)); UINT64_MAX disables it.  Takes effect at the next
 * im_build_sketches. */
int im_set_refresh_threshold(im_ctx* ctx, uint64_t min_batch);

/* Tuning: 2 (default) runs consecutive sketch batches on two streams so that one batch's
 * hashing (ALU-bound) overlaps another's union-find (latency-bound); 1 runs them in order on
 * the context stream.  Both lanes' scratch is allocated either way; results do not depend on it. */
int im_set_pipeline(im_ctx* ctx, uint32_t lanes);

/* Tuning: how a sketch batch's unions meet its sampling (Sec. 3: the live edges of Sample(e, r)
 * are united per sketch; Alg. 3).  IM_UNION_RECORDS: the live pairs are written to a record
 * buffer of the context (about 1.3 p m B x 16 bytes per lane) and united by a second kernel
 * that keeps several unions of each thread in flight.  IM_UNION_FUSED: one kernel hashes the
 * batch's (edge, sketch) pairs and unites the live ones through a per-warp queue in shared
 * memory, so that no live pair is stored (no record buffer).  IM_UNION_BUCKETS: the records
 * (8 bytes, in the same buffer) are grouped by sketch and by sampling block as they are written,
 * and the union kernel takes the sketches one after the other, so that the parents it climbs
 * belong to one or two sketches at a time (on large graphs these then stay in L2).
 * IM_UNION_AUTO (default): IM_UNION_BUCKETS when a batch's parent arrays (4 n B bytes) exceed
 * 256 MiB, else IM_UNION_RECORDS.  Results do not depend on it.  Takes effect at the next
 * im_build_sketches; IM_EINVAL for another value. */
#define IM_UNION_FUSED 0
#define IM_UNION_RECORDS 1
#define IM_UNION_BUCKETS 2
#define IM_UNION_AUTO 3
int im_set_union_path(im_ctx* ctx, int path);

/* Execution of the selection loop (Alg. 2 / Alg. 4 rounds).  1 (default): the whole loop is
 * one CUDA graph whose while / switch nodes are set by the device, so rounds and batches run
 * without the host; 0: the host launches every batch after reading the device's decision.
 * Both run the same kernels and give identical results. */
int im_set_graph(im_ctx* ctx, int on);

/* Tuning: while building, also sum for `candidates` likely first seeds c -- the vertices with
 * the largest gains over the first batch of sketches, ties to the smaller id --
 * ov_c(v) = sum_r |C_r(v)| [c in C_r(v)].  If the first seed is one of them, the second round's
 * batches are evaluated as Marginal(v | {c}) = gain0(v) - ov_c(v) (exact) instead of by
 * searches or by recomputing the sketches.  0 disables; default 4, at most 8; costs 8 n bytes
 * per candidate (twice with two lanes); takes effect at the next im_build_sketches.
 * Seeds, gains and evaluation counts do not depend on it. */
int im_set_seed_speculation(im_ctx* ctx, uint32_t candidates);

/*
 * im_mc_spread -- Monte-Carlo influence of a seed set: the paper's quality measure (Sec. 5
 * averages the number of vertices an IC cascade from S activates over independent
 * simulations).  An IC cascade activates exactly the vertices reachable from S over the live
 * edges of an independently sampled live-edge graph (Sec. 2), so simulation r is the
 * live-edge world that a sketch with index r would sample under the edge hash seed `mc_seed`
 * and the context's probabilities (the p of the last im_build_sketches, or the per-edge model
 * set then).  Different mc_seed values give independent simulations; the sketches' own seed
 * gives back their worlds.
 *   seeds     HOST array of k vertex ids (< n; duplicates allowed), k <= 16384; not modified.
 *   sims      number of simulations (0 gives 0).
 *   out       HOST: sum over the simulations of |vertices reachable from S|, an exact integer;
 *             the estimate of sigma(S) is *out / sims.
 * Reuses the build's per-batch scratch (the sketches themselves are untouched).  Blocks until
 * done.  Errors: IM_ESTATE (no build yet), IM_EINVAL (NULL arrays, k too large, an id >= n),
 * IM_ENOMEM, IM_ECUDA.
 */
int im_mc_spread(im_ctx* ctx, const uint32_t* seeds, uint32_t k, uint32_t sims, uint64_t mc_seed, uint64_t* out);

/*
 * im_run_batch -- many independent instances on the current device: for each, the whole of
 * Alg. 1 (im_create / im_load_graph, im_build_sketches, im_select_seeds, im_spread), with
 * results identical to running the instances one by one.  `workers` host threads each own a
 * context with its own stream and take the next instance (largest m R + n R first), so the
 * instances' kernels overlap on the GPU; a context keeps its buffers across the instances it
 * runs while they fit (no cudaMalloc / cudaFree, which would synchronise the device).
 *   inst[i].n, m, u, v      the graph: HOST edge lists of m entries (as im_create); not modified
 *   inst[i].R, seed, p, alpha, k   as im_build_sketches and im_select_seeds (the probability
 *                            model is one p per instance)
 *   inst[i].seeds_out, gains_out   HOST, k entries each; spread_out: HOST, 1 entry
 *   inst[i].status           out: IM_OK or the error of that instance's first failing call
 * Returns IM_OK if every instance succeeded, else the first failing instance's status (in
 * input order); IM_EINVAL if inst is NULL, workers is 0 or an output pointer is NULL.
 * Blocks until every instance is done.
 */
typedef struct {
    uint32_t n;
    uint64_t m;
    const uint32_t* u;
    const uint32_t* v;
    uint32_t R;
    uint32_t k;
    uint64_t seed;
    double p;
    double alpha;
    uint32_t* seeds_out;
    uint64_t* gains_out;
    uint64_t* spread_out;
    int status;
} im_instance;

int im_run_batch(im_instance* inst, uint32_t count, uint32_t workers);

/*
 * The batch as one CUDA graph (Alg. 1 for every instance, the instances' paths side by side).
 * im_batch_create plans a batch once: one context per instance with every buffer reserved, and
 * one CUDA graph holding each instance's whole path -- the upload of its edge lists, its CSR,
 * its sketch construction, its lazy-greedy loop (conditional nodes set by the device, as in
 * im_select_seeds), its spread and the copies of its results.  The instances form `branches`
 * chains, largest first and dealt round-robin, that the graph runs concurrently.
 * im_batch_run launches the graph once, waits, and writes every instance's seeds_out,
 * gains_out, spread_out and status -- identical to im_run_batch and to one-by-one runs.  It may
 * be called again: each call uploads the instances' edge lists anew from the same host
 * arrays (which stay valid and unchanged in size until im_batch_destroy; lists that are not
 * pinned are staged through pinned memory when the graph is captured, so later calls see their
 * contents of that time; pinned lists are read at every run).
 *   inst     as im_run_batch (the array itself must outlive the batch)
 *   sched    NULL for the defaults, or the schedule im_batch_tune chose: per size class
 *            (an instance's m R at most class_pairs[j], the last class unbounded) the sketch
 *            batch, lanes and union path of its context, and the number of branches.
 * Errors: IM_EINVAL (NULL pointers, an instance's n or R 0, k outside [1, min(n, 16384)],
 * alpha outside (0, 1], more than 4 classes), IM_ENOMEM, IM_ECUDA; im_batch_run returns the
 * first failing instance's status (IM_EINVAL for an edge id >= n or a self-loop, found on the
 * device; IM_EDEVICE if its selection stopped).  One batch is not thread-safe.
 *
 * im_batch_tune times the knobs on the batch itself: instances are grouped into size classes by
 * m R; on each class's largest instance im_autotune tries sketch batch, lanes (and hubs for
 * alpha < 1), and the three union paths (im_set_union_path) are compared; then whole batches with 4, 8 and 16
 * branches are built and run, and the fastest is kept.  *out receives the schedule.
 */
typedef struct {
    uint32_t branches;          /* chains run side by side (0: 8) */
    uint32_t classes;           /* size classes in use, 0..4 (0: default knobs everywhere) */
    uint64_t class_pairs[4];    /* upper bound of m R of classes 0 .. classes-2 */
    uint32_t sketch_batch[4];   /* im_set_sketch_batch of each class (0: automatic) */
    uint32_t lanes[4];          /* im_set_pipeline of each class (0: 2) */
    uint32_t union_path[4];     /* im_set_union_path of each class */
    double run_ms;              /* im_batch_tune: time of one im_batch_run with this schedule */
} im_batch_schedule;
typedef struct im_batch im_batch;
int im_batch_create(im_instance* inst, uint32_t count, const im_batch_schedule* sched, im_batch** out);
int im_batch_run(im_batch* batch);
int im_batch_destroy(im_batch* batch);
int im_batch_tune(im_instance* inst, uint32_t count, im_batch_schedule* out);

/*
 * Serving: sketch sets held in HBM under a memory budget, answering requests for seed sets
 * (the paper has no serving layer; this engine is built on its greedy-prefix property: Alg. 1
 * picks one seed per round, so the best k seeds it finds are the first k of one sequence,
 * whatever other k were asked).
 *
 * im_server_create     an empty engine on the current device; its budget is the device's free
 *                      memory at this call minus 2 GiB.
 * im_server_set_budget the device bytes resident models may hold together (IM_ESTATE if the
 *                      models resident now already hold more).
 * im_server_add_model  registers one model -- a graph (HOST edge lists, copied) with R, seed, p,
 *                      alpha (as im_build_sketches).  *footprint_out = its estimated device
 *                      bytes (im_footprint_estimate).  IM_ENOMEM, with nothing allocated, if
 *                      that exceeds the whole budget; IM_EINVAL for an invalid edge list.  The
 *                      sketches are built now if they fit beside the resident models, else at
 *                      the model's first request.  *model_out = its id (0, 1, ...).
 * im_server_replay     submits every request at its arrival time (arrival_ns after the call
 *                      starts) and returns when all are answered.  A model's thread takes all
 *                      of its pending requests at once; if the model's sequence known so far
 *                      answers them they need no GPU; otherwise the model is admitted -- when
 *                      its footprint does not fit under the budget, idle resident models are
 *                      evicted (least recently used first; their sequences stay on the host)
 *                      and, if none is idle, the request waits until one is -- and its
 *                      device-resident loop (im_serve_launch) extends the sequence to the
 *                      largest k.  The answer to (model, k) is the first k seeds, their
 *                      marginal gains and the spread estimate sum_{i<k} gain_i (= im_spread of
 *                      those seeds, by telescoping), whatever else was in flight and however
 *                      often the model was evicted and rebuilt.  submit_ns / done_ns: when the
 *                      request was queued and answered, from the call's start.  Returns IM_OK,
 *                      or the first failing request's status (IM_EINVAL for a model id or k out
 *                      of range).
 * im_server_stats      one model's footprint, builds, evictions, residency and seeds known, and
 *                      the engine's budget and bytes in use.
 * im_server_destroy    stops the threads and frees every model.
 * The control calls (create, set_budget, add_model, replay, stats, destroy) are made from one
 * thread, one at a time; the engine's own threads only touch their model.
 */
typedef struct im_server im_server;
typedef struct {
    uint32_t model;
    uint32_t k;
    uint64_t arrival_ns;
    uint32_t* seeds_out;    /* HOST, k entries (or NULL) */
    uint64_t* gains_out;    /* HOST, k entries (or NULL) */
    uint64_t* spread_out;   /* HOST, 1 entry (or NULL) */
    uint64_t submit_ns;     /* out */
    uint64_t done_ns;       /* out */
    int status;             /* out */
} im_request;

typedef struct {
    uint64_t footprint;     /* estimated device bytes while resident */
    uint32_t builds;        /* sketch builds so far (1 + rebuilds after evictions) */
    uint32_t evictions;
    uint32_t resident;      /* 1 if its sketches are in HBM now */
    uint32_t known_seeds;   /* length of its sequence known on the host */
    uint64_t budget;        /* the engine's budget and bytes held by resident models */
    uint64_t used;
} im_model_stats;

int im_server_create(im_server** out);
int im_server_set_budget(im_server* srv, uint64_t bytes);
int im_server_add_model(im_server* srv, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v, uint32_t R,
                        uint64_t seed, double p, double alpha, uint32_t* model_out, uint64_t* footprint_out);
int im_server_replay(im_server* srv, im_request* req, uint32_t count);
int im_server_stats(im_server* srv, uint32_t model, im_model_stats* out);
int im_server_destroy(im_server* srv);

/* Estimated device bytes of one context holding a graph of n vertices and m edges with R
 * sketches at probability p and center fraction alpha (graph, per-vertex arrays, two lanes of
 * union-find scratch and live-pair records, compact and hub rows); an upper bound on what
 * im_create + im_build_sketches allocate.  IM_EINVAL for n = 0, R = 0 or alpha outside (0, 1]. */
int im_footprint_estimate(uint32_t n, uint64_t m, uint32_t R, double p, double alpha, uint64_t* bytes_out);

/* Tuning: hubs.  GetCenter (Alg. 3) from a vertex whose component reaches a high-degree
 * non-center tests that vertex's whole adjacency list, in every sketch where it is reached.
 * With hubs, up to `cap` non-centers of degree >= `min_degree` (the largest degrees, ties to
 * the smaller id) also get a label and a size per sketch, kept after the compact sketch's
 * rho rows, so that a search stops at them as at a center.  Seeds, gains, spread and the
 * compact sketch (im_get_compact) do not depend on it.  cap = IM_HUBS_AUTO (default):
 * max(1024, n / 64); 0 disables; at most n - rho are used.  min_degree 0 is taken as 1
 * (default 32).  Costs 8 R bytes per hub; takes effect at the next im_build_sketches. */
#define IM_HUBS_AUTO 0xFFFFFFFFu
int im_set_hubs(im_ctx* ctx, uint32_t cap, uint32_t min_degree);

/*
 * Device-resident request loop (serving).  Alg. 1 picks one seed per round, so the answer to
 * "k seeds" is the first k seeds of one greedy sequence; a loop on the device answers requests
 * for k from a mailbox and extends the sequence only as far as the largest k asked.
 *
 * The mailbox lives in mapped pinned host memory (allocated by im_mailbox_create, owned by
 * the caller until im_mailbox_destroy): a ring of `ring` requested k values and room for the
 * first `kcap` seeds and gains.  im_serve_launch starts, on the context's stream, one CUDA
 * graph that repeats: wait for requests (the device polls the mailbox), run the lazy-greedy
 * rounds (Alg. 2 / Alg. 4, the same kernels as im_select_seeds) up to the largest pending k,
 * publish the new seeds and gains into the mailbox.  Requests pushed while it runs are taken
 * by its next wait -- no new launch, no host round trip.  Every wait of the device is bounded:
 * when no request arrives for idle_us microseconds (at most 10^7; also after 2^24 polls) the
 * loop ends with status IM_ETIMEOUT and clears its `running` flag; a request pushed after that
 * needs a new im_serve_launch.
 *
 * While a loop serves a context (from im_serve_launch to im_serve_finish) the context's other
 * calls that use the sequence or the sketches return IM_ESTATE.  One context is not thread-safe:
 * push, wait, launch and finish are made from one thread (or under the caller's lock).
 *
 *   im_mailbox_create   ring in [1, 65536], kcap in [1, n].  IM_ENOMEM without host memory.
 *   im_mailbox_push     queue a request for k in [1, kcap] seeds; IM_ESTATE when `ring`
 *                       requests are still untaken.
 *   im_serve_launch     start a loop (idle_us as above); a context that was rebuilt since the
 *                       last loop publishes its new sequence from the start.
 *   im_mailbox_wait     wait on the host until the first k seeds are published, then copy them
 *                       (and their marginal gains) to seeds / gains (caller-owned, k entries,
 *                       either may be NULL).  IM_ETIMEOUT after timeout_us; IM_ESTATE when no
 *                       loop is running and fewer than k seeds are published; IM_EDEVICE when
 *                       the loop's selection stopped on an error.
 *   im_mailbox_state    running flag, status of the last loop, seeds published.
 *   im_serve_finish     ask the loop to end at its next wait, wait for it, and bring the
 *                       context's own copy of the sequence up to date (im_select_seeds then
 *                       continues it).  *loop_status: IM_OK (ended by this call),
 *                       IM_ETIMEOUT (it had idled out), IM_EDEVICE.
 *   im_mailbox_destroy  IM_ESTATE while a loop still serves the mailbox.
 * The paper has no serving layer; the rounds are those of Alg. 2 / Alg. 4.
 */
typedef struct im_mailbox im_mailbox;
int im_mailbox_create(im_ctx* ctx, uint32_t ring, uint32_t kcap, im_mailbox** out);
int im_mailbox_push(im_mailbox* mb, uint32_t k);
int im_serve_launch(im_mailbox* mb, uint32_t idle_us);
int im_mailbox_wait(im_mailbox* mb, uint32_t k, uint32_t timeout_us, uint32_t* seeds, uint64_t* gains);
int im_mailbox_state(const im_mailbox* mb, uint32_t* running, int32_t* status, uint32_t* answered);
int im_serve_finish(im_mailbox* mb, int32_t* loop_status);
int im_mailbox_destroy(im_mailbox* mb);

/*
 * Autotuning of the knobs that leave every result unchanged: sketches per edge pass
 * (im_set_sketch_batch: automatic, 16, 8), sketch batches in flight (im_set_pipeline: 2, 1)
 * and, for compact sketches (alpha < 1), hubs (im_set_hubs: IM_HUBS_AUTO, none; the
 * context's minimum degree is kept).  Every combination builds the sketches of (R, seed, p,
 * alpha) and selects k seeds (Alg. 1) `reps` + 1 times, the first untimed (it may capture the
 * selection graph); its time is the smallest of the timed runs, on the host clock, whose
 * calls are synchronous.  The fastest combination is set on the context and
 * the sketches are built once more with it, so that the context is ready for
 * im_select_seeds.  Every combination must give the same seeds: if one does not, the call
 * fails with IM_EDEVICE.
 *
 * out (caller-owned) receives the chosen knobs, their times and those of the first
 * combination (the defaults).  Errors: IM_EINVAL for a NULL ctx or out, reps == 0 or
 * k outside [1, n], and any error of im_build_sketches or im_select_seeds, which stops the
 * search; the knobs are then left as the failing combination set them.
 */
typedef struct {
    uint32_t sketch_batch;   /* chosen im_set_sketch_batch value (0 = automatic)      */
    uint32_t lanes;          /* chosen im_set_pipeline value                          */
    uint32_t hub_cap;        /* chosen im_set_hubs cap (IM_HUBS_AUTO or 0)             */
    uint32_t tried;          /* combinations timed                                    */
    double build_ms;         /* im_build_sketches with the chosen knobs (ms)          */
    double select_ms;        /* im_select_seeds(k) with the chosen knobs (ms)         */
    double default_build_ms; /* the same for the first combination (the defaults)     */
    double default_select_ms;
} im_tuning;
int im_autotune(im_ctx* ctx, uint32_t R, uint64_t seed, double p, double alpha, uint32_t k, uint32_t reps,
                im_tuning* out);

/* Measurement: the rate of the sampling kernel's per-pair compute (64-bit add, high word of
 * the hash, compare, live-mask update) on register values only -- the ceiling of the
 * sampling with no memory traffic -- in (edge, sketch) pairs per second on the current
 * device; `iters` (a positive multiple of 32) sketches per key, 2 keys per thread, 1216 blocks
 * of 256 threads.  Blocks until done.  Errors: IM_EINVAL, IM_ECUDA. */
int im_hash_peak(uint32_t iters, double* pairs_per_s);

/* The context's stream (a cudaStream_t). */
void* im_stream(im_ctx* ctx);

const char* im_last_error(const im_ctx* ctx);
void im_destroy(im_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* IM_GB300_H */
