// im_internal.cuh -- device helpers and host-side plumbing shared by the CUDA sources.
// Internal to the library; the public contract is include/im_gb300.h.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/im_gb300.h"

namespace imk {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;   // splitmix64 increment
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kCovered = 0x80000000u;            // size word: component holds a seed
// parent entry of a root after the counting pass: the root has members (vertex ids are < 2^31),
// so its root word holds the component's size and key; an unflagged root is a singleton
constexpr uint32_t kRootFlag = 0x80000000u;
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr uint32_t kNoCenterTag = 0x80000000u;        // spread: component id without a center
constexpr uint32_t kQcap = 256;                       // per-warp BFS queue (shared memory)
constexpr uint32_t kSpreadKMax = 16384;
constexpr uint32_t kArcIdMask = 0x7FFFFFFFu;            // arc word 0: neighbour id | center bit
constexpr uint32_t kLabSlots = 256;                     // label cache: vertex slots (x mod 256)
constexpr size_t kCenterSelBytes = 4096;                // device state of the center radix select
constexpr uint32_t kHubsAuto = 0xFFFFFFFFu;                // im_ctx::hub_cap default
constexpr uint32_t kMaxLanes = 2;                          // sketch batches in flight at most (a third lane measured no faster)
constexpr uint32_t kSpecMax = 8;                        // candidate first seeds (see im_ctx::spec_req)
// per lane: record count and ticket (two words), or, for bucketed records, the overflow flag and
// its ticket, then one count per (sketch, sampling block) region: 8 + 32 x 152 x 4 words
constexpr uint32_t kLiveCounters = (8 + 32u * 152u * 4u) / 2 + 1;   // in 64-bit words

// splitmix64 output finaliser (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Live-edge rule of the "fusion" sampling (Sec. 2, Alg. 3 Sample): edge e is live in
// sketch r iff mix(key_e + (r+1) G) < T_e, key_e = mix(salt ^ e), salt = mix(seed + G),
// T_e = floor(p_e 2^64) -- one p for every edge (T, all_live for p >= 1), or per edge
// (Sec. 2's IC model gives each edge its own p_e): eT by edge, aT by arc, with the word
// kAllLive for p_e >= 1 (no p_e < 1 reaches it).
constexpr uint64_t kAllLive = ~0ull;

struct Sampler {
    uint64_t salt;
    uint64_t T;
    uint32_t all_live;
    const uint64_t* eT;   // per-edge threshold words (input edge order), or nullptr
    const uint64_t* aT;   // the same per arc (arc order), or nullptr
};

// The threshold word of every edge when there is one p.
__host__ __device__ __forceinline__ uint64_t uniform_T(const Sampler& s) {
    return s.all_live ? kAllLive : s.T;
}

__device__ __forceinline__ uint64_t edge_key(const Sampler& s, uint64_t e) {
    return mix64(s.salt ^ e);
}

__device__ __forceinline__ uint32_t mix64_hi(uint64_t x);

// Exact live test of a (key, sketch) pair against the threshold word T.
__device__ __forceinline__ bool live_T(uint64_t key, uint64_t rg, uint64_t T) {
    return T == kAllLive || mix64(key + rg) < T;
}

// Same decision, taken on the high word of the hash whenever it differs from the high word
// of T (all but a 2^-32 fraction of the pairs).
__device__ __forceinline__ bool live_T_fast(uint64_t key, uint64_t rg, uint64_t T) {
    if (T == kAllLive) return true;
    const uint32_t hh = mix64_hi(key + rg), th = (uint32_t)(T >> 32);
    if (hh != th) return hh < th;
    return mix64(key + rg) < T;
}

__device__ __forceinline__ bool edge_live(const Sampler& s, uint64_t key, uint32_t r) {
    return live_T(key, (uint64_t)(r + 1u) * kGamma, uniform_T(s));
}

// High 32 bits of mix64(x), computed without the low half of the last multiply and shift:
// if w = z * C2 (mod 2^64), the finaliser returns w ^ (w >> 31), whose high word is
// hi(w) ^ (hi(w) >> 31).  hi(mix64(x)) <= hi(T) is a superset test of mix64(x) < T (equal
// high words need the full value), so callers confirm those pairs with edge_live().
__device__ __forceinline__ uint32_t mix64_hi(uint64_t x) {
    uint64_t z = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = z ^ (z >> 27);
    const uint32_t zl = (uint32_t)z, zh = (uint32_t)(z >> 32);
    const uint32_t cl = 0x133111EBu, ch = 0x94D049BBu;          // 0x94D049BB133111EB
    const uint32_t wh = __umulhi(zl, cl) + zl * ch + zh * cl;  // hi 32 bits of z * C2
    return wh ^ (wh >> 31);
}

// High word of mix64(x) before its last step (w ^ (w >> 31) for the high word w of z * C2):
// the final high word differs from w at most in bit 0, so  final <= th  implies  w <= th + 1,
// which makes w a candidate test that needs neither the low half of the last product nor the
// last shift.
__device__ __forceinline__ uint32_t mix64_hi_raw(uint64_t x) {
    uint64_t z = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = z ^ (z >> 27);
    const uint32_t zl = (uint32_t)z, zh = (uint32_t)(z >> 32);
    return __umulhi(zl, 0x133111EBu) + zl * 0x94D049BBu + zh * 0x133111EBu;   // hi(z * C2)
}

struct GraphView {
    uint32_t n;
    uint64_t m;
    const uint2* edges;     // m (padded to even): (u, v)
    const uint64_t* off;    // n + 1 CSR offsets
    const uint4* arcs;      // 2m: (neighbour | center bit << 31, neighbour's center index or
                            // kNone, key lo, key hi), key = mix(salt ^ e); rewritten by every
                            // build, arcs to centers first in each adjacency list
    const uint32_t* ccnt;   // n: arcs to centers of each vertex (the first ccnt[x] of its list)
};

struct SketchView {
    uint32_t R, rho, all_centers;
    const uint32_t* cbits;   // center bitmap, ceil(n/32) words (unused when all_centers)
    const uint32_t* cidx;    // center index per vertex, kNone otherwise (unused when all)
    const uint32_t* label;   // [rho + hubs][R]
    uint32_t* size;          // [rho + hubs][R], bit 31 = covered by a seed
    const uint8_t* seed_flag;
    uint32_t pend;           // a seed whose flag is being set concurrently (kNone: none)
    uint32_t pend2;          // a second one: the candidate assumed to win (kNone: none)
    uint64_t* labcache;      // [kLabSlots][R] labels found by searches, reused by MarkSeed
    Sampler smp;
};

// Whether x is a seed: its flag, or a seed a step running in the same kernel is adding.
__device__ __forceinline__ bool is_seed(const SketchView& s, uint32_t x) {
    return s.seed_flag[x] || x == s.pend || x == s.pend2;
}

__device__ __forceinline__ bool is_center(const SketchView& s, uint32_t x) {
    return s.all_centers || ((__ldg(s.cbits + (x >> 5)) >> (x & 31)) & 1u);
}
__device__ __forceinline__ uint32_t center_index(const SketchView& s, uint32_t x) {
    return s.all_centers ? x : __ldg(s.cidx + x);
}

// Request mailbox of a device-resident selection loop (im_serve_launch), in mapped pinned host
// memory.  The host writes a requested k into the ring and raises head; the loop on the
// device takes every pending request, extends the greedy sequence to the largest k, copies
// the new seeds and gains behind the ring and raises `answered`.  Layout: this header, then
// k[ring] (u32), seeds[kcap] (u32), gains[kcap] (u64, 8-byte aligned).
struct MailboxShared {
    unsigned int head;           // host: requests pushed (counts up)
    unsigned int tail;           // device: requests taken (counts up)
    unsigned int answered;       // device: seeds published
    int status;                  // device: IM_ETIMEOUT after an idle exit, IM_EDEVICE after a
                                 // selection error, else IM_OK
    unsigned int running;        // host sets it before a launch; the device clears it when its loop
                                 // stops taking requests
    unsigned int stop;           // host: end the loop at its next wait
    unsigned int exits;          // device: loop launches that ended
    unsigned int ring;           // capacity of k[] (requests in flight)
    unsigned int kcap;           // capacity of seeds[] / gains[]
    unsigned int pad0;
    unsigned long long idle_ns;  // a wait with no request ends the loop after this long
    unsigned int pad[4];
};
static_assert(sizeof(MailboxShared) == 64, "mailbox header");

// Device-side selection state (one per context).
struct SelState {
    unsigned long long best;        // max fresh key this round
    unsigned long long stale_max;   // max stale key over unevaluated candidates
    unsigned long long n_unev;      // number of unevaluated candidates
    unsigned long long count_above; // unevaluated candidates whose stale key beats best
    unsigned long long best_prev;   // best fresh key when the current batch was chosen
    // radix selection of a batch (PH_SEL_PASS): key prefix so far, keys still to take, threshold
    unsigned long long prefix, prefmask, need, taken, theta, borig;
    int shift, done;
    unsigned long long eval_next;   // task counter of the chunk evaluation kernel
    unsigned int batch_n;
    unsigned int fb_n;              // fallback tasks queued
    unsigned int fb_overflow;
    unsigned long long evals_total;
    unsigned long long fb_total;
    unsigned long long hop1_arcs;       // arcs scanned by the first hop (per 32 sketches)
    unsigned long long hop2_calls;      // (vertex, sketch) searches needing more than one hop
    unsigned long long hop2_chunks;     // 32-arc chunks scanned by those searches
    unsigned int err;               // SelError: the selection stopped (the host reports it)
    unsigned int pad;
    // round and batch control, decided on the device (plan_step)
    unsigned int round;             // seeds chosen so far
    unsigned int round_end;         // stop after this many seeds
    unsigned int j;                 // batches evaluated in the current round
    unsigned int cont;              // the current round needs another batch
    unsigned int mode;              // SelMode of that batch
    unsigned int sd;                // the round's winner (valid once cont == 0)
    unsigned long long refresh_min; // batches at least this large are evaluated by refresh
    unsigned long long evals_mark;  // evals_total when the round started
    unsigned long long batches, refresh_batches;
    unsigned long long launches;    // kernels the selection graph launched
    unsigned int ticket;            // blocks of the current launch done (the last one runs its epilogue)
    unsigned int pending;           // a batch was evaluated and awaits its accounting
    // candidate first seeds whose overlaps the build accumulated (M_SPEC evaluates round 1)
    unsigned int spec_count;
    unsigned int spec_idx;          // which candidate the first seed is, else kNone
    unsigned int spec_ids[kSpecMax];
    unsigned long long spec_batches;
    unsigned int phase;             // SelPhase: what the next k_sel_step launch does
    unsigned int rare;              // SelRare: an evaluator outside k_sel_step is due
    unsigned int topb;              // batch size PH_TOPB selects (0: radix passes and a gather)
    unsigned int cond[3];           // the values last given to the graph's outer, inner and rare
                                    // conditions (a call to set one is skipped when unchanged)
    unsigned long long above_bound; // unevaluated candidates above the best fresh key before the
                                    // last batch: an upper bound on count_above
    unsigned long long stale_2nd;   // second largest stale key over the unevaluated candidates
    // a round evaluated ahead (M_MARK_PAIR): the next round's only candidate, evaluated as if
    // the current round's candidate had won; its stale key, and whether a search overflowed
    unsigned long long pair_kz;
    unsigned int pair;
    unsigned int pair_fail;
    unsigned int pair_penalty;      // grows when y lost, decays when it won or no pair ran: pairs
                                    // run while it is below kPairOff
    unsigned int pad2;
    // last: the radix pass histogram (plan_step never reads it, so its copy stops before it)
    unsigned int hist[256];
};

enum SelError : unsigned int {
    SEL_OK = 0, SEL_FB_OVERFLOW = 1, SEL_NO_PROGRESS = 2, SEL_NO_CANDIDATE = 3, SEL_RANGE = 4
};

// Launch sequences of one re-evaluation batch (the switch of the selection graph).
enum SelMode : unsigned int {
    M_DIRECT = 0,         // B = 1: the top stale key is the batch; one warp per search
    M_GATHER_SINGLE = 1,  // threshold known: gather, one warp per search
    M_HIST_SINGLE = 2,    // radix passes, gather, one warp per search
    M_GATHER_CHUNK = 3,   // gather, one warp per (member, 32 sketches)
    M_HIST_CHUNK = 4,     // radix passes, gather, one warp per (member, 32 sketches)
    M_REFRESH = 5,        // gather, recompute the sketches
    M_COUNT_ABOVE = 6,    // no batch yet: count the candidates above the best fresh key first
    // round 1 after a candidate first seed: the batch's Marginals are gain0 - its overlap sums
    M_SPEC_DIRECT = 7,    // B = 1
    M_SPEC_GATHER = 8,    // threshold known: gather
    M_SPEC_HIST = 9,      // radix passes, gather
    M_ROUND_START = 10,   // no batch: the reduction and planning step that open a round
    M_MARK = 11,          // MarkSeed of the last round's winner, then the next round opens
    M_MARK_DIRECT = 12,   // MarkSeed of the last round's winner fused with a B = 1 batch
    M_COUNT = 13,
    M_NONE = 14,          // nothing: the selection is over
    // M_MARK_DIRECT that also evaluates the second largest stale key z as the next round's
    // first batch, assuming the top key y wins this round (MarkSeed(y) applied in each sketch
    // after y's Marginal there, undone if y loses)
    M_MARK_PAIR = 15
};

// Phases of k_sel_step.  A batch of mode M runs as a few of them in a row: radix passes
// (PH_SEL_PASS, hist modes), the gather (PH_GATHER), then an evaluation phase that also scans
// the other candidates and plans the next batch (PH_EVAL, PH_MARK_EVAL), or PH_SPEC_EVAL +
// PH_SCAN.  A round opens with PH_SCAN or PH_MARK; PH_COUNT counts candidates above the best.
enum SelPhase : unsigned int {
    PH_NONE = 0, PH_SCAN, PH_MARK, PH_MARK_EVAL, PH_EVAL, PH_SEL_PASS, PH_GATHER, PH_SPEC_EVAL, PH_COUNT,
    PH_TOPB   // a batch of at most 32: the largest stale keys in one pass (replaces passes + gather)
};

// Evaluators with launch sequences of their own (the switch of the selection graph).
enum SelRare : unsigned int { RARE_CHUNK = 0, RARE_REFRESH = 1, RARE_COUNT = 2, RARE_NONE = 3 };

// Conditional-node handles of the selection graph; on == 0 outside the graph.
struct SelHandles {
    cudaGraphConditionalHandle outer, inner, rare;
    unsigned int on;
    unsigned int rare_launches[RARE_COUNT];   // kernels each rare evaluator launches
};

struct FbTask {
    uint32_t v, r, kind, idx;
};
enum FbKind : uint32_t { FB_EVAL = 0, FB_MARK = 1, FB_SPREAD = 2, FB_MARK_EVAL = 3 };

enum KernelId {
    K_PACK_EDGES = 0, K_CSR_DEGREE, K_SCAN_PARTIAL, K_SCAN_TOP, K_SCAN_APPLY, K_CSR_FILL,
    K_CENTER_HIST, K_CENTER_PICK, K_CENTER_FLAGS, K_CENTER_INDEX,
    K_BATCH_INIT, K_SAMPLE_UNION, K_COMPRESS_COUNT, K_GAIN_COMPACT, K_INIT_KEYS,
    K_REDUCE_RESET, K_REDUCE, K_SEL_INIT, K_SEL_HIST, K_SEL_PICK, K_GATHER, K_EVAL,
    K_FALLBACK, K_FINALIZE, K_MARK_SEED, K_SPREAD_TASKS, K_SPREAD_DEDUP, K_LABELS_MIN,
    K_LABELS_OUT, K_ARC_KEYS, K_SAMPLE_EMIT, K_UNION, K_COVER_ROOTS, K_REFRESH_GATHER, K_COUNT_ABOVE,
    K_ZERO, K_SELECT_GRAPH, K_SEL_BEGIN, K_SEL_STEP, K_COUNT
};

const char* kernel_name(int id);

}  // namespace imk

// ----------------------------------------------------------------------------------
// Host context.
// ----------------------------------------------------------------------------------
struct im_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    // graph
    uint32_t n = 0;
    uint64_t m = 0;
    uint2* d_edges = nullptr;
    uint64_t* d_off = nullptr;
    uint4* d_arcs = nullptr;
    uint2* d_adj = nullptr;          // static adjacency: (neighbour, edge id) per arc, CSR order
    uint32_t* d_src = nullptr;       // ... and its source
    uint32_t* d_arc_cur = nullptr;
    uint32_t graph_n_alloc = 0;      // n, m the graph buffers were allocated for
    uint64_t graph_m_alloc = 0;
    bool graph_ok = false;           // a valid edge list is loaded
    // per-edge IC probabilities (im_set_edge_probs)
    int prob_model = 0;              // IM_PROBS_*
    uint64_t* d_edgeT = nullptr;     // threshold words by edge (input order, padded to even)
    uint64_t* d_arcT = nullptr;      // the same by arc, written by every arc fill
    uint64_t edgeT_cap = 0;          // edges d_edgeT / d_arcT were allocated for
    double mean_p = 0.0;
    uint32_t* d_upload = nullptr;    // staging for host edge lists (2 x upload_cap ids)
    uint32_t* h_upload = nullptr;    // pinned staging for pageable host edge lists (same size)
    uint64_t upload_cap = 0;   // 2n arc-fill cursors (centers from the front, others from the back)
    uint64_t arc_salt = 0;
    bool arc_keys_valid = false;

    // sketches
    bool built = false;
    uint32_t R = 0, rho = 0, all_centers = 1, key_bits = 1;
    uint64_t seed = 0;
    double p = 0.0, alpha = 1.0;
    imk::Sampler smp{};
    uint32_t* d_cbits = nullptr;     // centers and hubs
    uint32_t* d_cidx = nullptr;      // center index (< rho), hub index (rho + i), or kNone
    uint32_t* d_centers = nullptr;
    uint32_t* d_label = nullptr;     // [rho + hub_rows][R]
    uint32_t* d_size = nullptr;      // [rho + hub_rows][R]
    uint64_t* d_gain0 = nullptr;
    size_t compact_cap = 0;          // entries allocated for label / size
    // Hubs: high-degree non-centers that the searches treat as centers (rows rho + i of
    // label / size, see im_select_hubs).  hub_cap = kHubsAuto: max(1024, n / 64); 0: none.
    uint32_t hub_cap = imk::kHubsAuto, hub_min_deg = 32;
    uint32_t hub_rows = 0;           // rows allocated after the rho compact rows
    uint32_t hubs = 0;               // hubs of the last build (<= hub_rows)

    // selection
    uint64_t* d_key = nullptr;
    uint32_t* d_stamp = nullptr;
    uint8_t* d_seedflag = nullptr;
    uint32_t* d_batch = nullptr;
    uint64_t* d_fresh = nullptr;
    imk::SelState* d_sel = nullptr;
    imk::SelState* h_sel = nullptr;  // pinned mirror
    uint32_t* d_seed_list = nullptr;   // seeds chosen so far, on the device (n entries)
    uint64_t* d_labcache = nullptr;    // [kLabSlots][R]: (vertex << 32) | label found by GetCenter
    uint32_t* d_pair_undo = nullptr;   // [R]: the size row an M_MARK_PAIR step covered, else kNone
    uint64_t refresh_min = 0;          // batches at least this large are evaluated by refresh
    uint64_t refresh_req = 0;          // user setting (0 = automatic)
    std::vector<uint32_t> seeds;
    std::vector<uint64_t> seed_gains;
    std::vector<uint64_t> round_evals;
    uint64_t* d_gain_list = nullptr;   // gain of each chosen seed (n entries)
    uint64_t* d_round_evals = nullptr; // re-evaluations of each round (n entries)
    // the selection loop as one CUDA graph (conditional nodes set by the device)
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;   // owned; only used to capture
    cudaGraph_t sel_graph = nullptr;
    cudaGraphExec_t sel_exec = nullptr;
    // the device-resident request loop (im_serve_launch): built for one mailbox at a time
    cudaGraph_t serve_graph = nullptr;
    cudaGraphExec_t serve_exec = nullptr;
    const void* serve_mb = nullptr;          // the mailbox serve_exec was built for
    bool serving = false;                    // a loop was launched and not finished: the host copy
                                             // of the sequence (seeds, seed_gains) is stale
    unsigned step_grid = 0;          // blocks of k_sel_step (resident at once)
    uint64_t* d_topb = nullptr;      // 32 keys per step-kernel block (PH_TOPB)
    bool capturing = false;              // launches go into a graph: no events, no counting
    bool deferred = false;               // the calls only queue work (batch graph): no host waits
    bool count_only = false;             // launches are only counted (dry run)
    uint64_t dry_count = 0;
    unsigned long long dev_launches_seen = 0;  // SelState::launches already added to launches
    unsigned long long build_live_pairs = 0;   // live pairs unioned by the last build
    // Candidate first seeds: the spec_count vertices with the largest gains over the first
    // batch of sketches (ties to the smaller id).  The build also sums, for each candidate c,
    // ov_c(v) = sum_r |C_r(v)| [c in C_r(v)], so that if the first seed is one of them round 1's
    // Marginals are gain0(v) - ov_c(v) without recomputing the sketches (exact).
    uint32_t spec_req = 4;               // user setting (0 disables)
    uint32_t spec_count = 0;             // candidates of the current build
    uint64_t* d_spec_keys = nullptr;     // kSpecMax packed gain keys, largest first
    uint32_t* d_spec_ids = nullptr;      // kSpecMax candidate ids

    // sketch-batch scratch: two lanes, each with its own stream, so that consecutive batches
    // overlap (one batch's hashing with the other's union-find)
    struct Lane {
        cudaStream_t stream = nullptr;
        uint32_t* parent = nullptr;
        uint64_t* word = nullptr;                // per root: size (low half), min label key (high)
        uint4* live = nullptr;                   // live (u, v, sketch) records of one batch
        unsigned long long* live_n = nullptr;
        uint64_t* gain = nullptr;                // lane 1: its share of the initial gains
        unsigned long long* fresh = nullptr;     // lane 1: its share of a refresh evaluation
        uint64_t* spec_ov = nullptr;             // [spec][n] overlap sums (lane 0's is the total)
    };
    Lane lane[imk::kMaxLanes];
    cudaStream_t lane_stream[imk::kMaxLanes] = {};    // lanes 1.. (owned); lane 0 is the context stream
    cudaEvent_t ev_fork = nullptr, ev_spec = nullptr;
    cudaEvent_t ev_join[imk::kMaxLanes] = {};
    cudaStream_t cur = nullptr;                  // stream the next launch goes to
    uint32_t lanes = 2;                          // sketch batches alternate between two streams
    int union_path = IM_UNION_AUTO;              // im_set_union_path
    int union_used = IM_UNION_RECORDS;           // the path the last build took (AUTO resolved)
    uint32_t batch_req = 0, batch_used = 0, batch_alloc = 0;
    uint64_t live_cap = 0;           // live-pair records allocated per lane
    // capacities of the sketch buffers (a later build that fits reuses them)
    uint32_t cap_n = 0, cap_R = 0, cap_nspec = 0;
    // sizes to allocate at least (im_create_reserved): a context that will serve several
    // instances allocates once, for the largest of each dimension
    uint32_t res_n = 0, res_R = 0;
    uint64_t res_m = 0, res_nc = 0, res_live = 0;
    unsigned long long* d_live_total = nullptr;  // live (edge, sketch) pairs unioned, cumulative

    // BFS fallback scratch
    uint32_t fb_slots = 0;
    uint32_t fb_cap = 0;
    uint32_t* d_fb_queue = nullptr;
    uint32_t* d_fb_bits = nullptr;
    imk::FbTask* d_fb_tasks = nullptr;

    // spread scratch
    uint64_t* d_spread_pairs = nullptr;
    size_t spread_cap = 0;
    uint32_t* d_spread_seeds = nullptr;
    unsigned long long* d_spread_total = nullptr;

    // center selection scratch
    uint32_t* d_cflags = nullptr;        // n: center flags
    uint64_t* d_cpos = nullptr;          // n + 1: their exclusive scan
    uint8_t* d_csel = nullptr;           // kCenterSelBytes: radix-select state
    unsigned long long* h_live = nullptr;   // pinned: live-pair counter before / after a build, hubs

    // misc scratch (scan partials, center select)
    void* d_tmp = nullptr;
    size_t tmp_bytes = 0;

    // accounting
    uint64_t launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<int, int>>> ev_pending;   // (kernel, (ev0, ev1))
    double prof_ms[imk::K_COUNT] = {};
    uint64_t prof_launches[imk::K_COUNT] = {};
};

// launch accounting (defined in im_api.cu)
void im_prof_begin(im_ctx* c, int kid, int* ev0, bool count_launch = true);
void im_prof_end(im_ctx* c, int kid, int ev0);

#define IM_LAUNCH(ctx, kid, kern, grid, block, smem, ...)                               \
    do {                                                                                \
        if ((ctx)->count_only) { (ctx)->dry_count++; break; }                           \
        int _ev0 = -1;                                                                  \
        im_prof_begin((ctx), (kid), &_ev0);                                             \
        kern<<<(grid), (block), (smem), (ctx)->cur>>>(__VA_ARGS__);                     \
        im_prof_end((ctx), (kid), _ev0);                                                \
    } while (0)

// ---- launch wrappers (host) ------------------------------------------------------
// im_graph.cu
int im_graph_build(im_ctx* c, const uint32_t* d_u, const uint32_t* d_v);
int im_arc_keys(im_ctx* c, uint64_t salt);   // keys and center bits of every arc
int im_edge_probs(im_ctx* c, int model, const double* d_p);   // per-edge thresholds
int im_scan_u32_to_u64(im_ctx* c, const uint32_t* d_in, uint64_t* d_out, uint64_t count);
int im_scan_reserve(im_ctx* c, uint64_t count);
// im_api.cu: the parts of im_build_sketches, and graph loading that only queues work
int build_prepare(im_ctx* c, uint32_t R, uint64_t seed, double p, double alpha);
int build_enqueue(im_ctx* c);
int build_finish(im_ctx* c);
int batch_load_reserve(im_ctx* c, uint32_t n, uint64_t m);
int spread_reserve(im_ctx* c, uint32_t k);
int batch_load_enqueue(im_ctx* c, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v);
// im_select.cu: the selection and spread of a batch graph
int im_select_prepare(im_ctx* c, uint32_t k);
int im_select_graph_append(im_ctx* c, cudaGraph_t g, cudaGraphNode_t after, uint32_t k, cudaGraphNode_t* last);
int im_spread_enqueue(im_ctx* c, uint32_t k, unsigned long long* h_total);
// im_sketch.cu
int im_select_centers(im_ctx* c, uint32_t* d_flags_tmp, uint64_t* d_scan_tmp);
int im_select_hubs(im_ctx* c, uint32_t* d_flags_tmp, uint64_t* d_scan_tmp);
// Minimum allocation sizes of a context that is to serve several instances.
struct ImReserve {
    uint32_t n, R;        // vertices, sketches
    uint64_t m;           // edges
    uint64_t nc;          // compact (and hub) label entries: rows x R
    double pm;            // largest p m (live-pair records per sketch)
};
int im_create_reserved(im_ctx** out, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v, int ptr_kind,
                       void* stream, const ImReserve* res);
int im_mc_run(im_ctx* c, const uint32_t* d_seeds, uint32_t k, uint32_t sims, uint64_t mc_seed,
              unsigned long long* d_total);
int im_sketch_batches(im_ctx* c);

int im_labels_min(im_ctx* c, uint32_t r, uint32_t* d_out);
int im_refresh_eval(im_ctx* c, const uint32_t* d_batch, const unsigned int* d_batch_n,
                    unsigned long long* d_fresh, const uint32_t* d_seeds, const unsigned int* d_nseeds);
// im_select.cu
int im_selection_init(im_ctx* c, bool fresh);
int im_select_run(im_ctx* c, uint32_t k);   // rounds until k seeds are chosen
void im_select_graph_free(im_ctx* c);
int im_spread_run(im_ctx* c, uint32_t k, uint64_t* out);
void im_serve_stop(im_ctx* c);   // asks a serving loop on the context to end (before a destroy)

int im_fail(im_ctx* c, int code, const std::string& msg);
// Every device allocation of the library goes through here: cudaMalloc, unless a failure was
// injected (im_debug_fail_alloc), in which case nothing is allocated and
// cudaErrorMemoryAllocation is returned.
cudaError_t im_dev_malloc(void** p, size_t bytes);
template <typename T>
inline cudaError_t im_dev_malloc(T** p, size_t bytes) { return im_dev_malloc(reinterpret_cast<void**>(p), bytes); }
// The record capacity the sketch kernels use: the allocated one, or less under im_debug_record_cap.
uint64_t im_record_cap(uint64_t allocated);
int im_cuda_check(im_ctx* c, cudaError_t e, const char* what);

#define IM_CUDA(c, call)                                                                \
    do {                                                                                \
        cudaError_t _e = (call);                                                        \
        if (_e != cudaSuccess) return im_cuda_check((c), _e, #call);                    \
    } while (0)

inline unsigned grid_for(uint64_t work, unsigned block, unsigned cap = 152u * 32u) {
    uint64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}
