// im_select.cu -- Step 2 of Alg. 1 on the device: lazy greedy seed selection (CELF, Alg. 2)
// with prefix-doubling batches of re-evaluations (the batch schedule of Alg. 4), the
// compact-sketch procedures GetCenter / Marginal / MarkSeed of Alg. 3, and the spread sum.
//
// Stale scores are kept as packed 64-bit keys  key = (gain << b) | (2^b - 1 - v), b = bit
// length of n, so a larger key means a larger gain and, for equal gains, a smaller id
// (Sec. 4 breaks ties by vertex id).  Within a round, a batch X of unevaluated candidates
// with the largest stale keys is re-evaluated; the round ends when the best fresh key beats
// every stale key not yet re-evaluated (Alg. 2's stop test on keys; Alg. 4's loop).  Stale
// keys are upper bounds by submodularity (Eq. 2), so the winner equals plain greedy's.
#include <cstring>

#include <chrono>
#include <new>
#include <thread>

#include "im_internal.cuh"

using namespace imk;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kEvalWarps = 4;   // warps per block of the search kernels
// batches with at most this many (member, sketch) searches use one warp per search
constexpr uint64_t kSingleTasks = 152ull * 64;
// chunks of 32 arcs a warp search loads per step
constexpr int kBfsChunks = 4;
// per-warp visited set of a search (open addressing, >= 2 x the queue capacity + one chunk)
constexpr uint32_t kHashSlots = 512;
// warps of a block that searches one (vertex, sketch) together (the first hop)
constexpr int kBlockWarps = 8;

// Insert y into a warp's visited set; true if it was not there.  The set never holds more
// than kQcap + 32 ids, so a free slot is always found.
__device__ __forceinline__ bool visit(uint32_t* hs, uint32_t y) {
    uint32_t h = (y * 0x9E3779B1u) >> (32 - 9);
    for (;;) {
        const uint32_t old = atomicCAS(hs + h, kNone, y);
        if (old == kNone) return true;
        if (old == y) return false;
        h = (h + 1) & (kHashSlots - 1);
    }
}

__device__ __forceinline__ uint64_t pack_key(uint64_t gain, uint32_t v, uint32_t bits) {
    const uint64_t mask = (1ull << bits) - 1ull;
    return (gain << bits) | (mask - v);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    return x;
}

// ---- GetCenter (Alg. 3) for a start vertex that is not a center ----------------------
// Warp-cooperative BFS on G'_r with the queue (= visited list) in shared memory.  Arcs of
// the current vertex are scanned 32 at a time, each lane re-hashing one arc.  Stops at the
// first center met (every center of a component carries the same label).  If the queue
// would exceed kQcap the search is abandoned (overflow) and redone by k_fallback.
struct BfsOut {
    uint32_t label;   // label of the component's centers, or kNone
    uint32_t count;   // vertices visited (the whole component when label == kNone)
    uint32_t minv;    // smallest vertex id visited
    uint32_t seen;    // a seed was visited
    uint32_t overflow;
};

// If init != nullptr, x's own arcs were already scanned: the queue starts as
// [x, init[0], init[stride], ...] (x's live non-center neighbours, distinct) with head = 1.
//
// The frontier is expanded up to 32 queued vertices at a time: lane i loads the offsets of
// queue entry head + i, a warp scan lays their arcs out one after the other, and every chunk
// of 32 arcs is tested at once (each lane finds the vertex owning its arc by a binary search
// over the prefix sums held in the lanes).  A search thus costs a few dependent load rounds
// per BFS level instead of two per visited vertex.
__device__ BfsOut warp_bfs_from(const GraphView& g, const SketchView& s, uint32_t v, uint32_t r,
                                uint32_t* q, bool want_seed, const uint32_t* init, uint32_t ninit,
                                uint32_t init_stride, SelState* st_counters) {
    const unsigned lane = threadIdx.x & 31;
    BfsOut o;
    o.label = kNone; o.count = 0; o.minv = v; o.seen = 0; o.overflow = 0;
    uint32_t chunks = 0;
    uint32_t head = 0, tail = 1;
    uint32_t seen = want_seed ? (uint32_t)is_seed(s, v) : 0u;
    uint32_t minv = v;
    const uint64_t rg = (uint64_t)(r + 1u) * kGamma;
    const uint64_t Tw = uniform_T(s.smp);   // every arc's threshold, unless they have their own
    uint32_t* hs = q + kQcap;   // visited set (the queue holds the same ids, in order)
    for (uint32_t i = lane; i < kHashSlots; i += 32) hs[i] = kNone;
    __syncwarp();
    if (lane == 0) {
        q[0] = v;
        visit(hs, v);
    }
    if (init) {
        for (uint32_t t = lane; t < ninit; t += 32) {
            const uint32_t y = init[t * init_stride];   // distinct neighbours of v
            q[1 + t] = y;
            visit(hs, y);
            if (want_seed && is_seed(s, y)) seen = 1;
            minv = min(minv, y);
        }
        head = 1;
        tail = 1 + ninit;
    }
    __syncwarp();
    while (head < tail) {
        const uint32_t nv = min(32u, tail - head);
        uint64_t a0 = 0;
        uint32_t deg = 0, cc = 0;
        if (lane < nv) {
            const uint32_t x = q[head + lane];
            a0 = g.off[x];
            deg = (uint32_t)(g.off[x + 1] - a0);
            cc = g.ccnt[x];   // its arcs to centers, stored first
        }
        // The step's arcs in two runs: the arcs to centers of every frontier vertex, then the
        // others, so that a live center anywhere in the frontier is met before any vertex's
        // long tail of non-center arcs.  Inclusive scans of both lengths:
        uint32_t preC = cc, preN = deg - cc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t yc = __shfl_up_sync(kFull, preC, d);
            const uint32_t yn = __shfl_up_sync(kFull, preN, d);
            if ((int)lane >= d) { preC += yc; preN += yn; }
        }
        const uint32_t totC = __shfl_sync(kFull, preC, 31);
        const uint32_t total = totC + __shfl_sync(kFull, preN, 31);
        preC -= cc;           // exclusive
        preN -= deg - cc;
        const uint64_t aN = a0 + cc;   // where the non-center arcs start
        head += nv;
        // kBfsChunks 32-arc chunks per step: their loads are in flight together
        for (uint32_t base = 0; base < total; base += 32u * kBfsChunks) {
            uint4 arcs4[kBfsChunks];
            uint64_t tk[kBfsChunks];
#pragma unroll
            for (int k = 0; k < kBfsChunks; ++k) {
                const uint32_t t = base + 32u * k + lane;
                const bool inC = t < totC;
                const uint32_t tt = inC ? t : t - totC;   // position within its run
                uint32_t lo = 0;
                if (nv > 1) {   // owner of arc tt in its run: the largest i < nv with pre_i <= tt
                    uint32_t hi = nv - 1;
#pragma unroll
                    for (int it = 0; it < 5; ++it) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        const uint32_t pc = __shfl_sync(kFull, preC, mid);
                        const uint32_t pn = __shfl_sync(kFull, preN, mid);
                        if ((inC ? pc : pn) <= tt) lo = mid; else hi = mid - 1;
                        if (lo > hi) hi = lo;
                    }
                }
                const uint64_t aoc = __shfl_sync(kFull, a0, lo);
                const uint64_t aon = __shfl_sync(kFull, aN, lo);
                const uint32_t poc = __shfl_sync(kFull, preC, lo);
                const uint32_t pon = __shfl_sync(kFull, preN, lo);
                const uint64_t ao = inC ? aoc : aon;
                const uint32_t po = inC ? poc : pon;
                const uint64_t ai = ao + (tt - po);
                arcs4[k] = (t < total) ? g.arcs[ai] : make_uint4(0, 0, 0, 0);
                tk[k] = (t < total && s.smp.aT) ? s.smp.aT[ai] : Tw;
            }
#pragma unroll
            for (int k = 0; k < kBfsChunks; ++k) {
                if (base + 32u * k >= total) break;
                ++chunks;
                const uint32_t t = base + 32u * k + lane;
                bool live = false, cen = false;
                uint32_t y = 0, ci = 0;
                if (t < total) {
                    const uint4 arc = arcs4[k];
                    y = arc.x & kArcIdMask;
                    cen = arc.x >> 31;
                    ci = arc.y;
                    live = live_T_fast(((uint64_t)arc.w << 32) | arc.z, rg, tk[k]);
                }
                const unsigned cb = __ballot_sync(kFull, live && cen);
                if (cb) {
                    const uint32_t c0 = __shfl_sync(kFull, ci, __ffs(cb) - 1);   // the arc's center index
                    o.label = s.label[(size_t)c0 * s.R + r];
                    if (lane == 0 && st_counters) atomicAdd(&st_counters->hop2_chunks, (unsigned long long)chunks);
                    return o;
                }
                // first visit (parallel edges or several frontier vertices reaching y in this
                // chunk: the set's CAS keeps exactly one lane)
                const bool fresh = live && visit(hs, y);
                const unsigned nbm = __ballot_sync(kFull, fresh);
                const uint32_t cnt = __popc(nbm);
                if (tail + cnt > kQcap) { o.overflow = 1; return o; }
                if (fresh) {
                    q[tail + __popc(nbm & ((1u << lane) - 1u))] = y;
                    if (want_seed && is_seed(s, y)) seen = 1;
                    minv = min(minv, y);
                }
                tail += cnt;
                __syncwarp();
            }
        }
    }
    if (lane == 0 && st_counters) atomicAdd(&st_counters->hop2_chunks, (unsigned long long)chunks);
    o.seen = __any_sync(kFull, seen) ? 1u : 0u;
#pragma unroll
    for (int d = 16; d; d >>= 1) minv = min(minv, __shfl_xor_sync(kFull, minv, d));
    o.minv = minv;
    o.count = tail;
    return o;
}

// ---- GetCenter by a whole block: the first hop shared by its warps -------------------------
// A hub's first hop (its own adjacency list) dominates its search when few of its arcs are
// live (small p_e on hub edges, e.g. the weighted cascade).  The block's warps scan x's arcs
// together, 4 chunks of 32 per warp in flight, and stop as soon as one meets a live center
// (every center of a component carries its label); otherwise the distinct live non-center
// neighbours they collected seed warp 0's warp_bfs_from, which finishes the search.
constexpr uint32_t kBlockSlots = 1024;   // the block's set of x's neighbours

struct BlockSearchSmem {
    uint32_t qw[kQcap + kHashSlots];   // warp 0's queue and visited set
    uint32_t list[kQcap];              // x's live non-center neighbours
    uint32_t set[kBlockSlots];         // ... deduplicated
    uint32_t label, count, overflow, seen;
};

// Insert y into the block's set with at most kBlockSlots probes: 1 new, 0 already there,
// -1 full (the warps may insert beyond the list's capacity before they see the overflow).
__device__ __forceinline__ int visit_bounded(uint32_t* set, uint32_t y) {
    uint32_t h = (y * 0x9E3779B1u) >> (32 - 10);
    for (uint32_t i = 0; i < kBlockSlots; ++i) {
        const uint32_t old = atomicCAS(set + h, kNone, y);
        if (old == kNone) return 1;
        if (old == y) return 0;
        h = (h + 1) & (kBlockSlots - 1);
    }
    return -1;
}

// Call with the whole block (it synchronises); the result is valid in warp 0.
__device__ BfsOut block_search(const GraphView& g, const SketchView& s, uint32_t x, uint32_t r, bool want_seed,
                               BlockSearchSmem& sm, SelState* st_counters) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t i = threadIdx.x; i < kBlockSlots; i += blockDim.x) sm.set[i] = kNone;
    if (threadIdx.x == 0) {
        sm.label = kNone;
        sm.count = 0;
        sm.overflow = 0;
        sm.seen = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) visit_bounded(sm.set, x);
    __syncthreads();
    const uint64_t a0 = g.off[x], a1 = g.off[x + 1];
    const uint64_t rg = (uint64_t)(r + 1u) * kGamma;
    const uint64_t Tw = uniform_T(s.smp);
    for (uint64_t base = a0 + (uint64_t)warp * 128; base < a1; base += (uint64_t)nwarps * 128) {
        // stop once a live center was met or the neighbour list overflowed (warp-uniform)
        const uint32_t stop = __shfl_sync(kFull, (*(volatile uint32_t*)&sm.label != kNone) |
                                                     *(volatile uint32_t*)&sm.overflow, 0);
        if (stop) break;
        uint4 arcs4[4];
        uint64_t tk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t a = base + 32u * k + lane;
            arcs4[k] = a < a1 ? g.arcs[a] : make_uint4(0, 0, 0, 0);
            tk[k] = (a < a1 && s.smp.aT) ? s.smp.aT[a] : Tw;
        }
        bool found = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t a = base + 32u * k + lane;
            bool live = false;
            if (a < a1) live = live_T_fast(((uint64_t)arcs4[k].w << 32) | arcs4[k].z, rg, tk[k]);
            const bool cen = arcs4[k].x >> 31;
            const unsigned cb = __ballot_sync(kFull, live && cen);
            if (cb) {
                if ((int)lane == __ffs(cb) - 1) atomicCAS(&sm.label, kNone, s.label[(size_t)arcs4[k].y * s.R + r]);
                found = true;
                break;
            }
            if (live) {
                const uint32_t y = arcs4[k].x & kArcIdMask;
                const int fresh = visit_bounded(sm.set, y);
                if (fresh < 0) {
                    sm.overflow = 1;
                } else if (fresh) {
                    const uint32_t pos = atomicAdd(&sm.count, 1u);
                    if (pos < kQcap - 1) sm.list[pos] = y;
                    else sm.overflow = 1;
                    if (want_seed && is_seed(s, y)) sm.seen = 1;
                }
            }
        }
        if (found) break;
    }
    __syncthreads();
    BfsOut o;
    o.label = sm.label; o.count = 0; o.minv = x; o.seen = 0; o.overflow = 0;
    if (o.label != kNone) return o;
    if (sm.overflow) {
        o.overflow = 1;
        return o;
    }
    if (warp == 0) o = warp_bfs_from(g, s, x, r, sm.qw, want_seed, sm.list, sm.count, 1, st_counters);
    return o;
}

// ---- GetCenter (Alg. 3) for 32 sketches at once: lane l answers sketch r_lo + l ---------
// First hop: the warp loads 32 arcs of the start vertex x with one coalesced load, then
// broadcasts them one by one (shuffles); every lane tests the arc in its own sketch.  A lane
// is done when it meets a center, or when x has no live arc in its sketch.  A lane that saw
// only non-center live neighbours keeps them (up to kLaneQ - 1, interleaved by lane in
// shared memory) and is finished by the warp-cooperative search, which starts from that
// frontier instead of rescanning x.  Searches that outgrow kQcap go to k_fallback.
constexpr uint32_t kLaneQ = 32;

struct LaneRes {
    uint32_t label, count, minv, seen, overflow;
};

__device__ BfsOut warp_bfs_from(const GraphView& g, const SketchView& s, uint32_t v, uint32_t r,
                                uint32_t* q, bool want_seed, const uint32_t* init, uint32_t ninit,
                                uint32_t init_stride, SelState* st_counters);

__device__ LaneRes get_center_32(const GraphView& g, const SketchView& s, uint32_t x, uint32_t r_lo,
                                 uint32_t r_hi, uint32_t* ql, uint32_t* qw, bool want_seed,
                                 SelState* st_counters) {
    const unsigned lane = threadIdx.x & 31;
    const uint32_t r = r_lo + lane;
    bool act = r < r_hi;
    LaneRes o;
    o.label = kNone; o.count = 1; o.minv = x; o.overflow = 0;
    o.seen = (act && want_seed) ? (uint32_t)is_seed(s, x) : 0u;
    uint32_t cnt = 0;        // live non-center neighbours of x recorded
    bool over = false;       // more than kLaneQ - 1 of them
    const uint64_t rg = (uint64_t)(r + 1u) * kGamma;
    const uint64_t Tw = uniform_T(s.smp);
    const uint64_t a0 = g.off[x], a1 = g.off[x + 1];
    for (uint64_t base = a0; base < a1; base += 32) {
        if (!__any_sync(kFull, act)) break;
        const uint64_t a = base + lane;
        uint4 arc = make_uint4(0, 0, 0, 0);
        uint64_t ta = Tw;
        if (a < a1) {
            arc = g.arcs[a];
            if (s.smp.aT) ta = s.smp.aT[a];
        }
        const uint32_t nv = (uint32_t)min((uint64_t)32, a1 - base);
        for (uint32_t i = 0; i < nv; ++i) {
            const uint32_t yc = __shfl_sync(kFull, arc.x, i);
            const uint32_t klo = __shfl_sync(kFull, arc.z, i);
            const uint32_t khi = __shfl_sync(kFull, arc.w, i);
            const uint64_t Ti = s.smp.aT ? __shfl_sync(kFull, ta, i) : Tw;
            if (act) {
                const uint64_t key = ((uint64_t)khi << 32) | klo;
                if (live_T_fast(key, rg, Ti)) {
                    const uint32_t y = yc & kArcIdMask;
                    if (yc >> 31) {
                        o.label = s.label[(size_t)center_index(s, y) * s.R + r];
                        act = false;
                    } else if (!over) {
                        bool dup = false;   // parallel edges reach the same neighbour twice
                        for (uint32_t t = 0; t < cnt; ++t)
                            if (ql[t * 32 + lane] == y) { dup = true; break; }
                        if (!dup) {
                            if (cnt == kLaneQ - 1) over = true;
                            else ql[(cnt++) * 32 + lane] = y;
                        }
                    }
                }
            }
        }
    }
    __syncwarp();
    // lanes still active: no center among x's neighbours; cnt == 0 means x is alone
    unsigned need = __ballot_sync(kFull, act && (cnt > 0 || over));
    if (lane == 0 && st_counters) {
        atomicAdd(&st_counters->hop1_arcs, (unsigned long long)(a1 - a0));
        atomicAdd(&st_counters->hop2_calls, (unsigned long long)__popc(need));
    }
    while (need) {
        const int l = __ffs(need) - 1;
        need &= need - 1;
        const uint32_t ninit = __shfl_sync(kFull, over ? 0xFFFFFFFFu : cnt, l);
        const BfsOut w = (ninit == 0xFFFFFFFFu)
                             ? warp_bfs_from(g, s, x, r_lo + l, qw, want_seed, nullptr, 0, 0, st_counters)
                             : warp_bfs_from(g, s, x, r_lo + l, qw, want_seed, ql + l, ninit, 32, st_counters);
        if ((int)lane == l) {
            o.label = w.label; o.count = w.count; o.minv = w.minv; o.seen = w.seen;
            o.overflow = w.overflow;
        }
        __syncwarp();
    }
    return o;
}

__device__ __forceinline__ void push_fallback(SelState* st, FbTask* tasks, uint32_t cap, uint32_t v,
                                              uint32_t r, uint32_t kind, uint32_t idx) {
    uint32_t t = atomicAdd(&st->fb_n, 1u);
    if (t < cap) {
        FbTask f;
        f.v = v; f.r = r; f.kind = kind; f.idx = idx;
        tasks[t] = f;
    } else {
        st->fb_overflow = 1;
    }
}

// ---- selection kernels ---------------------------------------------------------------
__global__ void k_init_keys(const uint64_t* __restrict__ gain0, uint32_t n, uint32_t bits,
                            uint64_t* __restrict__ key, uint32_t* __restrict__ stamp,
                            uint8_t* __restrict__ seedflag, uint32_t* __restrict__ size,
                            uint64_t nsize) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        key[i] = pack_key(gain0[i], (uint32_t)i, bits);
        stamp[i] = 0;
        seedflag[i] = 0;
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsize; i += stride)
        size[i] &= ~kCovered;
}


constexpr uint32_t kPending = 0x80000000u;   // stamp bit: batch member awaiting its fresh key
// M_MARK_PAIR steps pay off when the evaluated-ahead round is usually taken: a lost pair adds
// kPairLoss to the penalty, a taken one shrinks it by a quarter, and a round that could have
// had a pair but was refused takes kPairRetry off, so that pairs are tried again after a while
constexpr uint32_t kPairOff = 64, kPairLoss = 96, kPairRetry = 4;
constexpr uint32_t kTopB = 32;               // largest batch PH_TOPB selects (one key per lane)

// The first phase of a step of the given mode (PH_NONE: the selection is over).
__device__ __forceinline__ unsigned first_phase(unsigned mode) {
    switch (mode) {
    case M_ROUND_START: return PH_SCAN;
    case M_MARK: return PH_MARK;
    case M_MARK_DIRECT: case M_MARK_PAIR: return PH_MARK_EVAL;
    case M_COUNT_ABOVE: return PH_COUNT;
    case M_DIRECT: return PH_EVAL;
    case M_SPEC_DIRECT: return PH_SPEC_EVAL;
    case M_HIST_SINGLE: case M_HIST_CHUNK: case M_SPEC_HIST: return PH_SEL_PASS;
    case M_GATHER_SINGLE: case M_GATHER_CHUNK: case M_SPEC_GATHER: case M_REFRESH: return PH_GATHER;
    default: return PH_NONE;
    }
}

// A graph condition set from the device, skipped when it already holds the value (each call
// costs a device-runtime round trip; the loops' values rarely change).
__device__ __forceinline__ void set_cond(SelState* st, int which, cudaGraphConditionalHandle h, unsigned v) {
    if (st->cond[which] != v) {
        cudaGraphSetConditional(h, v);
        st->cond[which] = v;
    }
}

// The next step is `mode`: its first phase, and the graph's loops entered (or left).
__device__ void set_step(SelState* st, const SelHandles& hd, unsigned mode) {
    unsigned ph = first_phase(mode);
    if ((ph == PH_SEL_PASS || ph == PH_GATHER) && st->topb) ph = PH_TOPB;
    st->phase = ph;
    st->rare = RARE_NONE;
    if (hd.on) {
        set_cond(st, 0, hd.outer, ph != PH_NONE ? 1u : 0u);
        set_cond(st, 1, hd.inner, ph != PH_NONE ? 1u : 0u);
        set_cond(st, 2, hd.rare, RARE_NONE);
    }
}

// The batch is evaluated outside k_sel_step: leave the inner loop for the graph's switch.
__device__ void set_rare(SelState* st, const SelHandles& hd, unsigned rare) {
    st->phase = PH_NONE;
    st->rare = rare;
    atomicAdd(&st->launches, (unsigned long long)hd.rare_launches[rare]);   // block 0 counts concurrently
    if (hd.on) {
        set_cond(st, 1, hd.inner, 0u);
        set_cond(st, 2, hd.rare, rare);
    }
}

// The outcome of an M_MARK_PAIR step: MarkSeed(x), then in each sketch y's Marginal, MarkSeed(y)
// and z's Marginal with x and y as seeds (z: the largest stale key after y's).  Every other
// stale key is at most z's, so y wins its round iff its fresh key beats z's stale key.  If y
// wins, the state becomes what an M_MARK_DIRECT step for y followed by one for z would leave:
// y's round closed and recorded, z's round opened with z evaluated (the step's scan left out
// x, y and z, as the second step's would).  If a search of the step overflowed, z's value is
// incomplete: y's round is closed and the next step marks y everywhere (MarkSeed is
// idempotent) and opens z's round afresh.  If y loses, z's value is dropped (the step's
// epilogue has undone y's marks) and the round goes on from y's batch with z among the
// unevaluated candidates.  Returns true if the next step is already set.
__device__ bool pair_resolve(SelState* st, uint32_t* __restrict__ batch, unsigned long long* __restrict__ fresh,
                             uint64_t* __restrict__ key, uint32_t* __restrict__ stamp, uint8_t* __restrict__ seedflag,
                             uint32_t* __restrict__ seed_list, uint64_t* __restrict__ gain_list,
                             uint64_t* __restrict__ round_evals, uint32_t n, uint32_t bits, const SelHandles& hd) {
    st->pair = 0;
    const bool fail = st->pair_fail != 0;
    st->pair_fail = 0;
    const uint32_t y = batch[0], z = batch[1];
    const unsigned long long fy = key[y];   // finalised by the step
    if (st->err || st->fb_overflow) return false;   // the selection stops
    const bool won = fy > st->pair_kz;
    st->pair_penalty = (won && !fail) ? st->pair_penalty - st->pair_penalty / 4 : min(st->pair_penalty + kPairLoss, 1024u);
    if (!won) {
        // y loses: z is an unevaluated candidate again, the largest left
        st->stale_2nd = st->stale_max;
        st->stale_max = st->pair_kz;
        st->n_unev += 1;
        st->above_bound += 1;   // best_prev is 0 for this batch
        return false;
    }
    // y's batch accounted and its round closed, as plan_step does
    st->pending = 0;
    st->evals_total += 1;
    st->fb_total += min(st->fb_n, 0xFFFFFFFFu);
    st->fb_n = 0;
    const uint32_t rd = st->round;
    st->sd = y;
    seed_list[rd] = y;
    gain_list[rd] = fy >> bits;
    round_evals[rd] = st->evals_total - st->evals_mark;
    st->round = rd + 1;
    st->evals_mark = st->evals_total;
    seedflag[y] = 1;   // its components are marked (or it is the pending seed of its searches)
    key[y] = 0;
    if (fail) {
        st->j = 0;
        st->best = 0;
        st->stale_max = 0;
        st->stale_2nd = 0;
        st->n_unev = 0;
        st->above_bound = 0;
        st->count_above = 0;
        st->cont = 1;
        st->mode = M_MARK;
        set_step(st, hd, M_MARK);
        return true;
    }
    // z's round: its first batch {z} is evaluated
    const unsigned long long fz = pack_key(fresh[1], z, bits);
    key[z] = fz;
    stamp[z] = rd + 1;
    batch[0] = z;
    fresh[0] = fresh[1];
    st->batch_n = 1;
    st->eval_next = 0;
    st->best_prev = 0;
    st->borig = 1;
    st->need = 1;
    st->taken = 0;
    st->prefix = 0;
    st->theta = st->pair_kz;
    st->shift = 0;
    st->prefmask = 0;
    st->done = 1;
    st->pending = 1;
    st->j = 1;
    st->batches++;
    st->best = fz;
    st->count_above = 0;
    return false;
}

// Next step of the round, decided from the state the last reduction left (Alg. 2's stop
// test; Alg. 4's doubling batch size): either a batch of ~B of the largest stale keys, picked
// by radix selection on the key bytes below the top byte of stale_max (all of them when at
// most 2B remain, exactly the top key when B = 1), or the end of the round, whose winner
// (the best fresh key) is recorded.  Large batches are evaluated by recomputing the sketches
// (M_REFRESH) instead of by searches; that choice needs the number of candidates above the
// best fresh key, which a first M_COUNT_ABOVE step counts.  Errors stop the selection.  Run
// by one thread; sets the selection graph's batch loop and batch switch.
__device__ void plan_step(SelState* st, uint32_t* __restrict__ batch, unsigned long long* __restrict__ fresh,
                          uint64_t* __restrict__ key, uint32_t* __restrict__ stamp, uint8_t* __restrict__ seedflag,
                          uint32_t* __restrict__ seed_list, uint64_t* __restrict__ gain_list,
                          uint64_t* __restrict__ round_evals, uint32_t n, uint32_t R, uint32_t bits,
                          const SelHandles& hd, bool have_count) {
    const uint64_t mask = (1ull << bits) - 1ull;
    if (st->pair && pair_resolve(st, batch, fresh, key, stamp, seedflag, seed_list, gain_list, round_evals, n, bits,
                                 hd))
        return;
    unsigned cont = 0, mode = M_NONE;
    const unsigned long long nu = st->n_unev, smax = st->stale_max, best = st->best, s2 = st->stale_2nd;
    const unsigned j = st->j;
    if (j == 0 && st->round >= st->round_end) {   // every requested seed is chosen and marked
        st->best = 0;                              // a later run opens this round again
        st->stale_max = 0;
        st->stale_2nd = 0;
        st->n_unev = 0;
        st->above_bound = 0;
        st->count_above = 0;
        st->cont = 0;
        st->mode = M_NONE;
        set_step(st, hd, M_NONE);
        return;
    }
    if (st->pending) {   // the batch evaluated since the last step
        st->pending = 0;
        const unsigned bn = st->batch_n;
        st->evals_total += bn;
        st->fb_total += min(st->fb_n, 0xFFFFFFFFu);
        st->fb_n = 0;    // the fallback kernel has run; MarkSeed may queue its own searches
        if (!st->err && bn == 0) st->err = SEL_NO_PROGRESS;
    }
    if (!st->err && st->fb_overflow) st->err = SEL_FB_OVERFLOW;
    if (!st->err && nu > 0 && best <= smax) {
        if (j > 81) st->err = SEL_NO_PROGRESS;   // doubling covers any n within 64 batches
        else cont = 1;
    }
    // the count of candidates above the best fresh key only decides a recomputation, which
    // needs at least refresh_min of them: skipped when the scans' upper bound is below that
    if (cont && best && !have_count && st->above_bound >= st->refresh_min) {
        mode = M_COUNT_ABOVE;
        st->count_above = 0;
    } else if (cont) {
        unsigned long long B = 1ull << (j < 40 ? j : 40);
        if (B > nu) B = nu;
        unsigned long long expect = 2 * B < nu ? 2 * B : nu;
        // When many candidates could still beat the best fresh key (or the doubling batch
        // has grown large), evaluate every one of them at once by recomputing the sketches;
        // the round then ends, since all remaining stale keys are below the new best.
        const unsigned long long rmin = st->refresh_min;
        const unsigned long long above = st->count_above;
        const bool refresh = expect >= rmin || (best && above >= rmin);
        if (refresh) {
            B = nu;
            expect = best ? above : nu;
        }
        st->borig = B;
        st->need = B;
        st->taken = 0;
        st->prefix = 0;
        st->theta = 0;
        bool hist = false, direct = false;
        if (nu <= 2 * B || smax == 0) {
            st->done = 1;                // take every unevaluated candidate
            st->shift = 0;
            st->prefmask = 0;
        } else if (B == 1) {
            st->done = 1;                // keys are distinct: exactly the top stale key
            st->theta = smax;
            st->shift = 0;
            st->prefmask = 0;
            direct = best < smax;        // no gather needed: the key names the vertex
        } else {
            const int top = 63 - __clzll((long long)smax);
            const int shift = (top / 8) * 8;
            st->shift = shift;
            st->prefmask = (shift + 8 >= 64) ? 0ull : ~((1ull << (shift + 8)) - 1ull);
            st->done = 0;
            hist = true;
        }
        st->batch_n = 0;
        st->eval_next = 0;
        st->fb_n = 0;
        st->best_prev = best;
        st->best = 0;
        st->stale_max = 0;
        st->stale_2nd = 0;
        st->n_unev = 0;
        st->above_bound = 0;
        st->count_above = 0;
        if (direct) {
            const uint32_t x = (uint32_t)(mask - (smax & mask));
            batch[0] = x;
            fresh[0] = 0;
            key[x] = 0;                       // its batch slot
            stamp[x] = st->round | kPending;
            st->batch_n = 1;
        }
        const bool single = expect * R <= kSingleTasks;
        // Round 1 after a candidate first seed: the same batches, evaluated from the overlap sums
        const bool spec = st->round == 1 && st->spec_idx < st->spec_count;
        mode = spec    ? (direct ? M_SPEC_DIRECT : hist ? M_SPEC_HIST : M_SPEC_GATHER)
             : refresh ? M_REFRESH
             : direct  ? M_DIRECT
             : single  ? (hist ? M_HIST_SINGLE : M_GATHER_SINGLE)
                       : (hist ? M_HIST_CHUNK : M_GATHER_CHUNK);
        // a batch of at most kTopB -- the B largest stale keys, or every unevaluated candidate
        // when at most 2B remain -- is selected in one pass (PH_TOPB) instead of radix passes
        // and a gather
        const unsigned long long want = hist ? B : nu;
        st->topb = (!direct && !refresh && (single || spec) && want <= kTopB) ? (unsigned)want : 0u;
        st->pending = 1;
        st->j = j + 1;
        st->batches++;
        if (spec) st->spec_batches++;
        else if (refresh) st->refresh_batches++;
    } else if (!st->err) {
        // the round is over: the best fresh key beats every stale one
        const uint32_t sd = (uint32_t)(mask - (best & mask));
        if (best == 0) {
            st->err = SEL_NO_CANDIDATE;
        } else if (sd >= n) {
            st->err = SEL_RANGE;
        } else {
            const uint32_t rd = st->round;
            st->sd = sd;
            seed_list[rd] = sd;
            if (rd == 0)
                for (unsigned k = 0; k < st->spec_count; ++k)
                    if (st->spec_ids[k] == sd) st->spec_idx = k;
            gain_list[rd] = best >> bits;
            const unsigned long long evals = st->evals_total - st->evals_mark;
            round_evals[rd] = evals;
            // The next round.  If this one evaluated its winner only, every other key is as it
            // was at its start, so the next round's top key is this reduction's stale_max and
            // its first batch (B = 1, that key) is known now: it runs fused with the MarkSeed.
            st->round = rd + 1;
            st->j = 0;
            st->evals_mark = st->evals_total;
            st->best = 0;
            st->stale_max = 0;
            st->stale_2nd = 0;
            st->n_unev = 0;
            st->above_bound = 0;
            st->count_above = 0;
            cont = 1;
            mode = M_MARK;
            if (rd + 1 < st->round_end && rd >= 1 && evals == 1 && nu > 2 && smax > 0 && st->refresh_min > 2) {
                const uint32_t y = (uint32_t)(mask - (smax & mask));
                batch[0] = y;
                fresh[0] = 0;
                key[y] = 0;                        // its batch slot
                stamp[y] = (rd + 1) | kPending;
                st->batch_n = 1;
                st->eval_next = 0;
                st->fb_n = 0;
                st->best_prev = 0;
                st->borig = 1;
                st->need = 1;
                st->taken = 0;
                st->prefix = 0;
                st->theta = smax;
                st->shift = 0;
                st->prefmask = 0;
                st->done = 1;
                st->pending = 1;
                st->j = 1;
                st->batches++;
                mode = M_MARK_DIRECT;
                // the round after it too, if it needs one: its first batch is the second
                // largest stale key z, evaluated in the same step as if y wins
                const bool pair_ok = st->pair_penalty < kPairOff;
                if (!pair_ok) st->pair_penalty -= min(st->pair_penalty, kPairRetry);
                if (pair_ok && rd + 2 < st->round_end && nu > 3 && s2 > 0 && st->refresh_min > 3) {
                    batch[1] = (uint32_t)(mask - (s2 & mask));
                    fresh[1] = 0;
                    st->pair = 1;
                    st->pair_fail = 0;
                    st->pair_kz = s2;
                    mode = M_MARK_PAIR;
                }
            }
        }
    }
    st->cont = cont;
    st->mode = mode;
    set_step(st, hd, cont ? mode : M_NONE);
}


// plan_step by the last block of a launch: the state is copied to shared memory (its fields
// are read and written many times, one after the other), planned there and copied back.
// Every other block of the launch has finished, so nothing else touches the state meanwhile.
__device__ void plan_shared(SelState* st, uint32_t* __restrict__ batch, unsigned long long* __restrict__ fresh,
                            uint64_t* __restrict__ key, uint32_t* __restrict__ stamp, uint8_t* __restrict__ seedflag,
                            uint32_t* __restrict__ seed_list, uint64_t* __restrict__ gain_list,
                            uint64_t* __restrict__ round_evals, uint32_t n, uint32_t R, uint32_t bits,
                            const SelHandles& hd, bool have_count) {
    static_assert(offsetof(SelState, hist) % 8 == 0, "state copied in 8-byte words");
    constexpr uint32_t kWords = offsetof(SelState, hist) / 8;   // everything but the histogram
    __shared__ SelState ss;
    unsigned long long* g = reinterpret_cast<unsigned long long*>(st);
    unsigned long long* l = reinterpret_cast<unsigned long long*>(&ss);
    for (uint32_t i = threadIdx.x; i < kWords; i += blockDim.x) l[i] = __ldcg(g + i);
    __syncthreads();
    if (threadIdx.x == 0) plan_step(&ss, batch, fresh, key, stamp, seedflag, seed_list, gain_list, round_evals, n, R, bits, hd,
                                    have_count);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kWords; i += blockDim.x) g[i] = l[i];
}

// ---- BFS fallback: searches that outgrew the shared-memory queue ------------------------
// A search from v in sketch r with the queue and visited bitmap of a fallback slot (global
// memory: no size limit); the bitmap is cleared again before returning.
struct FbOut {
    uint32_t label, tail, seen, minv;
};

__device__ FbOut fb_search(const GraphView& g, const SketchView& s, uint32_t v, uint32_t r, bool want_seed,
                           uint32_t* __restrict__ q, uint32_t* __restrict__ bits) {
    const unsigned lane = threadIdx.x & 31;
    if (lane == 0) {
        q[0] = v;
        atomicOr(bits + (v >> 5), 1u << (v & 31));
    }
    __syncwarp();
    uint32_t head = 0, tail = 1, label = kNone, minv = v;
    uint32_t seen = want_seed ? (uint32_t)is_seed(s, v) : 0u;
    while (head < tail && label == kNone) {
        const uint32_t x = q[head++];
        const uint64_t a0 = g.off[x], a1 = g.off[x + 1];
        for (uint64_t base = a0; base < a1; base += 32) {
            const uint64_t a = base + lane;
            bool live = false;
            uint32_t y = 0, ci = 0;
            bool cen = false;
            if (a < a1) {
                const uint4 arc = g.arcs[a];
                y = arc.x & kArcIdMask;
                cen = arc.x >> 31;
                ci = arc.y;
                live = live_T_fast(((uint64_t)arc.w << 32) | arc.z, (uint64_t)(r + 1u) * kGamma,
                                   s.smp.aT ? s.smp.aT[a] : uniform_T(s.smp));
            }
            const unsigned cb = __ballot_sync(kFull, live && cen);
            if (cb) {
                const uint32_t c0 = __shfl_sync(kFull, ci, __ffs(cb) - 1);   // the arc's center index
                label = s.label[(size_t)c0 * s.R + r];
                break;
            }
            bool fresh_v = false;
            if (live) {
                const uint32_t bit = 1u << (y & 31);
                fresh_v = !(atomicOr(bits + (y >> 5), bit) & bit);
            }
            const unsigned nbm = __ballot_sync(kFull, fresh_v);
            if (fresh_v) {
                q[tail + __popc(nbm & ((1u << lane) - 1u))] = y;
                if (want_seed && is_seed(s, y)) seen = 1;
                minv = min(minv, y);
            }
            tail += __popc(nbm);
            __syncwarp();
        }
    }
    FbOut o;
    o.seen = __any_sync(kFull, seen) ? 1u : 0u;
#pragma unroll
    for (int d = 16; d; d >>= 1) minv = min(minv, __shfl_xor_sync(kFull, minv, d));
    for (uint32_t i = lane; i < tail; i += 32) bits[q[i] >> 5] = 0u;   // private slot
    __syncwarp();
    o.label = label;
    o.tail = tail;
    o.minv = minv;
    return o;
}

// Delta of one (candidate, sketch) from its search: the component's size unless a seed covers it.
__device__ __forceinline__ unsigned long long fb_delta(const SketchView& s, uint32_t r, const FbOut& o) {
    if (o.label != kNone) {
        const uint32_t sz = __ldcg(s.size + (size_t)o.label * s.R + r);   // a mark may precede it
        return (sz & kCovered) ? 0u : sz;
    }
    return o.seen ? 0u : o.tail;
}

// The queued fallback tasks, one warp per slot (`worker` of `nworkers`; slot = worker).
// FB_MARK_EVAL: MarkSeed of the winner f.v, then the Marginal of the candidate f.idx (batch
// slot 0), in order.
__device__ void fallback_run(const GraphView& g, const SketchView& s, SelState* st, const FbTask* __restrict__ fbt,
                             uint32_t fb_cap, uint32_t* __restrict__ fbq, uint32_t* __restrict__ fbb,
                             unsigned long long* __restrict__ fresh, uint64_t* __restrict__ spread_pairs,
                             uint32_t worker, uint32_t nworkers) {
    const unsigned lane = threadIdx.x & 31;
    const uint32_t ntask = min(__ldcg(&st->fb_n), fb_cap);
    const uint32_t n = g.n;
    const uint32_t nw = (n + 31) >> 5;
    uint32_t* q = fbq + (size_t)worker * n;
    uint32_t* bits = fbb + (size_t)worker * nw;
    for (uint32_t t = worker; t < ntask; t += nworkers) {
        const FbTask f = fbt[t];
        const uint32_t r = f.r;
        if (f.kind == FB_MARK_EVAL) {
            const FbOut a = fb_search(g, s, f.v, r, false, q, bits);
            if (lane == 0 && a.label != kNone) atomicOr(s.size + (size_t)a.label * s.R + r, kCovered);
            __syncwarp();
            SketchView sp = s;
            sp.pend = f.v;
            const FbOut b = fb_search(g, sp, f.idx, r, true, q, bits);
            if (lane == 0) {
                const unsigned long long d = fb_delta(sp, r, b);
                if (d) atomicAdd(fresh, d);
            }
            __syncwarp();
            continue;
        }
        const FbOut o = fb_search(g, s, f.v, r, f.kind == FB_EVAL, q, bits);
        if (lane == 0) {
            if (f.kind == FB_EVAL) {
                const unsigned long long d = fb_delta(s, r, o);
                if (d) atomicAdd(fresh + f.idx, d);
            } else if (f.kind == FB_MARK) {
                if (o.label != kNone) atomicOr(s.size + (size_t)o.label * s.R + r, kCovered);
            } else {
                uint64_t pr;
                if (o.label != kNone)
                    pr = ((uint64_t)o.label << 32) | (s.size[(size_t)o.label * s.R + r] & ~kCovered);
                else
                    pr = ((uint64_t)(kNoCenterTag | o.minv) << 32) | o.tail;
                spread_pairs[f.idx] = pr;
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32)
k_fallback(GraphView g, SketchView s, SelState* st, const FbTask* __restrict__ fbt, uint32_t fb_cap,
           uint32_t* __restrict__ fbq, uint32_t* __restrict__ fbb,
           unsigned long long* __restrict__ fresh, uint64_t* __restrict__ spread_pairs) {
    fallback_run(g, s, st, fbt, fb_cap, fbq, fbb, fresh, spread_pairs, blockIdx.x, gridDim.x);
}

// ---- the step kernel ----------------------------------------------------------------
// Everything one launch of k_sel_step needs.
struct StepArgs {
    GraphView g;
    SketchView s;
    SelState* st;
    uint64_t* key;
    uint32_t* stamp;
    uint8_t* seedflag;
    uint32_t* batch;
    unsigned long long* fresh;
    uint32_t* seed_list;
    uint64_t* gain_list;
    uint64_t* round_evals;
    const uint64_t* gain0;
    const uint64_t* spec_ov;
    FbTask* fbt;
    uint32_t* fbq;
    uint32_t* fbb;
    uint32_t fb_cap, fb_slots;
    uint32_t n, R, bits;
    uint64_t* topb;   // kTopB keys per block (PH_TOPB)
    uint32_t* pair_undo;   // [R]: the size row an M_MARK_PAIR step covered in each sketch, or kNone
    SelHandles hd;
};

union StepSmem {
    BlockSearchSmem bs;
    struct {
        unsigned int h[256];
        unsigned long long sfx[256];
    } sp;
    unsigned long long lists[kBlockWarps][kTopB];   // PH_TOPB: each warp's largest keys
};

// Block reduction (valid in thread 0): maxima of a and b, sums of c and e.
__device__ __forceinline__ void block_max_sum(unsigned long long& a, unsigned long long& b, unsigned long long& c,
                                              unsigned long long& e) {
    __shared__ unsigned long long s_a[8], s_b[8], s_c[8], s_e[8];
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        a = max(a, __shfl_xor_sync(kFull, a, d));
        b = max(b, __shfl_xor_sync(kFull, b, d));
        c += __shfl_xor_sync(kFull, c, d);
        e += __shfl_xor_sync(kFull, e, d);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_a[w] = a; s_b[w] = b; s_c[w] = c; s_e[w] = e; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            a = max(a, s_a[i]); b = max(b, s_b[i]); c += s_c[i]; e += s_e[i];
        }
    __syncthreads();
}

// The two largest of the block's (m1 >= m2) pairs; the result is valid in thread 0.
__device__ __forceinline__ void block_top2(unsigned long long& m1, unsigned long long& m2) {
    __shared__ unsigned long long s_1[8], s_2[8];
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(kFull, m1, d), o2 = __shfl_xor_sync(kFull, m2, d);
        m2 = max(min(m1, o1), max(m2, o2));
        m1 = max(m1, o1);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_1[w] = m1; s_2[w] = m2; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            m2 = max(min(m1, s_1[i]), max(m2, s_2[i]));
            m1 = max(m1, s_1[i]);
        }
    __syncthreads();
}

// f(v, seedflag[v], stamp[v], key[v]) for the candidates v assigned to thread t0 of nthr:
// four consecutive ids per iteration with one vector load per array, so that a thread has
// all its loads of an iteration in flight at once.
template <class F>
__device__ __forceinline__ void for_candidates(const StepArgs& a, uint32_t t0, uint32_t nthr, F f) {
    const uint32_t n4 = a.n >> 2;
    const uchar4* sf4 = reinterpret_cast<const uchar4*>(a.seedflag);
    const uint4* sp4 = reinterpret_cast<const uint4*>(a.stamp);
    const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(a.key);
    for (uint32_t i = t0; i < n4; i += nthr) {
        const uchar4 sf = sf4[i];
        const uint4 sp = sp4[i];
        const ulonglong2 ka = k2[2 * i], kb = k2[2 * i + 1];
        f(4 * i, sf.x, sp.x, ka.x);
        f(4 * i + 1, sf.y, sp.y, ka.y);
        f(4 * i + 2, sf.z, sp.z, kb.x);
        f(4 * i + 3, sf.w, sp.w, kb.y);
    }
    for (uint32_t v = 4 * n4 + t0; v < a.n; v += nthr) f(v, a.seedflag[v], a.stamp[v], a.key[v]);
}

// The reduction of a step over every candidate (Alg. 2's stale bound and stop test): best =
// max fresh key this round, stale_max / n_unev over the candidates not yet evaluated in it.
// With `finalize`, batch members awaiting their fresh key (stamp kPending, key = their batch
// slot) receive it here; otherwise an evaluation runs concurrently and they are skipped (the
// last block finalises them).  `skip` is a seed whose flag the step sets at its end, `skip2` a
// candidate evaluated ahead for the next round (left out).  With kTop2 (steps that evaluate a
// single candidate, which may close a round and open the next with a pair) the second largest
// stale key is kept too: a block's largest key m1 and second m2 go to stale_max and stale_2nd
// as old = atomicMax(stale_max, m1); atomicMax(stale_2nd, max(m2, min(old, m1))), which leaves
// the second largest of all keys in stale_2nd whatever the order of the blocks.
template <bool kTop2>
__device__ void scan_candidates(const StepArgs& a, bool finalize, uint32_t skip, uint32_t skip2, uint32_t t0,
                                uint32_t nthr) {
    SelState* st = a.st;
    const uint32_t round = st->round;
    const unsigned long long bp = st->best_prev;   // the best fresh key before this batch
    unsigned long long bf = 0, s1 = 0, s2 = 0, cnt = 0, above = 0, unused = 0;
    for_candidates(a, t0, nthr, [&](uint32_t v, uint8_t sf, uint32_t sp, unsigned long long k) {
        if (sf || v == skip || v == skip2) return;
        if (sp & kPending) {   // evaluated in this batch
            if (!finalize) return;
            k = pack_key(__ldcg(a.fresh + (uint32_t)k), v, a.bits);
            a.key[v] = k;
            a.stamp[v] = round;
            sp = round;
        }
        if (sp == round) {
            bf = max(bf, k);
        } else {
            if (kTop2) {
                if (k > s1) { s2 = s1; s1 = k; } else if (k > s2) { s2 = k; }
            } else {
                s1 = max(s1, k);
            }
            ++cnt;
            above += k > bp ? 1u : 0u;
        }
    });
    if (kTop2) block_top2(s1, s2);
    block_max_sum(bf, kTop2 ? unused : s1, cnt, above);
    if (threadIdx.x == 0) {
        if (bf) atomicMax(&st->best, bf);
        if (kTop2 && s1) {
            const unsigned long long old = atomicMax(&st->stale_max, s1);
            const unsigned long long sub = max(s2, min(old, s1));
            if (sub) atomicMax(&st->stale_2nd, sub);
        } else if (s1) {
            atomicMax(&st->stale_max, s1);
        }
        if (cnt) atomicAdd(&st->n_unev, cnt);
        if (above) atomicAdd(&st->above_bound, above);
    }
}

// scan_candidates over the whole grid
__device__ __forceinline__ void scan_all(const StepArgs& a, bool finalize, uint32_t skip) {
    scan_candidates<false>(a, finalize, skip, kNone, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Fresh keys of the batch members (last block, after the evaluation; every thread calls it).
__device__ void finalize_batch(const StepArgs& a) {
    SelState* st = a.st;
    const uint32_t round = st->round, bn = __ldcg(&st->batch_n);
    if (bn <= 32) {   // one warp, no block barrier
        if (threadIdx.x < 32) {
            unsigned long long k = 0;
            if (threadIdx.x < bn) {
                const uint32_t x = a.batch[threadIdx.x];
                k = pack_key(__ldcg(a.fresh + threadIdx.x), x, a.bits);
                a.key[x] = k;
                a.stamp[x] = round;
            }
#pragma unroll
            for (int d = 16; d; d >>= 1) k = max(k, __shfl_xor_sync(kFull, k, d));
            if (threadIdx.x == 0 && k) atomicMax(&st->best, k);
        }
        return;
    }
    unsigned long long bf = 0, unused_b = 0, unused_c = 0, unused_e = 0;
    for (uint32_t j = threadIdx.x; j < bn; j += blockDim.x) {
        const uint32_t x = a.batch[j];
        const unsigned long long k = pack_key(__ldcg(a.fresh + j), x, a.bits);
        a.key[x] = k;
        a.stamp[x] = round;
        bf = max(bf, k);
    }
    block_max_sum(bf, unused_b, unused_c, unused_e);
    if (threadIdx.x == 0 && bf) atomicMax(&st->best, bf);
}

// MarkSeed (Alg. 3): in every sketch, flag the component of the last round's winner as
// covered.  One block per sketch (a single vertex is marked per round, so latency, not
// total work, decides); labels the winner's evaluation already found are reused.
__device__ __forceinline__ uint32_t mark_label(const GraphView& g, const SketchView& s, uint32_t sd, uint32_t r,
                                               BlockSearchSmem& sm, SelState* st, bool* overflow) {
    *overflow = false;
    if (is_center(s, sd)) return s.label[(size_t)center_index(s, sd) * s.R + r];
    // a label found when sd was evaluated is still valid: labels depend on the sketch only
    const uint64_t e = s.labcache[(size_t)(sd & (kLabSlots - 1)) * s.R + r];
    if ((uint32_t)(e >> 32) == sd) return (uint32_t)e;
    const BfsOut o = block_search(g, s, sd, r, false, sm, st);   // block-uniform branch
    *overflow = o.overflow;
    return o.label;
}

__device__ void mark_tasks(const StepArgs& a, BlockSearchSmem& sm) {
    const uint32_t sd = a.st->sd;
    for (uint32_t r = blockIdx.x; r < a.R; r += gridDim.x) {   // uniform over the block
        bool over = false;
        const uint32_t l = mark_label(a.g, a.s, sd, r, sm, a.st, &over);
        if (threadIdx.x == 0) {
            if (over) push_fallback(a.st, a.fbt, a.fb_cap, sd, r, FB_MARK, 0);
            else if (l != kNone) atomicOr(a.s.size + (size_t)l * a.R + r, kCovered);
        }
        __syncthreads();
    }
}

constexpr uint32_t kLabelOverflow = 0xFFFFFFFEu;   // a search outgrew its queue (labels are < n)

// Marginal (Alg. 3) of a candidate in one sketch by a whole block; adds it to fresh[j].  With
// label_out, thread 0 also stores the component's label there (kNone: no center,
// kLabelOverflow: the search overflowed).  An `ahead` evaluation (M_MARK_PAIR's z) queues no
// fallback search: an overflow voids it.
__device__ void marginal_block(const StepArgs& a, const SketchView& s, uint32_t x, uint32_t r, uint32_t j,
                               BlockSearchSmem& sm, bool ahead = false, uint32_t* label_out = nullptr) {
    unsigned long long d = 0;
    if (is_center(s, x)) {
        const uint32_t l = s.label[(size_t)center_index(s, x) * s.R + r];
        const uint32_t sz = __ldcg(s.size + (size_t)l * s.R + r);
        d = (sz & kCovered) ? 0u : sz;
        if (threadIdx.x == 0 && label_out) *label_out = l;
    } else {
        const BfsOut o = block_search(a.g, s, x, r, true, sm, a.st);
        if (threadIdx.x == 0) {
            if (label_out) *label_out = o.overflow ? kLabelOverflow : o.label;
            if (!o.overflow)
                s.labcache[(size_t)(x & (kLabSlots - 1)) * s.R + r] = ((uint64_t)x << 32) | o.label;
            if (o.overflow) {
                if (ahead) a.st->pair_fail = 1;
                else push_fallback(a.st, a.fbt, a.fb_cap, x, r, FB_EVAL, j);
            } else if (o.label != kNone) {
                const uint32_t sz = __ldcg(s.size + (size_t)o.label * s.R + r);
                d = (sz & kCovered) ? 0u : sz;
            } else {
                d = o.seen ? 0u : o.count;
            }
        }
    }
    if (threadIdx.x == 0 && d) atomicAdd(a.fresh + j, d);
}

// Marginal for small batches: one block per (member j, sketch r), so that a round that
// re-evaluates a handful of vertices finishes in the latency of one search, the block's warps
// sharing the member's first hop (block_search).
__device__ void eval_tasks(const StepArgs& a, BlockSearchSmem& sm) {
    const unsigned long long total = (unsigned long long)__ldcg(&a.st->batch_n) * a.R;
    for (unsigned long long t = blockIdx.x; t < total; t += gridDim.x) {   // uniform over the block
        const uint32_t j = (uint32_t)(t / a.R), r = (uint32_t)(t % a.R);
        marginal_block(a, a.s, a.batch[j], r, j, sm);
        __syncthreads();
    }
}

// MarkSeed of the last round's winner x fused with the Marginal of this round's only
// candidate y (batch slot 0), one block per sketch: the block marks x's component first, so
// that y's search finds it covered; a component without a center that holds x counts as
// holding a seed through s.pend (x's flag is set at the end of the step).  If x's search
// overflows, the fallback does both for that sketch (FB_MARK_EVAL), in the same order.
__device__ void mark_eval_tasks(const StepArgs& a, BlockSearchSmem& sm) {
    __shared__ int s_marked;
    __shared__ uint32_t s_ly;
    const uint32_t x = a.st->sd, y = a.batch[0];
    const bool pair = a.st->pair != 0;
    SketchView s = a.s;
    s.pend = x;
    SketchView s2 = s;   // z's searches: x and y are seeds
    s2.pend2 = y;
    for (uint32_t r = blockIdx.x; r < a.R; r += gridDim.x) {   // uniform over the block
        bool over = false;
        const uint32_t lx = mark_label(a.g, s, x, r, sm, a.st, &over);
        if (threadIdx.x == 0) {
            s_marked = !over;
            s_ly = kLabelOverflow;
            if (over) push_fallback(a.st, a.fbt, a.fb_cap, x, r, FB_MARK_EVAL, y);
            else if (lx != kNone) atomicOr(s.size + (size_t)lx * s.R + r, kCovered);
        }
        __syncthreads();
        if (s_marked) marginal_block(a, s, y, r, 0, sm, false, pair ? &s_ly : nullptr);
        __syncthreads();
        if (!pair) continue;
        // M_MARK_PAIR: MarkSeed(y) here as if y wins (recorded, to be undone if it loses), then
        // z's Marginal; a sketch whose y search went to the fallback voids z's evaluation
        if (threadIdx.x == 0) {
            const uint32_t ly = s_ly;
            uint32_t undo = kNone;
            if (ly == kLabelOverflow) {
                a.st->pair_fail = 1;
            } else if (ly != kNone) {
                const uint32_t old = atomicOr(s.size + (size_t)ly * s.R + r, kCovered);
                if (!(old & kCovered)) undo = ly;
            }
            a.pair_undo[r] = undo;
            s_marked = ly != kLabelOverflow;
        }
        __syncthreads();
        if (s_marked) marginal_block(a, s2, a.batch[1], r, 1, sm, true, nullptr);
        __syncthreads();
    }
}

// Marginal(x | {s0}) = gain0(x) - sum_r |C_r(x)| [s0 in C_r(x)] for every batch member (round
// 1 after a candidate first seed s0).
__device__ void spec_eval_tasks(const StepArgs& a) {
    const uint32_t bn = __ldcg(&a.st->batch_n);
    const uint64_t* ov = a.spec_ov + (size_t)a.st->spec_idx * a.n;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < bn; j += gridDim.x * blockDim.x) {
        const uint32_t x = a.batch[j];
        a.fresh[j] = a.gain0[x] - ov[x];
    }
}

// Unevaluated candidates whose stale key beats the best fresh key of the round: an upper
// bound on what is left to evaluate in this round (the winner's fresh key is >= best).
__device__ void count_above_tasks(const StepArgs& a) {
    SelState* st = a.st;
    const unsigned long long best = st->best;
    // only needed when the round goes on (the next batch's size depends on it)
    const bool need = st->n_unev > 0 && best <= st->stale_max && best;
    const uint32_t round = st->round;
    unsigned long long cnt = 0, unused_a = 0, unused_b = 0, unused_e = 0;
    if (need)
        for_candidates(a, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
                       [&](uint32_t, uint8_t sf, uint32_t sp, unsigned long long k) {
                           if (!sf && sp != round && k > best) ++cnt;
                       });
    block_max_sum(unused_a, unused_b, cnt, unused_e);
    if (threadIdx.x == 0 && cnt) atomicAdd(&st->count_above, cnt);
}

// One radix pass over the unevaluated candidates: block histograms of the next key byte,
// added to st->hist; the last block picks the byte (sel_pass_pick).
__device__ void sel_pass_tasks(const StepArgs& a, StepSmem& sm) {
    SelState* st = a.st;
    const uint32_t round = st->round;
    unsigned int* h = sm.sp.h;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix, pm = st->prefmask;
    const int shift = st->shift;
    for_candidates(a, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
                   [&](uint32_t, uint8_t sf, uint32_t sp, unsigned long long k) {
                       if (!sf && sp != round && (k & pm) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
                   });
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

// Last block of a pass: either fix the threshold theta (batch between B and 2B, or exact at
// the last byte) or narrow the prefix for the next pass.
__device__ void sel_pass_pick(SelState* st, StepSmem& sm) {
    __shared__ unsigned long long s_wsum[8];
    __shared__ int s_d;
    unsigned long long* sfx = sm.sp.sfx;   // sfx[d]: candidates whose byte is >= d
    const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;   // blockDim.x == 256
    unsigned long long x = __ldcg(&st->hist[tid]);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {   // suffix sum within the warp
        const unsigned long long y = __shfl_down_sync(kFull, x, d);
        if (lane + d < 32) x += y;
    }
    if (lane == 0) s_wsum[warp] = x;
    if (tid == 0) s_d = 0;
    __syncthreads();
    for (unsigned w = warp + 1; w < 8; ++w) x += s_wsum[w];
    sfx[tid] = x;
    st->hist[tid] = 0;
    __syncthreads();
    const unsigned long long need = st->need;
    // the highest bin whose suffix reaches need (suffixes fall with the bin; bin 0 if none)
    if (x >= need && (tid == 255 || sfx[tid + 1] < need)) s_d = (int)tid;
    __syncthreads();
    if (tid == 0) {
        const int d = s_d;
        const unsigned long long above = (d < 255) ? sfx[d + 1] : 0ull;
        const unsigned long long with_bin = st->taken + sfx[d];
        if (with_bin <= 2 * st->borig || st->shift == 0) {
            st->theta = st->prefix | ((unsigned long long)d << st->shift);
            st->done = 1;
        } else {
            st->taken += above;
            st->need -= above;
            st->prefix |= (unsigned long long)d << st->shift;
            st->prefmask |= 255ull << st->shift;
            st->shift -= 8;
        }
    }
}

// The batch: every unevaluated candidate with a stale key >= theta (and above the best fresh
// key: one below it cannot win, keys being distinct).
__device__ void gather_tasks(const StepArgs& a) {
    SelState* st = a.st;
    const uint32_t round = st->round;
    const unsigned long long bp = st->best_prev;
    const unsigned long long theta = max(st->theta, bp ? bp + 1 : 0ull);
    const unsigned lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x * 4;
    // the loop bound is uniform over the warp: lanes cover ids base + 4 lane .. + 3
    for (uint32_t base = (blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) * 4; base < a.n; base += stride) {
        const uint32_t v0 = base + 4 * lane;
        uint32_t take = 0;   // bit e: candidate v0 + e joins the batch
        if (v0 + 3 < a.n) {
            const uchar4 sf = reinterpret_cast<const uchar4*>(a.seedflag)[v0 >> 2];
            const uint4 sp = reinterpret_cast<const uint4*>(a.stamp)[v0 >> 2];
            const ulonglong2 ka = reinterpret_cast<const ulonglong2*>(a.key)[v0 >> 1];
            const ulonglong2 kb = reinterpret_cast<const ulonglong2*>(a.key)[(v0 >> 1) + 1];
            take = (!sf.x && sp.x != round && ka.x >= theta ? 1u : 0u) | (!sf.y && sp.y != round && ka.y >= theta ? 2u : 0u) |
                   (!sf.z && sp.z != round && kb.x >= theta ? 4u : 0u) | (!sf.w && sp.w != round && kb.y >= theta ? 8u : 0u);
        } else {
            for (uint32_t e = 0; e < 4; ++e) {
                const uint32_t v = v0 + e;
                if (v < a.n && !a.seedflag[v] && a.stamp[v] != round && a.key[v] >= theta) take |= 1u << e;
            }
        }
        const uint32_t cnt = __popc(take);
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if ((int)lane >= d) incl += y;
        }
        const uint32_t wtot = __shfl_sync(kFull, incl, 31);
        if (!wtot) continue;
        uint32_t pos0 = 0;
        if (lane == 31) pos0 = atomicAdd(&st->batch_n, wtot);
        uint32_t j = __shfl_sync(kFull, pos0, 31) + incl - cnt;
        for (uint32_t t = take; t; t &= t - 1) {
            const uint32_t v = v0 + __ffs(t) - 1;
            a.batch[j] = v;
            a.fresh[j] = 0;
            a.key[v] = j;                      // its batch slot, until its fresh key
            a.stamp[v] = round | kPending;
            ++j;
        }
    }
}

// ---- PH_TOPB: the largest stale keys in one pass -------------------------------------
// A warp keeps the `want` (<= kTopB) largest keys seen so far sorted in its first lanes (lane
// i: the i-th largest; 0 = empty, every real key is >= 1).  A key above the list's last one
// is inserted at its rank, the entries below moving down one lane (lanes >= want hold no
// information).
__device__ __forceinline__ void warp_insert(unsigned long long& L, unsigned long long k, uint32_t want) {
    const unsigned lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(kFull, k > __shfl_sync(kFull, L, want - 1));
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const unsigned long long x = __shfl_sync(kFull, k, src);
        if (x <= __shfl_sync(kFull, L, want - 1)) continue;   // pushed out by the keys before it
        const int pos = __popc(__ballot_sync(kFull, L > x));
        const unsigned long long up = __shfl_up_sync(kFull, L, 1);
        if ((int)lane > pos) L = up;
        else if ((int)lane == pos) L = x;
    }
}

// The 8 lists of the block merged into warp 0's (every warp calls it).
__device__ __forceinline__ unsigned long long block_merge(unsigned long long L, uint32_t want, StepSmem& sm) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    sm.lists[warp][lane] = lane < want ? L : 0ull;
    __syncthreads();
    if (warp == 0)
        for (int w = 1; w < kBlockWarps; ++w) warp_insert(L, sm.lists[w][lane], want);
    __syncthreads();
    return L;
}

// Every block: its `want` largest eligible keys (unevaluated, above the best fresh key) into
// topb[block]; 4 consecutive candidates per lane and iteration (vector loads), skipped with
// one ballot when none of them beats the warp's last kept key.
__device__ void topb_tasks(const StepArgs& a, StepSmem& sm) {
    const SelState* st = a.st;
    const uint32_t round = st->round, want = st->topb;
    const unsigned long long bp = st->best_prev;
    const unsigned long long lo = bp ? bp + 1 : 1ull;
    const unsigned lane = threadIdx.x & 31;
    unsigned long long L = 0;
    const uint32_t stride = gridDim.x * blockDim.x * 4;
    for (uint32_t base = (blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) * 4; base < a.n; base += stride) {
        const uint32_t v0 = base + 4 * lane;   // the loop bound is uniform over the warp
        unsigned long long k[4] = {0, 0, 0, 0};
        if (v0 + 3 < a.n) {
            const uchar4 sf = reinterpret_cast<const uchar4*>(a.seedflag)[v0 >> 2];
            const uint4 sp = reinterpret_cast<const uint4*>(a.stamp)[v0 >> 2];
            const ulonglong2 ka = reinterpret_cast<const ulonglong2*>(a.key)[v0 >> 1];
            const ulonglong2 kb = reinterpret_cast<const ulonglong2*>(a.key)[(v0 >> 1) + 1];
            k[0] = (!sf.x && sp.x != round && ka.x >= lo) ? ka.x : 0;
            k[1] = (!sf.y && sp.y != round && ka.y >= lo) ? ka.y : 0;
            k[2] = (!sf.z && sp.z != round && kb.x >= lo) ? kb.x : 0;
            k[3] = (!sf.w && sp.w != round && kb.y >= lo) ? kb.y : 0;
        } else {
            for (uint32_t e = 0; e < 4; ++e) {
                const uint32_t v = v0 + e;
                if (v < a.n && !a.seedflag[v] && a.stamp[v] != round && a.key[v] >= lo) k[e] = a.key[v];
            }
        }
        const unsigned long long kmax = max(max(k[0], k[1]), max(k[2], k[3]));
        if (!__any_sync(kFull, kmax > __shfl_sync(kFull, L, want - 1))) continue;
#pragma unroll
        for (int e = 0; e < 4; ++e) warp_insert(L, k[e], want);
    }
    L = block_merge(L, want, sm);
    if ((threadIdx.x >> 5) == 0) a.topb[(size_t)blockIdx.x * kTopB + lane] = lane < want ? L : 0ull;
}

// Last block: the grid's lists merged (the first `want` entries of each); the largest become
// the batch.
__device__ void topb_pick(const StepArgs& a, StepSmem& sm) {
    SelState* st = a.st;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t want = st->topb, round = st->round;
    unsigned long long L = 0;
    // entry (block b, rank i < want) at b * kTopB + i: each warp takes blocks warp, warp + 8, ...
    // 32 / want of them per step
    const uint32_t per = kTopB / want;   // blocks per 32 lanes (want is at most kTopB)
    for (uint32_t b0 = warp * per; b0 < gridDim.x; b0 += kBlockWarps * per) {   // uniform over the warp
        const uint32_t b = b0 + lane / want, i = lane % want;
        warp_insert(L, (lane < per * want && b < gridDim.x) ? __ldcg(a.topb + (size_t)b * kTopB + i) : 0ull, want);
    }
    L = block_merge(L, want, sm);
    if (warp == 0) {
        const uint64_t mask = (1ull << a.bits) - 1ull;
        const bool take = lane < want && L != 0;
        if (take) {
            const uint32_t v = (uint32_t)(mask - (L & mask));
            a.batch[lane] = v;
            a.fresh[lane] = 0;
            a.key[v] = lane;                       // its batch slot, until its fresh key
            a.stamp[v] = round | kPending;
        }
        const unsigned cnt = __popc(__ballot_sync(kFull, take));
        if (lane == 0) st->batch_n = cnt;
    }
}

// One phase of the selection per launch (SelState::phase); the last block to finish runs the
// phase's epilogue: the radix pick, the next phase, or -- after an evaluation -- the queued
// fallback searches, the batch's fresh keys, MarkSeed's flag and the plan of the next step
// (plan_step).  The grid is fixed (about the resident blocks); phases stride over their work.
__global__ void __launch_bounds__(kBlockWarps * 32)
k_sel_step(StepArgs a) {
    __shared__ StepSmem sm;
    __shared__ unsigned int s_last;
    SelState* st = a.st;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->launches, 1ull);
    const unsigned phase = st->phase;
    if (phase == PH_NONE) return;
    const bool marking = phase == PH_MARK || phase == PH_MARK_EVAL;
    // evaluation phases: if enough blocks are left over, blocks [0, ntask) search (one task
    // each) while the others scan the candidates; else, or when every task is a lookup (the
    // vertices are centers or hubs: no search), every block scans after its tasks
    const unsigned long long ntask = phase == PH_EVAL ? (unsigned long long)__ldcg(&st->batch_n) * a.R : a.R;
    bool lookups = false;
    if (phase == PH_MARK) lookups = is_center(a.s, st->sd);
    else if (phase == PH_MARK_EVAL)
        lookups = is_center(a.s, st->sd) && is_center(a.s, a.batch[0]) && (!st->pair || is_center(a.s, a.batch[1]));
    else if (phase == PH_EVAL) lookups = __ldcg(&st->batch_n) == 1 && is_center(a.s, a.batch[0]);
    const uint32_t free0 = (!lookups && ntask + 64 <= gridDim.x) ? (uint32_t)ntask : 0u;
    const bool scanner = blockIdx.x >= free0;
    const uint32_t t0 = (blockIdx.x - (scanner ? free0 : 0u)) * blockDim.x + threadIdx.x;
    const uint32_t nthr = (gridDim.x - free0) * blockDim.x;
    switch (phase) {
    case PH_SCAN: scan_all(a, true, kNone); break;
    case PH_MARK:
        if (!free0 || !scanner) mark_tasks(a, sm.bs);
        if (scanner) scan_candidates<false>(a, false, st->sd, kNone, t0, nthr);
        break;
    case PH_MARK_EVAL:
        if (!free0 || !scanner) mark_eval_tasks(a, sm.bs);
        if (scanner) scan_candidates<true>(a, false, st->sd, st->pair ? a.batch[1] : kNone, t0, nthr);
        break;
    case PH_EVAL:
        if (!free0 || !scanner) eval_tasks(a, sm.bs);
        if (scanner) {
            if (__ldcg(&st->batch_n) == 1) scan_candidates<true>(a, false, kNone, kNone, t0, nthr);
            else scan_candidates<false>(a, false, kNone, kNone, t0, nthr);
        }
        break;
    case PH_SEL_PASS: sel_pass_tasks(a, sm); break;
    case PH_GATHER: gather_tasks(a); break;
    case PH_TOPB: topb_tasks(a, sm); break;
    case PH_SPEC_EVAL: spec_eval_tasks(a); break;
    case PH_COUNT: count_above_tasks(a); break;
    default: break;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) st->ticket = 0;
    switch (phase) {
    case PH_SEL_PASS:
        sel_pass_pick(st, sm);
        if (threadIdx.x == 0) st->phase = st->done ? PH_GATHER : PH_SEL_PASS;
        return;
    case PH_TOPB:
        topb_pick(a, sm);
        if (threadIdx.x == 0) st->phase = (st->mode == M_SPEC_GATHER || st->mode == M_SPEC_HIST) ? PH_SPEC_EVAL : PH_EVAL;
        return;
    case PH_GATHER:
        if (threadIdx.x == 0) {
            const unsigned mode = st->mode;
            if (mode == M_GATHER_CHUNK || mode == M_HIST_CHUNK) set_rare(st, a.hd, RARE_CHUNK);
            else if (mode == M_REFRESH) set_rare(st, a.hd, RARE_REFRESH);
            else if (mode == M_SPEC_GATHER || mode == M_SPEC_HIST) st->phase = PH_SPEC_EVAL;
            else st->phase = PH_EVAL;
        }
        return;
    case PH_SPEC_EVAL:
        if (threadIdx.x == 0) st->phase = PH_SCAN;
        return;
    default: break;
    }
    if (phase == PH_MARK || phase == PH_MARK_EVAL || phase == PH_EVAL) {
        // searches that outgrew the shared queue, one warp per fallback slot
        if (__ldcg(&st->fb_n)) {
            const uint32_t nwk = min((uint32_t)(blockDim.x >> 5), a.fb_slots);
            if ((threadIdx.x >> 5) < nwk)
                fallback_run(a.g, a.s, st, a.fbt, a.fb_cap, a.fbq, a.fbb, a.fresh, nullptr, threadIdx.x >> 5, nwk);
            __threadfence();
            __syncthreads();
        }
        if (phase != PH_MARK) finalize_batch(a);
        if (marking && threadIdx.x == 0) {
            a.seedflag[st->sd] = 1;
            a.key[st->sd] = 0;
        }
        // M_MARK_PAIR: if y lost its round (its fresh key is not above z's stale key), the
        // MarkSeed(y) the step applied is undone (plan_step resolves the rest)
        if (phase == PH_MARK_EVAL && st->pair) {
            const unsigned long long fy = pack_key(__ldcg(a.fresh), a.batch[0], a.bits);
            if (fy <= st->pair_kz)
                for (uint32_t r = threadIdx.x; r < a.R; r += blockDim.x) {
                    const uint32_t l = a.pair_undo[r];
                    if (l != kNone) atomicAnd(a.s.size + (size_t)l * a.R + r, ~kCovered);
                }
        }
    }
    __threadfence();
    __syncthreads();
    plan_shared(st, a.batch, a.fresh, a.key, a.stamp, a.seedflag, a.seed_list, a.gain_list, a.round_evals, a.n, a.R,
                a.bits, a.hd, phase == PH_COUNT);
}

// The reduction and plan after an evaluator outside k_sel_step (PH_SCAN's work as a kernel).
__global__ void __launch_bounds__(256)
k_reduce_plan(StepArgs a) {
    __shared__ unsigned int s_last;
    SelState* st = a.st;
    scan_all(a, true, kNone);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) st->ticket = 0;
    __syncthreads();
    plan_shared(st, a.batch, a.fresh, a.key, a.stamp, a.seedflag, a.seed_list, a.gain_list, a.round_evals, a.n, a.R,
                a.bits, a.hd, false);
}

// Candidate first seeds of this build.
__global__ void k_spec_init(SelState* st, const uint32_t* __restrict__ ids, uint32_t count) {
    if (threadIdx.x == 0) {
        st->spec_count = count;
        st->spec_idx = kNone;
        for (uint32_t k = 0; k < count; ++k) st->spec_ids[k] = ids[k];
    }
}

// Before a selection run: the number of seeds to reach and the refresh threshold.
__global__ void k_set_target(SelState* st, uint32_t round_end, unsigned long long refresh_min) {
    if (threadIdx.x == 0) {
        st->round_end = round_end;
        st->refresh_min = refresh_min;
    }
}

// First node of a selection run: open a round (PH_SCAN) if seeds are missing.
__global__ void k_sel_begin(SelState* st, SelHandles hd) {
    if (threadIdx.x == 0) {
        const unsigned go = (!st->err && st->round < st->round_end) ? 1u : 0u;
        st->launches += 1;
        st->phase = go ? PH_SCAN : PH_NONE;
        st->rare = RARE_NONE;
        if (hd.on) {   // every launch of the graph starts from these values
            cudaGraphSetConditional(hd.outer, go);
            cudaGraphSetConditional(hd.inner, go);
            cudaGraphSetConditional(hd.rare, RARE_NONE);
            st->cond[0] = go;
            st->cond[1] = go;
            st->cond[2] = RARE_NONE;
        }
    }
}

__global__ void k_phase_reset(SelState* st) {
    if (threadIdx.x == 0) { st->fb_n = 0; st->eval_next = 0; st->batch_n = 0; }
}

// Marginal (Alg. 3) of every batch member: tasks (member j, chunk of 32 sketches).
__global__ void __launch_bounds__(kEvalWarps * 32)
k_eval(GraphView g, SketchView s, SelState* st, const uint32_t* __restrict__ batch,
       unsigned long long* __restrict__ fresh, FbTask* __restrict__ fbt, uint32_t fb_cap,
       uint32_t nchunk) {
    __shared__ uint32_t qls[kEvalWarps][32 * kLaneQ];
    __shared__ uint32_t qws[kEvalWarps][kQcap + kHashSlots];
    uint32_t* ql = qls[threadIdx.x >> 5];
    uint32_t* qw = qws[threadIdx.x >> 5];
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long total = (unsigned long long)st->batch_n * nchunk;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&st->eval_next, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t >= total) break;
        const uint32_t j = (uint32_t)(t / nchunk), ch = (uint32_t)(t % nchunk);
        const uint32_t x = batch[j];
        const uint32_t r_lo = ch * 32, r_hi = min(s.R, r_lo + 32);
        const uint32_t r = r_lo + lane;
        unsigned long long d = 0;
        if (is_center(s, x)) {
            if (r < r_hi) {
                const uint32_t l = s.label[(size_t)center_index(s, x) * s.R + r];
                const uint32_t sz = s.size[(size_t)l * s.R + r];
                d = (sz & kCovered) ? 0u : sz;
            }
        } else {
            const LaneRes o = get_center_32(g, s, x, r_lo, r_hi, ql, qw, true, st);
            if (r < r_hi && !o.overflow)
                s.labcache[(size_t)(x & (kLabSlots - 1)) * s.R + r] = ((uint64_t)x << 32) | o.label;
            if (r < r_hi) {
                if (o.overflow) {
                    push_fallback(st, fbt, fb_cap, x, r, FB_EVAL, j);
                } else if (o.label != kNone) {
                    const uint32_t sz = s.size[(size_t)o.label * s.R + r];
                    d = (sz & kCovered) ? 0u : sz;
                } else {
                    d = o.seen ? 0u : o.count;
                }
            }
        }
        const unsigned long long sum = warp_sum_u64(d);
        if (lane == 0 && sum) atomicAdd(fresh + j, sum);
    }
}

// Marginal for small batches: one block per (member j, sketch r), so that a round that
// re-evaluates a handful of vertices finishes in the latency of one search, the block's warps

// ---- spread: per (seed i, sketch r) the component's identity and size, then dedup -----
__global__ void __launch_bounds__(kEvalWarps * 32)
k_spread_tasks(GraphView g, SketchView s, SelState* st, const uint32_t* __restrict__ sd, uint32_t k,
               uint32_t nchunk, FbTask* __restrict__ fbt, uint32_t fb_cap,
               uint64_t* __restrict__ pairs) {
    __shared__ uint32_t qls[kEvalWarps][32 * kLaneQ];
    __shared__ uint32_t qws[kEvalWarps][kQcap + kHashSlots];
    uint32_t* ql = qls[threadIdx.x >> 5];
    uint32_t* qw = qws[threadIdx.x >> 5];
    const unsigned lane = threadIdx.x & 31;
    const uint64_t total = (uint64_t)k * nchunk;
    const uint64_t wstride = (uint64_t)gridDim.x * kEvalWarps;
    for (uint64_t t = (uint64_t)blockIdx.x * kEvalWarps + (threadIdx.x >> 5); t < total; t += wstride) {
        const uint32_t i = (uint32_t)(t / nchunk), ch = (uint32_t)(t % nchunk);
        const uint32_t x = sd[i];
        const uint32_t r_lo = ch * 32, r_hi = min(s.R, r_lo + 32);
        const uint32_t r = r_lo + lane;
        const size_t idx = (size_t)r * k + i;
        if (is_center(s, x)) {
            if (r < r_hi) {
                const uint32_t l = s.label[(size_t)center_index(s, x) * s.R + r];
                const uint32_t sz = s.size[(size_t)l * s.R + r] & ~kCovered;
                pairs[idx] = ((uint64_t)l << 32) | sz;
            }
        } else {
            const LaneRes o = get_center_32(g, s, x, r_lo, r_hi, ql, qw, false, st);
            if (r < r_hi) {
                if (o.overflow) {
                    push_fallback(st, fbt, fb_cap, x, r, FB_SPREAD, (uint32_t)idx);
                } else if (o.label != kNone) {
                    pairs[idx] = ((uint64_t)o.label << 32) | (s.size[(size_t)o.label * s.R + r] & ~kCovered);
                } else {
                    pairs[idx] = ((uint64_t)(kNoCenterTag | o.minv) << 32) | o.count;
                }
            }
        }
    }
}

// one block per sketch: sort the k (component id, size) words, add sizes of distinct ones
__global__ void __launch_bounds__(1024)
k_spread_dedup(const uint64_t* __restrict__ pairs, uint32_t k, uint32_t kp2,
               unsigned long long* __restrict__ total) {
    extern __shared__ uint64_t sv[];
    const uint64_t* row = pairs + (size_t)blockIdx.x * k;
    for (uint32_t i = threadIdx.x; i < kp2; i += blockDim.x) sv[i] = i < k ? row[i] : ~0ull;
    __syncthreads();
    for (uint32_t len = 2; len <= kp2; len <<= 1) {
        for (uint32_t stp = len >> 1; stp > 0; stp >>= 1) {
            for (uint32_t i = threadIdx.x; i < kp2; i += blockDim.x) {
                const uint32_t jx = i ^ stp;
                if (jx > i) {
                    const bool up = (i & len) == 0;
                    const uint64_t a = sv[i], b = sv[jx];
                    if ((a > b) == up) { sv[i] = b; sv[jx] = a; }
                }
            }
            __syncthreads();
        }
    }
    unsigned long long acc = 0;
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x)
        if (i == 0 || sv[i] != sv[i - 1]) acc += sv[i] & 0xFFFFFFFFull;
    acc = warp_sum_u64(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

GraphView graph_view(const im_ctx* c) {
    GraphView g;
    g.n = c->n; g.m = c->m; g.edges = c->d_edges; g.off = c->d_off; g.arcs = c->d_arcs;
    g.ccnt = c->d_arc_cur;   // the arc fill's front cursors: arcs to centers per vertex
    return g;
}

SketchView sketch_view(const im_ctx* c) {
    SketchView s;
    s.R = c->R; s.rho = c->rho; s.all_centers = c->all_centers;
    s.cbits = c->d_cbits; s.cidx = c->d_cidx; s.label = c->d_label; s.size = c->d_size;
    s.seed_flag = c->d_seedflag; s.labcache = c->d_labcache; s.smp = c->smp;
    s.pend = kNone;
    s.pend2 = kNone;
    return s;
}

StepArgs step_args(const im_ctx* c, const SelHandles& hd) {
    StepArgs a;
    a.g = graph_view(c);
    a.s = sketch_view(c);
    a.st = c->d_sel;
    a.key = c->d_key; a.stamp = c->d_stamp; a.seedflag = c->d_seedflag;
    a.batch = c->d_batch; a.fresh = (unsigned long long*)c->d_fresh;
    a.seed_list = c->d_seed_list; a.gain_list = c->d_gain_list; a.round_evals = c->d_round_evals;
    a.gain0 = c->d_gain0; a.spec_ov = c->lane[0].spec_ov;
    a.fbt = c->d_fb_tasks; a.fbq = c->d_fb_queue; a.fbb = c->d_fb_bits;
    a.fb_cap = c->fb_cap;
    a.fb_slots = (c->all_centers || !c->d_fb_queue) ? 0u : c->fb_slots;
    a.n = c->n; a.R = c->R; a.bits = c->key_bits;
    a.topb = c->d_topb;
    a.pair_undo = c->d_pair_undo;
    a.hd = hd;
    return a;
}

// copy the device state to the pinned mirror and wait
int pull_state(im_ctx* c) {
    IM_CUDA(c, cudaMemcpyAsync(c->h_sel, c->d_sel, sizeof(SelState), cudaMemcpyDeviceToHost, c->stream));
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    return IM_OK;
}

int sync_state(im_ctx* c) {
    IM_CUDA(c, cudaMemcpyAsync(c->h_sel, c->d_sel, sizeof(SelState), cudaMemcpyDeviceToHost, c->stream));
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->h_sel->fb_overflow) return im_fail(c, IM_EDEVICE, "BFS fallback queue capacity exceeded");
    if (c->h_sel->err) return im_fail(c, IM_EDEVICE, "selection kernel reported an error");
    return IM_OK;
}

void launch_fallback(im_ctx* c, const GraphView& g, const SketchView& s) {
    if (c->all_centers || c->fb_slots == 0) return;
    IM_LAUNCH(c, K_FALLBACK, k_fallback, c->fb_slots, 32, 0, g, s, c->d_sel, c->d_fb_tasks, c->fb_cap,
              c->d_fb_queue, c->d_fb_bits, (unsigned long long*)c->d_fresh, c->d_spread_pairs);
}

unsigned search_grid(uint64_t tasks) {
    return grid_for(tasks, kEvalWarps, 152u * 16u);   // one task per warp to start
}

}  // namespace

// Reset the selection state: keys from the initial gains, no seeds, no coverage.  Right after
// a build every size entry was just written without its covered bit (fresh = true), so only
// a reset of an earlier selection clears the bits.
int im_selection_init(im_ctx* c, bool fresh) {
    const unsigned T = 256;
    const uint64_t nsize = fresh ? 0 : ((uint64_t)c->rho + c->hub_rows) * c->R;   // compact and hub rows
    IM_LAUNCH(c, K_INIT_KEYS, k_init_keys, grid_for(c->n > nsize ? c->n : nsize, T, 152u * 16u), T, 0,
              c->d_gain0, c->n, c->key_bits, c->d_key, c->d_stamp, c->d_seedflag, c->d_size, nsize);
    IM_CUDA(c, cudaMemsetAsync(c->d_sel, 0, sizeof(SelState), c->stream));
    IM_CUDA(c, cudaMemsetAsync(c->d_labcache, 0xFF, (size_t)kLabSlots * c->R * sizeof(uint64_t), c->stream));
    IM_LAUNCH(c, K_SEL_BEGIN, k_spec_init, 1, 32, 0, c->d_sel, c->d_spec_ids, c->spec_count);
    IM_CUDA(c, cudaGetLastError());
    c->seeds.clear();
    c->seed_gains.clear();
    c->round_evals.clear();
    c->dev_launches_seen = 0;
    return IM_OK;
}

namespace {

// The grid of k_sel_step: the blocks that fit on the device at once.
int size_step_grid(im_ctx* c) {
    if (c->step_grid) return IM_OK;
    int per_sm = 0, sms = 0;
    IM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sel_step, kBlockWarps * 32, 0));
    IM_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const unsigned grid = (unsigned)std::max(1, per_sm) * (unsigned)std::max(1, sms);
    if (im_dev_malloc(&c->d_topb, (size_t)grid * kTopB * sizeof(uint64_t)) != cudaSuccess)
        return im_fail(c, IM_ENOMEM, "top-B scratch");
    c->step_grid = grid;
    return IM_OK;
}

// One phase of the selection (k_sel_step).
int launch_step(im_ctx* c, const SelHandles& hd) {
    const int rc = size_step_grid(c);
    if (rc) return rc;
    IM_LAUNCH(c, K_SEL_STEP, k_sel_step, c->step_grid, kBlockWarps * 32, 0, step_args(c, hd));
    return IM_OK;
}

int launch_reduce_plan(im_ctx* c, const SelHandles& hd) {
    IM_LAUNCH(c, K_REDUCE, k_reduce_plan, grid_for(c->n, 256, 152u * 8u), 256, 0, step_args(c, hd));
    return IM_OK;
}

// The launches of an evaluator outside k_sel_step (a case of the graph's switch), once the
// batch is gathered: large batches by one warp per (member, 32 sketches), very large ones by
// recomputing the sketches; then the reduction and plan.
int enqueue_rare(im_ctx* c, unsigned rare, const SelHandles& hd) {
    SelState* st = c->d_sel;
    unsigned long long* fresh = (unsigned long long*)c->d_fresh;
    if (rare == RARE_CHUNK) {
        const GraphView g = graph_view(c);
        const SketchView s = sketch_view(c);
        const uint32_t nchunk = (c->R + 31) / 32;
        IM_LAUNCH(c, K_EVAL, k_eval, search_grid((uint64_t)c->n * nchunk), kEvalWarps * 32, 0, g, s, st, c->d_batch,
                  fresh, c->d_fb_tasks, c->fb_cap, nchunk);
        launch_fallback(c, g, s);
    } else if (rare == RARE_REFRESH) {
        const int rc = im_refresh_eval(c, c->d_batch, &st->batch_n, fresh, c->d_seed_list, &st->round);
        if (rc) return rc;
    } else {
        return im_fail(c, IM_EDEVICE, "unknown batch evaluator");
    }
    return launch_reduce_plan(c, hd);
}

int cap_begin(im_ctx* c, cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps) {
    IM_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, graph, deps, nullptr, ndeps,
                                             cudaStreamCaptureModeRelaxed));
    c->cur = c->cap_stream;
    c->capturing = true;
    return IM_OK;
}

int cap_end(im_ctx* c) {
    cudaGraph_t out = nullptr;
    c->capturing = false;
    c->cur = c->stream;
    IM_CUDA(c, cudaStreamEndCapture(c->cap_stream, &out));
    return IM_OK;
}

// The single node the capture currently ends at.
int cap_frontier(im_ctx* c, cudaGraphNode_t* node) {
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    IM_CUDA(c, cudaStreamGetCaptureInfo(c->cap_stream, &status, nullptr, nullptr, &deps, nullptr, &ndeps));
    if (status != cudaStreamCaptureStatusActive || ndeps != 1) return im_fail(c, IM_ECUDA, "selection graph capture");
    *node = deps[0];
    return IM_OK;
}

// A conditional node without dependencies, added to a graph directly.
int add_conditional(im_ctx* c, cudaGraph_t graph, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    unsigned size, cudaGraph_t* bodies, cudaGraphNode_t* node) {
    cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
    memset(&prm, 0, sizeof prm);   // reserved fields and padding must be zero
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = type;
    prm.conditional.size = size;
    IM_CUDA(c, cudaGraphAddNode(node, graph, nullptr, nullptr, 0, &prm));
    for (unsigned i = 0; i < size; ++i) bodies[i] = prm.conditional.phGraph_out[i];
    return IM_OK;
}

// Append a conditional node after the captured work and continue the capture after it.
int cap_conditional(im_ctx* c, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    unsigned size, cudaGraph_t* bodies) {
    cudaStreamCaptureStatus status;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    IM_CUDA(c, cudaStreamGetCaptureInfo(c->cap_stream, &status, nullptr, &cg, &deps, &edata, &ndeps));
    if (status != cudaStreamCaptureStatusActive) return im_fail(c, IM_ECUDA, "selection graph capture");
    cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
    memset(&prm, 0, sizeof prm);   // reserved fields and padding must be zero
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = type;
    prm.conditional.size = size;
    cudaGraphNode_t node = nullptr;
    IM_CUDA(c, cudaGraphAddNode(&node, cg, deps, edata, ndeps, &prm));
    for (unsigned i = 0; i < size; ++i) bodies[i] = prm.conditional.phGraph_out[i];
    IM_CUDA(c, cudaStreamUpdateCaptureDependencies(c->cap_stream, &node, nullptr, 1,
                                                   cudaStreamSetCaptureDependencies));
    return IM_OK;
}
// The whole lazy-greedy loop as one graph, so that rounds run back to back without the host:
//   sel_begin;
//   while (outer) {
//       while (inner) { k_sel_step x kStepsPerLoop }      -- one phase per launch
//       switch (rare) { chunk evaluation | recomputation, then k_reduce_plan }
//   }
// Every decision is taken on the device (plan_step, run by the last block of a step).  An
// iteration of a while loop or a switch costs several microseconds, a kernel node about one,
// so the phases of ordinary batches are launches of one kernel in a loop, not cases of a
// switch.  The loop is bounded: a round ends after at most 82 batches, the selection after
// round_end rounds.
constexpr int kStepsPerLoop = 8;

// The selection loop added to `root` after the nodes `deps`: k_sel_begin, then
//   while (outer) { while (inner) { k_sel_step x kStepsPerLoop }; switch (rare) { ... } }
// *last receives the outer loop node.  hd carries the rare evaluators' launch counts on entry.
int add_selection(im_ctx* c, cudaGraph_t root, const cudaGraphNode_t* deps, size_t ndeps, SelHandles& hd,
                  cudaGraphNode_t* last) {
    int rc = IM_OK;
    // the outer loop node first, so that the handles sel_begin sets exist before it is captured
    IM_CUDA(c, cudaGraphConditionalHandleCreate(&hd.outer, root, 0, 0));
    cudaGraph_t obody = nullptr, ibody = nullptr, rcases[RARE_COUNT] = {};
    cudaGraphNode_t onode = nullptr;
    if ((rc = add_conditional(c, root, hd.outer, cudaGraphCondTypeWhile, 1, &obody, &onode))) return rc;
    IM_CUDA(c, cudaGraphConditionalHandleCreate(&hd.inner, obody, 0, 0));
    IM_CUDA(c, cudaGraphConditionalHandleCreate(&hd.rare, obody, RARE_NONE, 0));
    if ((rc = cap_begin(c, root, deps, ndeps))) return rc;
    IM_LAUNCH(c, K_SEL_BEGIN, k_sel_begin, 1, 32, 0, c->d_sel, hd);
    cudaGraphNode_t first = nullptr;
    if ((rc = cap_frontier(c, &first))) return rc;
    if ((rc = cap_end(c))) return rc;
    IM_CUDA(c, cudaGraphAddDependencies(root, &first, &onode, nullptr, 1));

    if ((rc = cap_begin(c, obody, nullptr, 0))) return rc;
    if ((rc = cap_conditional(c, hd.inner, cudaGraphCondTypeWhile, 1, &ibody))) return rc;
    if ((rc = cap_conditional(c, hd.rare, cudaGraphCondTypeSwitch, RARE_COUNT, rcases))) return rc;
    if ((rc = cap_end(c))) return rc;
    if ((rc = cap_begin(c, ibody, nullptr, 0))) return rc;
    for (int i = 0; i < kStepsPerLoop && !rc; ++i) rc = launch_step(c, hd);
    if (rc) return rc;
    if ((rc = cap_end(c))) return rc;
    for (unsigned m = 0; m < RARE_COUNT; ++m) {
        if ((rc = cap_begin(c, rcases[m], nullptr, 0))) return rc;
        if ((rc = enqueue_rare(c, m, hd))) return rc;
        if ((rc = cap_end(c))) return rc;
    }
    *last = onode;
    return IM_OK;
}

int build_select_graph_steps(im_ctx* c) {
    SelHandles hd{};
    hd.on = 1;
    // launches of each rare evaluator, counted by dry runs of the same code
    c->count_only = true;
    int rc = IM_OK;
    for (unsigned m = 0; m < RARE_COUNT && !rc; ++m) {
        c->dry_count = 0;
        rc = enqueue_rare(c, m, hd);
        hd.rare_launches[m] = (unsigned)c->dry_count;
    }
    c->count_only = false;
    if (rc) return rc;
    if ((rc = size_step_grid(c))) return rc;   // before the capture

    IM_CUDA(c, cudaGraphCreate(&c->sel_graph, 0));
    cudaGraphNode_t onode = nullptr;
    if ((rc = add_selection(c, c->sel_graph, nullptr, 0, hd, &onode))) return rc;
    IM_CUDA(c, cudaGraphInstantiate(&c->sel_exec, c->sel_graph, 0));
    return IM_OK;
}

int build_select_graph(im_ctx* c) {
    if (c->sel_exec) return IM_OK;
    if (!c->cap_stream) IM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const int rc = build_select_graph_steps(c);
    if (rc) {
        c->count_only = false;
        if (c->capturing) {
            cudaGraph_t out = nullptr;
            cudaStreamEndCapture(c->cap_stream, &out);
            c->capturing = false;
        }
        c->cur = c->stream;
        cudaGetLastError();
        im_select_graph_free(c);
    }
    return rc;
}

const char* sel_error_text(unsigned e) {
    switch (e) {
    case SEL_FB_OVERFLOW: return "BFS fallback queue capacity exceeded";
    case SEL_NO_PROGRESS: return "re-evaluation batch made no progress";
    case SEL_NO_CANDIDATE: return "no candidate left for the next seed";
    case SEL_RANGE: return "selected id out of range";
    default: return "selection kernel reported an error";
    }
}

// The same phases driven from the host: one synchronisation per launch to read the decision.
int run_rounds_host(im_ctx* c) {
    const SelHandles none{};
    IM_LAUNCH(c, K_SEL_BEGIN, k_sel_begin, 1, 32, 0, c->d_sel, none);
    for (;;) {
        int rc = pull_state(c);
        if (rc) return rc;
        const SelState& h = *c->h_sel;
        if (h.rare != RARE_NONE) rc = enqueue_rare(c, h.rare, none);
        else if (h.phase != PH_NONE) rc = launch_step(c, none);
        else return IM_OK;
        if (rc) return rc;
    }
}

// ---- the device-resident request loop -------------------------------------------------
// serve graph:  while (serve) { k_mb_take; <selection loop>; k_mb_publish }
// k_mb_take waits (bounded) for requests in the mailbox and sets the selection's target to the
// largest requested k; the selection loop runs the rounds up to it (Alg. 1, Alg. 2 / Alg. 4);
// k_mb_publish copies the new seeds and gains into the mailbox.  A wait that sees no request
// for idle_ns (or kMbMaxPolls polls) ends the loop with IM_ETIMEOUT; the host launches it again
// for its next request.

__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys(unsigned* p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned kMbMaxPolls = 1u << 24;   // polls of one wait at most, whatever the clock says

__global__ void k_mb_take(MailboxShared* mb, SelState* st, cudaGraphConditionalHandle serve, uint32_t n,
                          unsigned long long refresh_min) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned* kring = reinterpret_cast<const unsigned*>(mb + 1);
    const unsigned ring = mb->ring, kcap = mb->kcap;
    const unsigned long long idle_ns = mb->idle_ns;
    const unsigned tail = mb->tail;   // only this kernel writes it
    const unsigned long long t0 = global_ns();
    for (unsigned polls = 0;; ++polls) {
        const unsigned stop = ld_acquire_sys(&mb->stop);
        unsigned head = ld_acquire_sys(&mb->head);
        bool idle = false;
        if (!stop && head == tail && (polls >= kMbMaxPolls || global_ns() - t0 >= idle_ns)) {
            // idle: clear `running`, then look once more -- a request pushed before the host read
            // running == 0 is taken now; one pushed after it gets a new launch from the host
            atomicExch_system(&mb->running, 0u);
            __threadfence_system();
            head = ld_acquire_sys(&mb->head);
            if (head == tail) idle = true;
            else atomicExch_system(&mb->running, 1u);
        }
        if (stop || idle) {
            if (stop) atomicExch_system(&mb->running, 0u);
            *reinterpret_cast<volatile int*>(&mb->status) = stop ? IM_OK : IM_ETIMEOUT;
            st->round_end = st->round;   // no round in this pass of the loop
            __threadfence_system();
            atomicAdd_system(&mb->exits, 1u);
            cudaGraphSetConditional(serve, 0);
            return;
        }
        if (head != tail) {
            const unsigned cnt = head - tail < ring ? head - tail : ring;   // the host keeps <= ring in flight
            unsigned kmax = 0;
            for (unsigned i = 0; i < cnt; ++i) kmax = max(kmax, kring[(tail + i) % ring]);
            st_release_sys(&mb->tail, tail + cnt);
            kmax = min(min(kmax, n), kcap);
            st->round_end = max(st->round, kmax);   // the sequence only grows
            st->refresh_min = refresh_min;
            *reinterpret_cast<volatile int*>(&mb->status) = IM_OK;
            cudaGraphSetConditional(serve, 1);
            return;
        }
        __nanosleep(500);
    }
}

__global__ void k_mb_publish(MailboxShared* mb, const SelState* st, const uint32_t* __restrict__ seed_list,
                             const uint64_t* __restrict__ gain_list, cudaGraphConditionalHandle serve) {
    __shared__ unsigned from, to;
    if (threadIdx.x == 0) {
        from = *reinterpret_cast<volatile unsigned*>(&mb->answered);
        to = min(st->round, mb->kcap);
    }
    __syncthreads();
    unsigned* seeds = reinterpret_cast<unsigned*>(mb + 1) + mb->ring;
    const size_t goff = ((size_t)(mb->ring + mb->kcap) * 4 + 7) & ~(size_t)7;
    unsigned long long* gains = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(mb + 1) + goff);
    for (unsigned i = from + threadIdx.x; i < to; i += blockDim.x) {
        seeds[i] = seed_list[i];
        gains[i] = gain_list[i];
    }
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (to > from) st_release_sys(&mb->answered, to);
        if (st->err || st->fb_overflow) {   // the selection stopped: so does the loop
            *reinterpret_cast<volatile int*>(&mb->status) = IM_EDEVICE;
            atomicExch_system(&mb->running, 0u);
            __threadfence_system();
            atomicAdd_system(&mb->exits, 1u);
            cudaGraphSetConditional(serve, 0);
        }
    }
}

size_t mailbox_bytes(uint32_t ring, uint32_t kcap) {
    return sizeof(MailboxShared) + ((((size_t)ring + kcap) * 4 + 7) & ~(size_t)7) + (size_t)kcap * 8;
}

int build_serve_graph(im_ctx* c, MailboxShared* dmb) {
    SelHandles hd{};
    hd.on = 1;
    c->count_only = true;
    int rc = IM_OK;
    for (unsigned m = 0; m < RARE_COUNT && !rc; ++m) {
        c->dry_count = 0;
        rc = enqueue_rare(c, m, hd);
        hd.rare_launches[m] = (unsigned)c->dry_count;
    }
    c->count_only = false;
    if (rc) return rc;
    if ((rc = size_step_grid(c))) return rc;
    IM_CUDA(c, cudaGraphCreate(&c->serve_graph, 0));
    cudaGraphConditionalHandle hserve;
    IM_CUDA(c, cudaGraphConditionalHandleCreate(&hserve, c->serve_graph, 1, cudaGraphCondAssignDefault));
    cudaGraph_t body = nullptr;
    cudaGraphNode_t snode = nullptr;
    if ((rc = add_conditional(c, c->serve_graph, hserve, cudaGraphCondTypeWhile, 1, &body, &snode))) return rc;
    if ((rc = cap_begin(c, body, nullptr, 0))) return rc;
    IM_LAUNCH(c, K_SEL_BEGIN, k_mb_take, 1, 32, 0, dmb, c->d_sel, hserve, c->n, (unsigned long long)c->refresh_min);
    cudaGraphNode_t take = nullptr;
    if ((rc = cap_frontier(c, &take))) return rc;
    if ((rc = cap_end(c))) return rc;
    cudaGraphNode_t onode = nullptr;
    if ((rc = add_selection(c, body, &take, 1, hd, &onode))) return rc;
    if ((rc = cap_begin(c, body, &onode, 1))) return rc;
    IM_LAUNCH(c, K_SEL_BEGIN, k_mb_publish, 1, 256, 0, dmb, c->d_sel, c->d_seed_list, c->d_gain_list, hserve);
    if ((rc = cap_end(c))) return rc;
    IM_CUDA(c, cudaGraphInstantiate(&c->serve_exec, c->serve_graph, 0));
    return IM_OK;
}

}  // namespace

void im_select_graph_free(im_ctx* c) {
    if (c->sel_exec) cudaGraphExecDestroy(c->sel_exec);
    if (c->sel_graph) cudaGraphDestroy(c->sel_graph);
    c->sel_exec = nullptr;
    c->sel_graph = nullptr;
    if (c->serve_exec) cudaGraphExecDestroy(c->serve_exec);
    if (c->serve_graph) cudaGraphDestroy(c->serve_graph);
    c->serve_exec = nullptr;
    c->serve_graph = nullptr;
    c->serve_mb = nullptr;
}

// Appends the device's seeds, gains and evaluation counts of rounds [r0, r1) to the host copy.
static int copy_new_seeds(im_ctx* c, uint32_t r0, uint32_t r1) {
    if (r1 <= r0) return IM_OK;
    const size_t cnt = r1 - r0;
    std::vector<uint32_t> sd(cnt);
    std::vector<uint64_t> gn(cnt), ev(cnt);
    IM_CUDA(c, cudaMemcpyAsync(sd.data(), c->d_seed_list + r0, cnt * 4, cudaMemcpyDeviceToHost, c->stream));
    IM_CUDA(c, cudaMemcpyAsync(gn.data(), c->d_gain_list + r0, cnt * 8, cudaMemcpyDeviceToHost, c->stream));
    IM_CUDA(c, cudaMemcpyAsync(ev.data(), c->d_round_evals + r0, cnt * 8, cudaMemcpyDeviceToHost, c->stream));
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->seeds.insert(c->seeds.end(), sd.begin(), sd.end());
    c->seed_gains.insert(c->seed_gains.end(), gn.begin(), gn.end());
    c->round_evals.insert(c->round_evals.end(), ev.begin(), ev.end());
    return IM_OK;
}

// Rounds of lazy greedy (NextSeed + MarkSeed) until k seeds are chosen.
int im_select_run(im_ctx* c, uint32_t k) {
    const uint32_t r0 = (uint32_t)c->seeds.size();
    if (r0 >= k) return IM_OK;
    IM_LAUNCH(c, K_SEL_BEGIN, k_set_target, 1, 32, 0, c->d_sel, k, (unsigned long long)c->refresh_min);
    int rc = IM_OK;
    if (c->use_graph) {
        if ((rc = build_select_graph(c))) return rc;
        int ev0 = -1;
        im_prof_begin(c, K_SELECT_GRAPH, &ev0, false);
        IM_CUDA(c, cudaGraphLaunch(c->sel_exec, c->stream));
        im_prof_end(c, K_SELECT_GRAPH, ev0);
    } else {
        rc = run_rounds_host(c);
        if (rc) return rc;
    }
    if ((rc = pull_state(c))) return rc;
    const SelState& h = *c->h_sel;
    if (c->use_graph) c->launches += h.launches - c->dev_launches_seen;
    c->dev_launches_seen = h.launches;
    // rounds completed before any error keep their seeds
    const uint32_t r1 = h.round < k ? h.round : k;
    if ((rc = copy_new_seeds(c, r0, r1))) return rc;    if (h.err) return im_fail(c, IM_EDEVICE, sel_error_text(h.err));
    if (h.fb_overflow) return im_fail(c, IM_EDEVICE, sel_error_text(SEL_FB_OVERFLOW));
    if (r1 < k) return im_fail(c, IM_EDEVICE, "selection stopped early");
    return IM_OK;
}

int im_spread_run(im_ctx* c, uint32_t k, uint64_t* out) {
    const GraphView g = graph_view(c);
    const SketchView s = sketch_view(c);
    const uint32_t nchunk = (c->R + 31) / 32;
    IM_LAUNCH(c, K_REDUCE_RESET, k_phase_reset, 1, 32, 0, c->d_sel);
    IM_CUDA(c, cudaMemsetAsync(c->d_spread_total, 0, sizeof(unsigned long long), c->stream));
    if (k > 0) {
        IM_LAUNCH(c, K_SPREAD_TASKS, k_spread_tasks, search_grid((uint64_t)k * nchunk), kEvalWarps * 32, 0,
                  g, s, c->d_sel, c->d_spread_seeds, k, nchunk, c->d_fb_tasks, c->fb_cap,
                  c->d_spread_pairs);
        launch_fallback(c, g, s);
        uint32_t kp2 = 1;
        while (kp2 < k) kp2 <<= 1;
        const size_t smem = (size_t)kp2 * sizeof(uint64_t);
        IM_CUDA(c, cudaFuncSetAttribute(k_spread_dedup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(smem > 48 * 1024 ? smem : 48 * 1024)));
        IM_LAUNCH(c, K_SPREAD_DEDUP, k_spread_dedup, c->R, 1024, smem, c->d_spread_pairs, k, kp2,
                  c->d_spread_total);
    }
    IM_CUDA(c, cudaGetLastError());
    unsigned long long h = 0;
    IM_CUDA(c, cudaMemcpyAsync(&h, c->d_spread_total, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    int rc = sync_state(c);
    if (rc) return rc;
    *out = h;
    return IM_OK;
}

// ---- the selection and spread of one instance in a batch graph --------------------------
int im_select_prepare(im_ctx* c, uint32_t k) {
    if (!c->cap_stream) IM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    int rc = size_step_grid(c);
    if (!rc) rc = spread_reserve(c, k);
    return rc;
}

// The selection of the first k seeds of the context, appended to g after `after`: the target
// (k_set_target), then the selection loop.
int im_select_graph_append(im_ctx* c, cudaGraph_t g, cudaGraphNode_t after, uint32_t k, cudaGraphNode_t* last) {
    SelHandles hd{};
    hd.on = 1;
    c->count_only = true;
    int rc = IM_OK;
    for (unsigned m = 0; m < RARE_COUNT && !rc; ++m) {
        c->dry_count = 0;
        rc = enqueue_rare(c, m, hd);
        hd.rare_launches[m] = (unsigned)c->dry_count;
    }
    c->count_only = false;
    if (rc) return rc;
    if ((rc = cap_begin(c, g, &after, 1))) return rc;
    IM_LAUNCH(c, K_SEL_BEGIN, k_set_target, 1, 32, 0, c->d_sel, k, (unsigned long long)c->refresh_min);
    cudaGraphNode_t target = nullptr;
    rc = cap_frontier(c, &target);
    const int re = cap_end(c);
    if (!rc) rc = re;
    if (!rc) rc = add_selection(c, g, &target, 1, hd, last);
    c->cur = c->stream;
    return rc;
}

// Spread of the first k selected seeds (still on the device), total to pinned host memory.
int im_spread_enqueue(im_ctx* c, uint32_t k, unsigned long long* h_total) {
    const GraphView g = graph_view(c);
    const SketchView s = sketch_view(c);
    const uint32_t nchunk = (c->R + 31) / 32;
    IM_CUDA(c, cudaMemcpyAsync(c->d_spread_seeds, c->d_seed_list, (size_t)k * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, c->stream));
    IM_LAUNCH(c, K_REDUCE_RESET, k_phase_reset, 1, 32, 0, c->d_sel);
    IM_CUDA(c, cudaMemsetAsync(c->d_spread_total, 0, sizeof(unsigned long long), c->stream));
    IM_LAUNCH(c, K_SPREAD_TASKS, k_spread_tasks, search_grid((uint64_t)k * nchunk), kEvalWarps * 32, 0, g, s,
              c->d_sel, c->d_spread_seeds, k, nchunk, c->d_fb_tasks, c->fb_cap, c->d_spread_pairs);
    launch_fallback(c, g, s);
    uint32_t kp2 = 1;
    while (kp2 < k) kp2 <<= 1;
    const size_t smem = (size_t)kp2 * sizeof(uint64_t);
    IM_CUDA(c, cudaFuncSetAttribute(k_spread_dedup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(smem > 48 * 1024 ? smem : 48 * 1024)));
    IM_LAUNCH(c, K_SPREAD_DEDUP, k_spread_dedup, c->R, 1024, smem, c->d_spread_pairs, k, kp2, c->d_spread_total);
    IM_CUDA(c, cudaMemcpyAsync(h_total, c->d_spread_total, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               c->stream));
    return IM_OK;
}

// ---- device-resident request loop: host side -------------------------------------------
struct im_mailbox {
    im_ctx* ctx = nullptr;
    MailboxShared* h = nullptr;   // host view (mapped pinned memory)
    MailboxShared* d = nullptr;   // device view
};

namespace {

unsigned* mb_ring(const im_mailbox* mb) { return reinterpret_cast<unsigned*>(mb->h + 1); }
unsigned* mb_seeds(const im_mailbox* mb) { return mb_ring(mb) + mb->h->ring; }
unsigned long long* mb_gains(const im_mailbox* mb) {
    const size_t goff = (((size_t)mb->h->ring + mb->h->kcap) * 4 + 7) & ~(size_t)7;
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(mb->h + 1) + goff);
}
template <typename T> T load_acq(const T* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
template <typename T> void store_rel(T* p, T v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }

}  // namespace

// A context destroyed while a loop serves it asks that loop to stop first.
void im_serve_stop(im_ctx* c) {
    if (c->serving && c->serve_mb)
        store_rel(&static_cast<im_mailbox*>(const_cast<void*>(c->serve_mb))->h->stop, 1u);
}

extern "C" {

int im_mailbox_create(im_ctx* c, uint32_t ring, uint32_t kcap, im_mailbox** out) {
    if (!c || !out) return IM_EINVAL;
    if (ring == 0 || ring > 65536) return im_fail(c, IM_EINVAL, "ring must be in [1, 65536]");
    if (kcap == 0 || kcap > c->n) return im_fail(c, IM_EINVAL, "kcap must be in [1, n]");
    im_mailbox* mb = new (std::nothrow) im_mailbox();
    if (!mb) return im_fail(c, IM_ENOMEM, "mailbox");
    void* p = nullptr;
    const size_t bytes = mailbox_bytes(ring, kcap);
    if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        delete mb;
        return im_fail(c, IM_ENOMEM, "mailbox (mapped host memory)");
    }
    memset(p, 0, bytes);
    mb->ctx = c;
    mb->h = static_cast<MailboxShared*>(p);
    mb->h->ring = ring;
    mb->h->kcap = kcap;
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, p, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(p);
        delete mb;
        return im_fail(c, IM_ECUDA, "mailbox device pointer");
    }
    mb->d = static_cast<MailboxShared*>(dp);
    *out = mb;
    return IM_OK;
}

int im_mailbox_destroy(im_mailbox* mb) {
    if (!mb) return IM_EINVAL;
    im_ctx* c = mb->ctx;
    if (c->serving && c->serve_mb == mb) return im_fail(c, IM_ESTATE, "a loop still serves this mailbox");
    if (c->serve_mb == mb) {   // its graph points at this mailbox
        if (c->serve_exec) cudaGraphExecDestroy(c->serve_exec);
        if (c->serve_graph) cudaGraphDestroy(c->serve_graph);
        c->serve_exec = nullptr;
        c->serve_graph = nullptr;
        c->serve_mb = nullptr;
    }
    cudaFreeHost(mb->h);
    delete mb;
    return IM_OK;
}

int im_mailbox_push(im_mailbox* mb, uint32_t k) {
    if (!mb) return IM_EINVAL;
    MailboxShared* h = mb->h;
    if (k == 0 || k > h->kcap) return im_fail(mb->ctx, IM_EINVAL, "k must be in [1, kcap]");
    const unsigned head = h->head, tail = load_acq(&h->tail);
    if (head - tail >= h->ring) return im_fail(mb->ctx, IM_ESTATE, "mailbox ring is full");
    mb_ring(mb)[head % h->ring] = k;
    store_rel(&h->head, head + 1);
    return IM_OK;
}

int im_mailbox_state(const im_mailbox* mb, uint32_t* running, int32_t* status, uint32_t* answered) {
    if (!mb) return IM_EINVAL;
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    if (running) *running = load_acq(&mb->h->running);
    if (status) *status = load_acq(&mb->h->status);
    if (answered) *answered = load_acq(&mb->h->answered);
    return IM_OK;
}

int im_serve_launch(im_mailbox* mb, uint32_t idle_us) {
    if (!mb) return IM_EINVAL;
    im_ctx* c = mb->ctx;
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    if (idle_us == 0 || idle_us > 10000000u) return im_fail(c, IM_EINVAL, "idle_us must be in [1, 10^7]");
    if (c->serving && c->serve_mb != mb) return im_fail(c, IM_ESTATE, "another mailbox's loop serves the context");
    if (!c->serving) {
        // a new loop publishes the context's sequence from its start (the sketches may have been
        // rebuilt since this mailbox was last served)
        store_rel(&mb->h->answered, 0u);
        store_rel(&mb->h->status, (int)IM_OK);
    }
    if (c->serve_mb != mb || !c->serve_exec) {
        if (c->serve_exec) cudaGraphExecDestroy(c->serve_exec);
        if (c->serve_graph) cudaGraphDestroy(c->serve_graph);
        c->serve_exec = nullptr;
        c->serve_graph = nullptr;
        c->serve_mb = nullptr;
        if (!c->cap_stream) IM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        const int rc = build_serve_graph(c, mb->d);
        if (rc) {
            c->count_only = false;
            if (c->capturing) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(c->cap_stream, &g);
                c->capturing = false;
            }
            c->cur = c->stream;
            cudaGetLastError();
            if (c->serve_exec) cudaGraphExecDestroy(c->serve_exec);
            if (c->serve_graph) cudaGraphDestroy(c->serve_graph);
            c->serve_exec = nullptr;
            c->serve_graph = nullptr;
            return rc;
        }
        c->serve_mb = mb;
    }
    mb->h->idle_ns = (unsigned long long)idle_us * 1000ull;
    store_rel(&mb->h->stop, 0u);
    store_rel(&mb->h->running, 1u);
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    c->serving = true;
    IM_CUDA(c, cudaGraphLaunch(c->serve_exec, c->stream));
    return IM_OK;
}

int im_mailbox_wait(im_mailbox* mb, uint32_t k, uint32_t timeout_us, uint32_t* seeds, uint64_t* gains) {
    if (!mb) return IM_EINVAL;
    im_ctx* c = mb->ctx;
    MailboxShared* h = mb->h;
    if (k == 0 || k > h->kcap) return im_fail(c, IM_EINVAL, "k must be in [1, kcap]");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    for (;;) {
        __atomic_thread_fence(__ATOMIC_SEQ_CST);
        unsigned answered = load_acq(&h->answered);
        if (answered < k) {
            if (load_acq(&h->status) == IM_EDEVICE) return im_fail(c, IM_EDEVICE, "the serving loop's selection stopped");
            if (!load_acq(&h->running)) {
                answered = load_acq(&h->answered);   // published before the loop stopped
                if (answered < k) return im_fail(c, IM_ESTATE, "no loop serves this mailbox (launch one)");
            }
        }
        if (answered >= k) {
            for (uint32_t i = 0; i < k; ++i) {
                if (seeds) seeds[i] = mb_seeds(mb)[i];
                if (gains) gains[i] = mb_gains(mb)[i];
            }
            return IM_OK;
        }
        if (std::chrono::steady_clock::now() >= deadline) return im_fail(c, IM_ETIMEOUT, "no answer in time");
        std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
}

int im_serve_finish(im_mailbox* mb, int32_t* loop_status) {
    if (!mb) return IM_EINVAL;
    im_ctx* c = mb->ctx;
    store_rel(&mb->h->stop, 1u);
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (loop_status) *loop_status = load_acq(&mb->h->status);
    store_rel(&mb->h->stop, 0u);
    if (!c->serving) return IM_OK;
    c->serving = false;
    // the host copy of the sequence catches up with the rounds the loop ran
    int rc = pull_state(c);
    if (rc) return rc;
    const SelState& hs = *c->h_sel;
    if (c->use_graph) c->launches += hs.launches - c->dev_launches_seen;
    c->dev_launches_seen = hs.launches;
    rc = copy_new_seeds(c, (uint32_t)c->seeds.size(), hs.round);
    if (rc) return rc;
    if (hs.err) return im_fail(c, IM_EDEVICE, sel_error_text(hs.err));
    if (hs.fb_overflow) return im_fail(c, IM_EDEVICE, sel_error_text(SEL_FB_OVERFLOW));
    return IM_OK;
}

}  // extern "C"
