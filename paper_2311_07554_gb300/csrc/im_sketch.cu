// im_sketch.cu -- Step 1 of Alg. 1: sketch construction (Sec. 3, Alg. 3 Sketch(r)).
//
// Batches of B sketches share one pass over the edge list.  Per sketch b of a batch:
//   init        P[b][v] = v;  W[b][v] = (key = lk(v), count = 1)
//   sample      every live (edge, sketch) pair of the batch becomes a record (u, v, b), or on
//               the bucketed path (large graphs) a record (u, v) in a region of sketch b
//   union       one thread per record, Rem's union with splicing (parents below children);
//               the bucketed path unites the sketches one after the other
//   compress    P[b][v] <- root; per root, for every other member: count += 1 and
//               key = min over members of the
//               label key of its centers (center index) -- with every vertex a center this
//               is the smallest id (Alg. 3's canonical label)
//   gain        Delta[v] += sum_b count(root_b(v)); for a center c_i: label[i] = key of its
//               root (the smallest center index in its component), size[i] = count if
//               label[i] = i, else 0 (Alg. 3)
// W[b][x] is one 64-bit word per root: low half = component size (bit 31 is the "holds a
// seed" flag of the recomputation evaluator), high half = the component's minimum key.  A
// root with members carries kRootFlag on its own parent entry, so that the gain pass knows
// singletons (size 1, own key) without reading their root words.
#include <algorithm>

#include "im_internal.cuh"
#include "im_uf.cuh"

using namespace imk;

namespace {

__device__ __forceinline__ uint32_t* w_count(uint64_t* w) { return reinterpret_cast<uint32_t*>(w); }
__device__ __forceinline__ uint32_t* w_key(uint64_t* w) { return reinterpret_cast<uint32_t*>(w) + 1; }

// Every vertex starts as the root of its own component: size 1, key = its own label key.
// Compression then only has to add the vertices that stopped being roots.
__device__ __forceinline__ uint32_t label_key(uint32_t v, int key_mode, const uint32_t* cidx) {
    return key_mode == 0 ? v : (key_mode == 1 ? cidx[v] : kNone);
}

__global__ void k_batch_init(uint32_t* __restrict__ parent, uint64_t* __restrict__ word,
                             uint32_t n, uint32_t nb, const uint32_t* __restrict__ cidx, int key_mode) {
    const uint64_t total = (uint64_t)n * nb;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const uint32_t v = (uint32_t)(i % n);
        parent[i] = v;
        if (word) word[i] = ((uint64_t)label_key(v, key_mode, cidx) << 32) | 1u;
    }
}

// Fused sampling + union (used when the record buffer is absent or overflows).
template <int B>
__device__ __forceinline__ void sample_union_pair(const uint4& two, uint64_t i, uint64_t m,
                                                  const Sampler& smp, uint64_t g0, uint32_t nb,
                                                  uint32_t* parent, uint32_t n) {
    const uint64_t k0 = mix64(smp.salt ^ (2 * i)), k1 = mix64(smp.salt ^ (2 * i + 1));
    const bool has1 = 2 * i + 1 < m;
    const uint64_t T0 = smp.eT ? smp.eT[2 * i] : uniform_T(smp);
    const uint64_t T1 = (smp.eT && has1) ? smp.eT[2 * i + 1] : uniform_T(smp);
    uint64_t rg = g0;
    for (uint32_t b = 0; b < nb; ++b) {
        if (live_T(k0, rg, T0)) unite_rem(parent + (size_t)b * n, two.x, two.y);
        if (has1 && live_T(k1, rg, T1)) unite_rem(parent + (size_t)b * n, two.z, two.w);
        rg += kGamma;
    }
}

template <int B>
__global__ void __launch_bounds__(256)
k_sample_union(const uint4* __restrict__ edge_pairs, uint64_t m, Sampler smp, uint32_t r0,
               uint32_t nb, uint32_t* __restrict__ parent, uint32_t n) {
    const uint64_t npairs = (m + 1) >> 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g0 = (uint64_t)(r0 + 1u) * kGamma;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += stride)
        sample_union_pair<B>(edge_pairs[i], i, m, smp, g0, nb, parent, n);
}

// Live (edge, sketch) pairs of one edge pair (edges 2i, 2i + 1) in sketches r0 .. r0+nb-1:
// bit b of live0 / live1 is set iff edge 2i / 2i+1 is live in sketch r0 + b.  Candidates are
// found on the high word of the hash (a superset of the live pairs, about 2^-31 larger) and
// settled with the full hash; the edge key mix(salt ^ e) is computed once for the batch.
template <int B>
__device__ __forceinline__ void pair_live_masks(uint64_t i, uint64_t m, const Sampler& smp, uint32_t r0,
                                                uint32_t nb, uint64_t g0, uint32_t& live0, uint32_t& live1) {
    const uint64_t e0 = 2 * i, e1 = 2 * i + 1;
    const uint64_t k0 = mix64(smp.salt ^ e0), k1 = mix64(smp.salt ^ e1);
    uint64_t T0 = uniform_T(smp), T1 = T0;
    if (smp.eT) {   // per-edge thresholds, stored pairwise like the edges
        const ulonglong2 tt = __ldcs(reinterpret_cast<const ulonglong2*>(smp.eT) + i);
        T0 = tt.x;
        T1 = tt.y;
    }
    const uint32_t all = (nb >= 32) ? 0xFFFFFFFFu : ((1u << nb) - 1u);
    live0 = live1 = 0;
    if (T0 == kAllLive && T1 == kAllLive) {
        live0 = live1 = all;
    } else {
        const uint32_t h0 = (uint32_t)(T0 >> 32), h1 = (uint32_t)(T1 >> 32);
        const uint32_t th0 = h0 == 0xFFFFFFFFu ? h0 : h0 + 1u;
        const uint32_t th1 = h1 == 0xFFFFFFFFu ? h1 : h1 + 1u;
        uint64_t x0 = k0 + g0, x1 = k1 + g0;
        if (nb == (uint32_t)B) {
#pragma unroll
            for (int b = 0; b < B; ++b) {
                if (mix64_hi_raw(x0) <= th0) live0 |= 1u << b;
                if (mix64_hi_raw(x1) <= th1) live1 |= 1u << b;
                x0 += kGamma;
                x1 += kGamma;
            }
        } else {
#pragma unroll
            for (int b = 0; b < B; ++b) {
                if (b < (int)nb) {
                    if (mix64_hi_raw(x0) <= th0) live0 |= 1u << b;
                    if (mix64_hi_raw(x1) <= th1) live1 |= 1u << b;
                }
                x0 += kGamma;
                x1 += kGamma;
            }
        }
        // exact test for the candidates (about a fraction p of all pairs)
        if (T0 == kAllLive) live0 = all;
        else
            for (uint32_t t = live0; t; t &= t - 1) {
                const int b = __ffs(t) - 1;
                if (!live_T(k0, (uint64_t)(r0 + b + 1u) * kGamma, T0)) live0 &= ~(1u << b);
            }
        if (T1 == kAllLive) live1 = all;
        else
            for (uint32_t t = live1; t; t &= t - 1) {
                const int b = __ffs(t) - 1;
                if (!live_T(k1, (uint64_t)(r0 + b + 1u) * kGamma, T1)) live1 &= ~(1u << b);
            }
    }
    if (e1 >= m) live1 = 0;
}

// Sampling alone: every live (edge, sketch) pair of the batch becomes a record (u, v, b, 0),
// appended with one atomic per warp.  The hash work (nb mixes per edge) is pure ALU; the
// latency-bound unions then run one thread per record in k_union_live.  The kernel also
// initialises the batch's forest (k_batch_init's stores), which the memory system drains
// while the hashing runs.
template <int B>
__global__ void __launch_bounds__(256)
k_sample_emit(const uint4* __restrict__ edge_pairs, uint64_t m, Sampler smp, uint32_t r0,
              uint32_t nb, uint4* __restrict__ out, unsigned long long* __restrict__ out_n,
              uint64_t cap, uint32_t* __restrict__ parent, uint64_t* __restrict__ word, uint32_t n,
              const uint32_t* __restrict__ cidx, int key_mode) {
    const uint64_t npairs = (m + 1) >> 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g0 = (uint64_t)(r0 + 1u) * kGamma;
    const unsigned lane = threadIdx.x & 31;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t w = ((uint64_t)label_key(v, key_mode, cidx) << 32) | 1u;
        for (uint32_t b = 0; b < nb; ++b) {
            parent[(size_t)b * n + v] = v;
            word[(size_t)b * n + v] = w;
        }
    }
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < npairs; base += stride) {
        const uint64_t i = base + threadIdx.x;
        uint32_t live0 = 0, live1 = 0;
        uint4 two = make_uint4(0, 0, 0, 0);
        if (i < npairs) {
            two = __ldcs(edge_pairs + i);   // streamed once per batch: keep L2 for the forest
            pair_live_masks<B>(i, m, smp, r0, nb, g0, live0, live1);
        }
        const uint32_t cntl = __popc(live0) + __popc(live1);
        uint32_t incl = cntl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if ((int)lane >= d) incl += y;
        }
        const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
        if (wtotal == 0) continue;
        unsigned long long wbase = 0;
        if (lane == 31) wbase = atomicAdd(out_n, (unsigned long long)wtotal);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        uint64_t pos = wbase + incl - cntl;
        while (live0) {
            const uint32_t b = __ffs(live0) - 1;
            live0 &= live0 - 1;
            if (pos < cap) out[pos] = make_uint4(two.x, two.y, b, 0u);
            ++pos;
        }
        while (live1) {
            const uint32_t b = __ffs(live1) - 1;
            live1 &= live1 - 1;
            if (pos < cap) out[pos] = make_uint4(two.z, two.w, b, 0u);
            ++pos;
        }
    }
}

// Unions each thread of the union kernels keeps in flight.
constexpr int kUnionChains = 4;

// 32 x 32 bit transpose across a warp: lane i holds row i (bit j = entry (i, j)); afterwards
// lane j holds column j (bit i = entry (i, j)).  Five rounds swap the off-diagonal blocks of
// size s between lanes i and i ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, unsigned lane) {
    const uint32_t masks[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu, 0xAAAAAAAAu};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int sh = 16 >> k;
        const uint32_t hi = masks[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sh);
        x = (lane & sh) ? ((x & hi) | ((y & hi) >> sh)) : ((x & ~hi) | ((y & ~hi) << sh));
    }
    return x;
}

// Sampling with the live pairs grouped by sketch and by block: block k writes the records (8
// bytes, (u, v)) of sketch b into region b * gridDim.x + k of the record buffer, counting them in
// shared memory, so no global atomic is needed; the unions then take the regions sketch by
// sketch, while one sketch's parent array stays in L2.  Per warp and pair of edges per lane, the
// live masks are transposed so that lane b holds sketch b's live edges; lane b reserves room in
// its block's region of sketch b with one shared-memory atomic and writes them (the endpoints
// come from their lanes by shuffles).  At the end every block stores its region counts (and
// raises *overflow if a region did not fit).  Also initialises the batch's forest, as
// k_sample_emit does.
template <int B>
__global__ void __launch_bounds__(256)
k_sample_bucket(const uint4* __restrict__ edge_pairs, uint64_t m, Sampler smp, uint32_t r0, uint32_t nb,
                uint2* __restrict__ out, uint32_t* __restrict__ region_n, uint32_t capr,
                unsigned int* __restrict__ overflow, uint32_t* __restrict__ parent, uint64_t* __restrict__ word,
                uint32_t n, const uint32_t* __restrict__ cidx, int key_mode) {
    __shared__ uint32_t cnt[32];
    const uint64_t npairs = (m + 1) >> 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g0 = (uint64_t)(r0 + 1u) * kGamma;
    const unsigned lane = threadIdx.x & 31;
    if (threadIdx.x < 32) cnt[threadIdx.x] = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t w = ((uint64_t)label_key(v, key_mode, cidx) << 32) | 1u;
        for (uint32_t b = 0; b < nb; ++b) {
            parent[(size_t)b * n + v] = v;
            word[(size_t)b * n + v] = w;
        }
    }
    __syncthreads();
    uint2* mine = out + ((size_t)lane * gridDim.x + blockIdx.x) * capr;   // lane b: sketch b's region
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < npairs; base += stride) {
        const uint64_t i = base + threadIdx.x;
        uint32_t live0 = 0, live1 = 0;
        uint4 two = make_uint4(0, 0, 0, 0);
        if (i < npairs) {
            two = __ldcs(edge_pairs + i);
            pair_live_masks<B>(i, m, smp, r0, nb, g0, live0, live1);
        }
        if (!__any_sync(0xffffffffu, (live0 | live1) != 0u)) continue;
        uint32_t t0 = warp_transpose32(live0, lane), t1 = warp_transpose32(live1, lane);
        const uint32_t c = __popc(t0) + __popc(t1);
        uint32_t pos = 0;
        if (c) pos = atomicAdd(&cnt[lane], c);
        for (;;) {   // rounds: each lane writes its next record
            const bool has = (t0 | t1) != 0u;
            if (!__any_sync(0xffffffffu, has)) break;
            int src = 0;
            bool second = false;
            if (t0) { src = __ffs(t0) - 1; t0 &= t0 - 1; }
            else if (t1) { src = __ffs(t1) - 1; t1 &= t1 - 1; second = true; }
            const uint32_t ex = __shfl_sync(0xffffffffu, two.x, src), ey = __shfl_sync(0xffffffffu, two.y, src);
            const uint32_t ez = __shfl_sync(0xffffffffu, two.z, src), ew = __shfl_sync(0xffffffffu, two.w, src);
            if (has) {
                if (pos < capr) mine[pos] = second ? make_uint2(ez, ew) : make_uint2(ex, ey);
                ++pos;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < nb) {
        const uint32_t k = cnt[threadIdx.x];
        region_n[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = k;
        if (k > capr) atomicOr(overflow, 1u);
    }
}

// Unions of the bucketed records: block (b, q) = blockIdx.x / groups, % groups unites the records
// of sketch b written by sampling blocks q * rpb .. q * rpb + rpb - 1 (its regions, taken as one
// list: each thread walks it with its own cursor), so the grid sweeps the sketches in order and
// the parents being climbed belong to a few sketches at a time.  Several unions in flight per
// thread, as k_union_live.  The last block resets the overflow flag; if it was raised, the
// batch is redone with the fused sample+union loop.
constexpr uint32_t kBucketRegionsPerBlock = 64;
constexpr uint32_t kBucketBlocksPerSM = 4;
template <int B>
__global__ void __launch_bounds__(256)
k_union_bucket(const uint2* __restrict__ recs, const uint32_t* __restrict__ region_n, uint32_t regions,
               uint32_t rpb, uint32_t capr, unsigned int* __restrict__ overflow, uint32_t* __restrict__ parent,
               uint32_t n, const uint4* __restrict__ edge_pairs, uint64_t m, Sampler smp, uint32_t r0,
               uint32_t nb, unsigned long long* __restrict__ total) {
    __shared__ unsigned int s_over;
    __shared__ uint32_t s_cnt[kBucketRegionsPerBlock];
    const uint32_t groups = (regions + rpb - 1) / rpb;
    const uint32_t b = blockIdx.x / groups;
    const uint32_t k0 = (blockIdx.x % groups) * rpb;
    const uint32_t nreg = min(rpb, regions - k0);
    const uint32_t reg0 = b * regions + k0;   // first region: sketch b, sampling block k0
    if (threadIdx.x < nreg) {
        const uint32_t c = region_n[reg0 + threadIdx.x];
        s_cnt[threadIdx.x] = c < capr ? c : capr;
        if (c) atomicAdd(total, (unsigned long long)c);
    }
    if (threadIdx.x == 0) {
        s_over = *reinterpret_cast<volatile unsigned int*>(overflow);
        __threadfence();
        if (atomicAdd(overflow + 1, 1u) == gridDim.x - 1u) {   // every block has read the flag
            overflow[0] = 0;
            overflow[1] = 0;
        }
    }
    __syncthreads();
    if (s_over) {
        const uint64_t npairs = (m + 1) >> 1;
        const uint64_t g0 = (uint64_t)(r0 + 1u) * kGamma;
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += stride)
            sample_union_pair<B>(edge_pairs[i], i, m, smp, g0, nb, parent, n);
        return;
    }
    uint32_t* Pb = parent + (size_t)b * n;
    // cursor: record j of region r (of this block's list); advanced by blockDim.x records
    uint32_t r = 0, j = threadIdx.x;
    while (r < nreg && j >= s_cnt[r]) j -= s_cnt[r++];
    constexpr int K = kUnionChains;
    uint32_t rx[K], ry[K], px[K], py[K], hres[K];
    bool act[K], hooked[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        act[k] = false;
        hooked[k] = false;
        rx[k] = ry[k] = px[k] = py[k] = hres[k] = 0;
    }
    for (;;) {
        bool any = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!act[k] && r < nreg) {
                const uint2 rc = recs[(size_t)(reg0 + r) * capr + j];
                j += blockDim.x;
                while (r < nreg && j >= s_cnt[r]) j -= s_cnt[r++];
                rx[k] = rc.x;
                ry[k] = rc.y;
                px[k] = __ldca(Pb + rx[k]);
                py[k] = __ldca(Pb + ry[k]);
                act[k] = true;
            }
            any |= act[k];
        }
        if (!any) break;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!act[k]) continue;
            if (hooked[k]) {
                hooked[k] = false;
                if (hres[k] == rx[k]) { act[k] = false; continue; }
                px[k] = hres[k];
            }
            if (px[k] == py[k]) { act[k] = false; continue; }
            if (px[k] < py[k]) {
                uint32_t t = rx[k]; rx[k] = ry[k]; ry[k] = t;
                t = px[k]; px[k] = py[k]; py[k] = t;
            }
            if (rx[k] == px[k]) {
                hres[k] = atomicCAS(Pb + rx[k], rx[k], py[k]);
                hooked[k] = true;
            } else {
                atomicCAS(Pb + rx[k], px[k], py[k]);
                rx[k] = px[k];
                px[k] = __ldca(Pb + rx[k]);
            }
        }
    }
}

// Forest of one batch: P[b][v] = v, W[b][v] = (label key of v, size 1).  grid.y = sketch.
__global__ void __launch_bounds__(256)
k_forest_init(uint32_t* __restrict__ parent, uint64_t* __restrict__ word, uint32_t n,
              const uint32_t* __restrict__ cidx, int key_mode) {
    uint32_t* P = parent + (size_t)blockIdx.y * n;
    uint64_t* W = word + (size_t)blockIdx.y * n;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        P[v] = v;
        W[v] = ((uint64_t)label_key(v, key_mode, cidx) << 32) | 1u;
    }
}

// Sampling and unions of one batch in one pass over the edges (the forest initialised
// before).  The live pairs a warp finds go to a queue of the warp in shared memory, one per
// lane and round; whenever 32 are queued, every lane unites one of them (Rem's union).  The
// unions are latency-bound and the hashing ALU-bound: while a warp waits on its unions, the
// SM issues the other warps' hashing, so no record of a live pair ever reaches device memory.
constexpr int kUnionQ = 64;      // queue entries per warp: at most 31 left + 32 appended
constexpr int kUniteWarps = 8;

template <int B>
__global__ void __launch_bounds__(kUniteWarps * 32)
k_sample_unite(const uint4* __restrict__ edge_pairs, uint64_t m, Sampler smp, uint32_t r0, uint32_t nb,
               uint32_t* __restrict__ parent, uint32_t n, unsigned long long* __restrict__ live_total) {
    __shared__ uint32_t qx[kUniteWarps][kUnionQ], qy[kUniteWarps][kUnionQ];
    __shared__ uint8_t qb[kUniteWarps][kUnionQ];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* QX = qx[warp];
    uint32_t* QY = qy[warp];
    uint8_t* QB = qb[warp];
    uint32_t qn = 0;              // queued entries (the same in every lane)
    uint32_t mine = 0;            // live pairs this lane found
    const uint64_t npairs = (m + 1) >> 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g0 = (uint64_t)(r0 + 1u) * kGamma;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < npairs; base += stride) {
        const uint64_t i = base + threadIdx.x;
        uint32_t l0 = 0, l1 = 0;
        uint4 two = make_uint4(0, 0, 0, 0);
        if (i < npairs) {
            two = __ldcs(edge_pairs + i);
            pair_live_masks<B>(i, m, smp, r0, nb, g0, l0, l1);
        }
        mine += __popc(l0) + __popc(l1);
        for (;;) {
            const bool has = (l0 | l1) != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, has);
            if (!bal) break;
            if (has) {
                uint32_t x, y, b;
                if (l0) { b = __ffs(l0) - 1; l0 &= l0 - 1; x = two.x; y = two.y; }
                else    { b = __ffs(l1) - 1; l1 &= l1 - 1; x = two.z; y = two.w; }
                const uint32_t pos = qn + __popc(bal & lt);
                QX[pos] = x;
                QY[pos] = y;
                QB[pos] = (uint8_t)b;
            }
            qn += __popc(bal);
            __syncwarp();
            if (qn >= 32) {
                qn -= 32;
                const uint32_t x = QX[qn + lane], y = QY[qn + lane], b = QB[qn + lane];
                __syncwarp();   // every lane has its entry before the queue grows again
                unite_rem(parent + (size_t)b * n, x, y);
            }
        }
    }
    __syncwarp();
    if (lane < qn) unite_rem(parent + (size_t)QB[lane] * n, QX[lane], QY[lane]);
#pragma unroll
    for (int d = 16; d; d >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, d);
    if (lane == 0 && mine) atomicAdd(live_total, (unsigned long long)mine);
}

// Rem's union of the batch's live records.  Each thread keeps kUnionChains records in flight
// (the state of their climbs in registers): every round issues one memory operation per chain
// -- a parent load or a hooking CAS -- and uses its result in the next round, so a thread
// waits for one round trip per round instead of one per step of every union.  The record
// count rec_n[0] is reset by the last block to read it (ticket rec_n[1]), ready for the lane's
// next batch.  If the record buffer overflowed, the batch is redone with the fused
// sample+union loop instead (decided on the device, so no host round trip).
template <int B>
__global__ void __launch_bounds__(256)
k_union_live(const uint4* __restrict__ recs, unsigned long long* __restrict__ rec_n, uint64_t cap,
             uint32_t* __restrict__ parent, uint32_t n, const uint4* __restrict__ edge_pairs,
             uint64_t m, Sampler smp, uint32_t r0, uint32_t nb, unsigned long long* __restrict__ total) {
    __shared__ unsigned long long s_cnt;
    if (threadIdx.x == 0) {
        const unsigned long long c0 = *reinterpret_cast<volatile unsigned long long*>(rec_n);
        s_cnt = c0;
        __threadfence();
        if (atomicAdd(rec_n + 1, 1ull) == gridDim.x - 1ull) {   // every block has the count
            rec_n[0] = 0;
            rec_n[1] = 0;
            atomicAdd(total, c0);
        }
    }
    __syncthreads();
    const unsigned long long cnt = s_cnt;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (cnt > cap) {
        const uint64_t npairs = (m + 1) >> 1;
        const uint64_t g0 = (uint64_t)(r0 + 1u) * kGamma;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += stride)
            sample_union_pair<B>(edge_pairs[i], i, m, smp, g0, nb, parent, n);
        return;
    }
    constexpr int K = kUnionChains;
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t* P[K];
    uint32_t rx[K], ry[K], px[K], py[K], hres[K];
    bool act[K], hooked[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        act[k] = false;
        hooked[k] = false;
        P[k] = parent;
        rx[k] = ry[k] = px[k] = py[k] = hres[k] = 0;
    }
    for (;;) {
        // chains without a record take the next one and load both endpoints' parents
        bool any = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!act[k] && j < cnt) {
                const uint4 rc = recs[j];
                j += stride;
                P[k] = parent + (size_t)rc.z * n;
                rx[k] = rc.x;
                ry[k] = rc.y;
                px[k] = __ldca(P[k] + rx[k]);
                py[k] = __ldca(P[k] + ry[k]);
                act[k] = true;
            }
            any |= act[k];
        }
        if (!any) break;
        // one step of every chain (Rem's union with splicing, im_uf.cuh), its memory operation
        // left in flight for the next round
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!act[k]) continue;
            if (hooked[k]) {
                hooked[k] = false;
                if (hres[k] == rx[k]) { act[k] = false; continue; }   // hooked rx under py
                px[k] = hres[k];                                       // rx got a parent meanwhile
            }
            if (px[k] == py[k]) { act[k] = false; continue; }          // the paths met
            if (px[k] < py[k]) {
                uint32_t t = rx[k]; rx[k] = ry[k]; ry[k] = t;
                t = px[k]; px[k] = py[k]; py[k] = t;
            }
            if (rx[k] == px[k]) {
                hres[k] = atomicCAS(P[k] + rx[k], rx[k], py[k]);      // hook the root rx under py
                hooked[k] = true;
            } else {
                atomicCAS(P[k] + rx[k], px[k], py[k]);                 // splice
                rx[k] = px[k];
                px[k] = __ldca(P[k] + rx[k]);
            }
        }
    }
}

constexpr int kCountSlots = 64;

// A warp's members and their roots: equal roots merged (match_any), counted in the block's
// root cache, or straight into the root word when the cache slot belongs to another root.
__device__ __forceinline__ void count_members(bool member, uint32_t root, uint32_t lk, unsigned lane,
                                              uint32_t* P, uint64_t* W, uint32_t* tkey, uint32_t* tcnt,
                                              uint32_t* tmin) {
    const unsigned am = __ballot_sync(0xffffffffu, member);
    if (!member) return;
    const unsigned grp = __match_any_sync(am, root);
    const uint32_t gmin = __reduce_min_sync(grp, lk);
    if (lane != (unsigned)(__ffs(grp) - 1)) return;
    const uint32_t cnt = (uint32_t)__popc(grp);
    const uint32_t h = (root * 0x9E3779B1u) >> (32 - 6);
    uint32_t k = tkey[h];
    if (k == kNone) {
        k = atomicCAS(&tkey[h], kNone, root);
        if (k == kNone) k = root;
    }
    if (k == root) {
        atomicAdd(&tcnt[h], cnt);
        if (gmin != kNone) atomicMin(&tmin[h], gmin);
    } else {
        __stcg(P + root, root | kRootFlag);
        atomicAdd(w_count(W + root), cnt);
        if (gmin != kNone) atomicMin(w_key(W + root), gmin);
    }
}


// grid.y = sketch within the batch.  Full compression, then per root the component size and
// the minimum label key.  Equal roots are merged inside a warp (match_any); each block keeps
// a small direct-mapped cache of roots (claimed by the first root that maps to a slot), so
// the roots that recur within a block -- a giant component's above all -- cost one global
// atomic pair per block, flushed once at its end; other roots are updated in place.  Every
// root that receives members gets kRootFlag on its parent entry (same value from every
// writer), so that the gain pass reads root words only for vertices in components of two or
// more: an unflagged root is a singleton of size 1 whose key is its own.
// key_mode 0: every vertex offers lk(v) = v (the smallest id); 1: only centers offer their
// center index (components without a center need no label); 2: sizes only.
__global__ void __launch_bounds__(256)
k_compress_count(uint32_t* __restrict__ parent, uint64_t* __restrict__ word, uint32_t n,
                 const uint32_t* __restrict__ cidx, int key_mode) {
    __shared__ uint32_t tkey[kCountSlots];
    __shared__ uint32_t tcnt[kCountSlots];
    __shared__ uint32_t tmin[kCountSlots];

    uint32_t* P = parent + (size_t)blockIdx.y * n;
    uint64_t* W = word + (size_t)blockIdx.y * n;
    const unsigned lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kCountSlots; i += blockDim.x) { tkey[i] = kNone; tcnt[i] = 0; tmin[i] = kNone; }
    __syncthreads();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v - threadIdx.x < n; v += stride) {
        const bool act = v < n;
        uint32_t root = 0, lk = kNone;
        bool member = false;   // v stopped being a root: its root must count it
        if (act) {
            root = compress_to_root(P, v);
            member = root != v;
            if (member) lk = label_key(v, key_mode, cidx);
        }
        const unsigned am = __ballot_sync(0xffffffffu, member);
        if (member) {
            const unsigned grp = __match_any_sync(am, root);
            const uint32_t gmin = __reduce_min_sync(grp, lk);
            if (lane == (unsigned)(__ffs(grp) - 1)) {
                const uint32_t cnt = (uint32_t)__popc(grp);
                const uint32_t h = (root * 0x9E3779B1u) >> (32 - 6);
                uint32_t k = tkey[h];
                if (k == kNone) {
                    k = atomicCAS(&tkey[h], kNone, root);
                    if (k == kNone) k = root;
                }
                if (k == root) {
                    atomicAdd(&tcnt[h], cnt);
                    if (gmin != kNone) atomicMin(&tmin[h], gmin);
                } else {
                    __stcg(P + root, root | kRootFlag);
                    atomicAdd(w_count(W + root), cnt);
                    if (gmin != kNone) atomicMin(w_key(W + root), gmin);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCountSlots; i += blockDim.x) {
        const uint32_t rt = tkey[i];
        if (rt != kNone) {
            __stcg(P + rt, rt | kRootFlag);
            atomicAdd(w_count(W + rt), tcnt[i]);
            if (tmin[i] != kNone) atomicMin(w_key(W + rt), tmin[i]);
        }
    }
}

// The same counting with the members gathered first: a warp appends the members of each 32
// vertices it reads (parent != self) to a queue in shared memory and climbs them 32 at a time,
// so the climbs and the root updates run with full warps instead of the few members of each
// group of 32 vertices.
__global__ void __launch_bounds__(256)
k_compress_queue(uint32_t* __restrict__ parent, uint64_t* __restrict__ word, uint32_t n,
                 const uint32_t* __restrict__ cidx, int key_mode) {
    __shared__ uint32_t tkey[kCountSlots];
    __shared__ uint32_t tcnt[kCountSlots];
    __shared__ uint32_t tmin[kCountSlots];
    __shared__ uint32_t queue[8][64];

    uint32_t* P = parent + (size_t)blockIdx.y * n;
    uint64_t* W = word + (size_t)blockIdx.y * n;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* q = queue[warp];
    for (int i = threadIdx.x; i < kCountSlots; i += blockDim.x) { tkey[i] = kNone; tcnt[i] = 0; tmin[i] = kNone; }
    __syncthreads();
    uint32_t qn = 0;   // the same in every lane of the warp
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v - threadIdx.x < n; v += stride) {
        const bool member = v < n && (__ldca(P + v) & kIdMask) != v;
        const unsigned mb = __ballot_sync(0xffffffffu, member);
        if (member) q[qn + __popc(mb & ((1u << lane) - 1u))] = v;
        qn += __popc(mb);
        __syncwarp();
        if (qn >= 32) {
            const uint32_t x = q[lane];
            const uint32_t root = compress_to_root(P, x);
            count_members(true, root, label_key(x, key_mode, cidx), lane, P, W, tkey, tcnt, tmin);
            __syncwarp();
            if (lane + 32 < qn) q[lane] = q[lane + 32];
            qn -= 32;
            __syncwarp();
        }
    }
    {
        const bool member = lane < qn;
        uint32_t root = 0, lk = kNone;
        if (member) {
            const uint32_t x = q[lane];
            root = compress_to_root(P, x);
            lk = label_key(x, key_mode, cidx);
        }
        count_members(member, root, lk, lane, P, W, tkey, tcnt, tmin);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCountSlots; i += blockDim.x) {
        const uint32_t rt = tkey[i];
        if (rt != kNone) {
            __stcg(P + rt, rt | kRootFlag);
            atomicAdd(w_count(W + rt), tcnt[i]);
            if (tmin[i] != kNone) atomicMin(w_key(W + rt), tmin[i]);
        }
    }
}

// sketches whose loads a gain thread keeps in flight together (fewer with overlap sums, whose
// accumulators take the registers)
template <int kSpec> struct GainUnroll { static constexpr int value = kSpec > 0 ? 4 : 8; };

// Initial gains and compact sketches of one batch; with nspec > 0 also the overlap sums of
// the candidate first seeds (their roots per sketch staged in shared memory).  kSpec is the
// capacity of the per-thread overlap accumulators (0, 4 or 8; nspec <= kSpec).
template <bool kAll, int kSpec>
__global__ void __launch_bounds__(256, kSpec > 0 ? 6 : 8)
k_gain_compact(const uint32_t* __restrict__ parent, const uint64_t* __restrict__ word, uint32_t n,
               uint32_t nb, uint32_t r0, uint32_t R, uint64_t* __restrict__ gain, int first,
               const uint32_t* __restrict__ cidx, uint32_t* __restrict__ label,
               uint32_t* __restrict__ size, const uint32_t* __restrict__ spec_ids, uint32_t nspec,
               uint64_t* __restrict__ spec_ov) {
    __shared__ uint32_t sroot[32][kSpec > 0 ? kSpec : 1];
    if (kSpec > 0) {
        for (uint32_t i = threadIdx.x; i < nb * nspec; i += blockDim.x) {
            const uint32_t b = i / nspec, k = i % nspec;
            sroot[b][k] = parent[(size_t)b * n + spec_ids[k]] & kIdMask;
        }
        __syncthreads();
    }
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint64_t g = 0;
        uint64_t ov[kSpec > 0 ? kSpec : 1];
#pragma unroll
        for (int k = 0; k < kSpec; ++k) ov[k] = 0;
        const uint32_t ci = kAll ? v : cidx[v];
        // U sketches at a time: their parent loads, then their root words, are
        // independent, so a thread waits for two memory round trips per group, not per sketch.
        // A singleton (unflagged root of itself) needs no root word: size 1, its own key.
        constexpr int U = GainUnroll<kSpec>::value;
        const uint64_t own = ((uint64_t)ci << 32) | 1u;
        for (uint32_t b0 = 0; b0 < nb; b0 += U) {
            uint32_t rt[U];
            uint64_t wv[U];
#pragma unroll
            for (int j = 0; j < U; ++j) rt[j] = b0 + j < nb ? parent[(size_t)(b0 + j) * n + v] : v;
#pragma unroll
            for (int j = 0; j < U; ++j)
                wv[j] = rt[j] != v ? word[(size_t)(b0 + j) * n + (rt[j] & kIdMask)] : own;
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t b = b0 + j;
                if (b >= nb) break;
                const uint32_t root = rt[j] & kIdMask;
                const uint64_t w = wv[j];
                const uint32_t c = (uint32_t)w;
                g += c;
#pragma unroll
                for (int k = 0; k < kSpec; ++k)
                    if ((uint32_t)k < nspec && root == sroot[b][k]) ov[k] += c;
                if (ci != kNone) {
                    const uint32_t l = (uint32_t)(w >> 32);   // smallest center index of the component
                    const size_t o = (size_t)ci * R + r0 + b;
                    label[o] = l;
                    size[o] = (l == ci) ? c : 0u;
                }
            }
        }
        gain[v] = first ? g : gain[v] + g;
#pragma unroll
        for (int k = 0; k < kSpec; ++k)
            if ((uint32_t)k < nspec && ov[k]) spec_ov[(size_t)k * n + v] += ov[k];
    }
}

// The same when every vertex is a center (full labels): every vertex writes a row segment
// [r0, r0 + nb) of labels and sizes, which one thread per vertex would write 4 bytes at a
// time, R entries apart from its neighbours'.  A block takes tiles of 32 consecutive
// vertices (lane = vertex); warp w reads sketches b = w, w + 8, ... of the batch (coalesced
// parent loads), and the tile's labels and sizes are staged in shared memory, so that each
// row segment is written by one warp in one coalesced store.
constexpr int kGainWarps = 8;

template <int kSpec>
__global__ void __launch_bounds__(kGainWarps * 32)
k_gain_full(const uint32_t* __restrict__ parent, const uint64_t* __restrict__ word, uint32_t n,
            uint32_t nb, uint32_t r0, uint32_t R, uint64_t* __restrict__ gain, int first,
            uint32_t* __restrict__ label, uint32_t* __restrict__ size, const uint32_t* __restrict__ spec_ids,
            uint32_t nspec, uint64_t* __restrict__ spec_ov) {
    constexpr int KS = kSpec > 0 ? kSpec : 1;
    __shared__ uint32_t sroot[32][KS];
    __shared__ uint32_t tl[32][33], ts[32][33];          // [sketch][vertex] of the tile
    __shared__ uint32_t tci[32];                          // the tile's center indices
    __shared__ unsigned long long tg[kGainWarps][32];     // per-warp partial gains
    __shared__ unsigned long long tov[kSpec > 0 ? kGainWarps : 1][KS][32];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (kSpec > 0) {
        for (uint32_t i = threadIdx.x; i < nb * nspec; i += blockDim.x) {
            const uint32_t bb = i / nspec, k = i % nspec;
            sroot[bb][k] = parent[(size_t)bb * n + spec_ids[k]] & kIdMask;
        }
        __syncthreads();
    }
    for (uint32_t v0 = blockIdx.x * 32u; v0 < n; v0 += gridDim.x * 32u) {   // uniform over the block
        const uint32_t v = v0 + lane;
        const bool valid = v < n;
        const uint32_t ci = valid ? v : kNone;
        unsigned long long g = 0;
        unsigned long long ov[KS];
#pragma unroll
        for (int k = 0; k < KS; ++k) ov[k] = 0;
        if (valid) {
            for (uint32_t bb = warp; bb < nb; bb += kGainWarps) {
                const uint32_t pv = parent[(size_t)bb * n + v];
                const uint32_t root = pv & kIdMask;
                const uint64_t w = pv != v ? word[(size_t)bb * n + root] : (((uint64_t)v << 32) | 1u);
                const uint32_t c = (uint32_t)w;
                g += c;
#pragma unroll
                for (int k = 0; k < kSpec; ++k)
                    if ((uint32_t)k < nspec && root == sroot[bb][k]) ov[k] += c;
                if (ci != kNone) {
                    const uint32_t l = (uint32_t)(w >> 32);   // smallest center index of the component
                    tl[bb][lane] = l;
                    ts[bb][lane] = (l == ci) ? c : 0u;
                }
            }
        }
        tg[warp][lane] = g;
#pragma unroll
        for (int k = 0; k < kSpec; ++k) tov[kSpec > 0 ? warp : 0][k][lane] = ov[k];
        if (warp == 0) tci[lane] = ci;
        __syncthreads();
        if (warp == 0 && valid) {
            unsigned long long t = 0;
#pragma unroll
            for (int w = 0; w < kGainWarps; ++w) t += tg[w][lane];
            gain[v] = first ? t : gain[v] + t;
#pragma unroll
            for (int k = 0; k < kSpec; ++k) {
                if ((uint32_t)k >= nspec) continue;
                unsigned long long o = 0;
#pragma unroll
                for (int w = 0; w < kGainWarps; ++w) o += tov[kSpec > 0 ? w : 0][k][lane];
                if (o) spec_ov[(size_t)k * n + v] += o;
            }
        }
        // rows: warp w writes the row segments of the tile's vertices w, w + 8, ...
        for (uint32_t j = warp; j < 32; j += kGainWarps) {
            const uint32_t cj = tci[j];
            if (cj != kNone && lane < nb) {
                const size_t o = (size_t)cj * R + r0 + lane;
                label[o] = tl[lane][j];
                size[o] = ts[lane][j];
            }
        }
        __syncthreads();
    }
}

// The first batch's overlap sums, once the candidates are known (its forest is still there).
__global__ void __launch_bounds__(256)
k_spec_overlap(const uint32_t* __restrict__ parent, const uint64_t* __restrict__ word, uint32_t n,
               uint32_t nb, const uint32_t* __restrict__ spec_ids, uint32_t nspec,
               uint64_t* __restrict__ spec_ov) {
    __shared__ uint32_t sroot[32][kSpecMax];
    for (uint32_t i = threadIdx.x; i < nb * nspec; i += blockDim.x) {
        const uint32_t b = i / nspec, k = i % nspec;
        sroot[b][k] = parent[(size_t)b * n + spec_ids[k]] & kIdMask;
    }
    __syncthreads();
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t ov[kSpecMax];
#pragma unroll
        for (uint32_t k = 0; k < kSpecMax; ++k) ov[k] = 0;
        for (uint32_t b = 0; b < nb; ++b) {
            const uint32_t root = parent[(size_t)b * n + v] & kIdMask;
            bool any = false;
#pragma unroll
            for (uint32_t k = 0; k < kSpecMax; ++k) any |= k < nspec && root == sroot[b][k];
            if (!any) continue;
            const uint32_t c = (uint32_t)word[(size_t)b * n + root];
#pragma unroll
            for (uint32_t k = 0; k < kSpecMax; ++k)
                if (k < nspec && root == sroot[b][k]) ov[k] += c;
        }
#pragma unroll
        for (uint32_t k = 0; k < kSpecMax; ++k)
            if (k < nspec) spec_ov[(size_t)k * n + v] = ov[k];
    }
}

// Candidate first seeds: launch i finds the largest gain key (gain << bits | (2^bits - 1 - v))
// below the one launch i - 1 found (keys are distinct), so keys[0..count) belong to the count
// largest gains, ties to the smaller id; the last launch converts them to ids.
__global__ void __launch_bounds__(256)
k_top_gain(const uint64_t* __restrict__ gain, uint32_t n, uint32_t bits, uint64_t* __restrict__ keys,
           uint32_t i, uint32_t* __restrict__ ids) {
    const uint64_t mask = (1ull << bits) - 1ull;
    const uint64_t bound = i ? keys[i - 1] : ~0ull;
    unsigned long long best = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t k = (gain[v] << bits) | (mask - v);
        if (k < bound && k > best) best = k;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, d));
    if ((threadIdx.x & 31) == 0 && best) atomicMax((unsigned long long*)keys + i, best);
}

__global__ void k_spec_ids(const uint64_t* __restrict__ keys, uint32_t count, uint32_t bits,
                           uint32_t* __restrict__ ids) {
    const uint64_t mask = (1ull << bits) - 1ull;
    if (threadIdx.x < count) ids[threadIdx.x] = (uint32_t)(mask - (keys[threadIdx.x] & mask));
}


// Recomputation evaluator: flag the components that hold a seed (bit 31 of their size).
__global__ void k_cover_roots(const uint32_t* __restrict__ parent, uint64_t* __restrict__ word,
                              uint32_t n, uint32_t nb, const uint32_t* __restrict__ seeds,
                              const unsigned int* __restrict__ nseeds_dev) {
    const uint32_t nseeds = *nseeds_dev;
    const uint32_t total = nb * nseeds;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t b = i / nseeds, sd = seeds[i % nseeds];
        const uint32_t root = parent[(size_t)b * n + sd] & kIdMask;
        atomicOr(w_count(word + (size_t)b * n + root), kCovered);
    }
}

// Monte-Carlo spread of one batch of simulations: every seed's root is flagged (kCovered on
// its root word's size), and the first seed to flag a root adds that component's size.
__global__ void __launch_bounds__(256)
k_mc_cover(const uint32_t* __restrict__ parent, uint64_t* __restrict__ word, uint32_t n, uint32_t nb,
           const uint32_t* __restrict__ seeds, uint32_t k, unsigned long long* __restrict__ total) {
    const uint32_t tasks = nb * k;
    unsigned long long acc = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < tasks; i += gridDim.x * blockDim.x) {
        const uint32_t b = i / k, sd = seeds[i % k];
        const uint32_t root = parent[(size_t)b * n + sd] & kIdMask;
        const uint32_t old = atomicOr(w_count(word + (size_t)b * n + root), kCovered);
        if (!(old & kCovered)) acc += old;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

// Recomputation evaluator: fresh[j] += sum_b size of member j's component unless covered.
__global__ void k_refresh_gather(const uint32_t* __restrict__ parent, const uint64_t* __restrict__ word,
                                 uint32_t n, uint32_t nb, const uint32_t* __restrict__ batch,
                                 const unsigned int* __restrict__ batch_n,
                                 unsigned long long* __restrict__ fresh) {
    const uint32_t bn = *batch_n;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < bn; j += gridDim.x * blockDim.x) {
        const uint32_t x = batch[j];
        unsigned long long d = 0;
        for (uint32_t b = 0; b < nb; ++b) {
            const uint32_t c = (uint32_t)word[(size_t)b * n + (parent[(size_t)b * n + x] & kIdMask)];
            d += (c & kCovered) ? 0u : c;
        }
        fresh[j] += d;
    }
}

__global__ void k_labels_out(const uint32_t* __restrict__ P, const uint64_t* __restrict__ W, uint32_t n,
                             uint32_t* __restrict__ out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = (uint32_t)(W[P[v] & kIdMask] >> 32);
}

// ---- centers: the rho smallest ckey(v) = mix(v ^ csalt) (distinct: mix is a bijection) ----
// Radix selection of the need-th smallest 64-bit key, 8 bits per pass from the top: a pass
// histograms the digit of the keys that match the prefix chosen so far, and the last of its
// blocks (ticket) picks the digit that holds the need-th key.
struct CenterSel {
    unsigned long long prefix, prefmask, need;
    int shift;
    unsigned int ticket;
    unsigned int hist[256];
};

__global__ void k_center_init(CenterSel* st, uint32_t need) {
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->prefmask = 0;
        st->need = need;
        st->shift = 56;
        st->ticket = 0;
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) st->hist[i] = 0;
}

__global__ void k_center_flags(uint32_t n, uint64_t csalt, const CenterSel* st,
                               uint32_t* __restrict__ flags, uint32_t* __restrict__ cbits) {
    const unsigned long long theta = st->prefix;   // the rho-th smallest key
    // blockDim.x is a multiple of 32, so every warp covers one aligned 32-vertex word
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        bool f = false;
        if (v < n) f = mix64((uint64_t)v ^ csalt) <= theta;
        unsigned bal = __ballot_sync(0xffffffffu, f);
        if (v < n) flags[v] = f ? 1u : 0u;
        if ((threadIdx.x & 31) == 0 && v < n) cbits[v >> 5] = bal;
    }
}

__global__ void k_center_index(uint32_t n, uint32_t rho, const uint32_t* __restrict__ flags,
                               const uint64_t* __restrict__ pos, uint32_t* __restrict__ cidx,
                               uint32_t* __restrict__ centers) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (flags[v] && pos[v] < rho) {
            uint32_t i = (uint32_t)pos[v];
            cidx[v] = i;
            centers[i] = v;
        } else {
            cidx[v] = kNone;
        }
    }
}


// ---- hubs: high-degree non-centers that the searches treat as centers -----------------
// GetCenter from a vertex whose component reaches a high-degree vertex tests that vertex's
// whole adjacency list unless it is a center -- nearly every time when its edges have small
// probabilities (the weighted cascade).  The hubs, at most hub_rows non-centers of degree
// >= min_deg with the largest degrees (ties to the smaller id), get label / size rows of
// their own after the rho compact rows (index rho + i) and are offered to the union-find's
// minimum like centers.  A component's key is then its smallest center index if it has a
// center, else its smallest hub index: every search that meets one of its centers or hubs
// reads the same size row, which MarkSeed flags.  Rows [0, rho) stay the compact sketch of
// Sec. 3 bit for bit; the hub rows only shorten searches and change no value.
__device__ __forceinline__ uint64_t hub_key(uint32_t v, const uint64_t* __restrict__ off,
                                            const uint32_t* __restrict__ cidx, uint32_t min_deg) {
    if (cidx[v] != kNone) return ~0ull;   // a center already
    const uint64_t d = off[v + 1] - off[v];
    if (d < min_deg) return ~0ull;        // min_deg >= 1, so every eligible key is below ~0
    const uint32_t dd = d >= 0xFFFFFFFFull ? 0xFFFFFFFEu : (uint32_t)d;
    return ((uint64_t)(0xFFFFFFFFu - dd) << 32) | v;
}

// One pass of the radix selection over the center keys (kHub = false) or the hub keys.
template <bool kHub>
__global__ void __launch_bounds__(256)
k_select_pass(uint32_t n, uint64_t csalt, const uint64_t* __restrict__ off, const uint32_t* __restrict__ cidx,
              uint32_t min_deg, CenterSel* st) {
    __shared__ unsigned int h[256];
    __shared__ unsigned int wsum[8];
    __shared__ unsigned int s_last, s_d;
    __shared__ unsigned long long s_cum;
    const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;   // blockDim.x == 256
    h[tid] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix, pm = st->prefmask;
    const int shift = st->shift;
    for (uint32_t v = blockIdx.x * blockDim.x + tid; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t key = kHub ? hub_key(v, off, cidx, min_deg) : mix64((uint64_t)v ^ csalt);
        if ((key & pm) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[tid]) atomicAdd(&st->hist[tid], h[tid]);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    // the last block: every block's counts are in st->hist
    __threadfence();
    const unsigned cnt = __ldcg(&st->hist[tid]);
    unsigned incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, d);
        if ((int)lane >= d) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    if (tid == 0) s_d = 255;
    __syncthreads();
    for (unsigned w = 0; w < warp; ++w) incl += wsum[w];
    const unsigned long long need = st->need;
    // the digit: the first bin whose inclusive count reaches need (bin 255 if none before it)
    if (tid < 255 && incl >= need && incl - cnt < need) s_d = tid;
    __syncthreads();
    if (tid == s_d) s_cum = incl - cnt;
    __syncthreads();
    if (tid == 0) {
        st->need = need - s_cum;
        st->prefix = prefix | ((unsigned long long)s_d << shift);
        st->prefmask = pm | (255ull << shift);
        st->shift = shift - 8;
        st->ticket = 0;
    }
    st->hist[tid] = 0;
}

__global__ void k_hub_flags(uint32_t n, const uint64_t* __restrict__ off, const uint32_t* __restrict__ cidx,
                            uint32_t min_deg, const CenterSel* st, uint32_t* __restrict__ flags,
                            uint32_t* __restrict__ cbits) {
    const unsigned long long theta = st->prefix;   // the hub_rows-th smallest key
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        bool f = false;
        if (v < n) {
            const uint64_t key = hub_key(v, off, cidx, min_deg);
            f = key <= theta && key != ~0ull;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (v < n) flags[v] = f ? 1u : 0u;
        if ((threadIdx.x & 31) == 0 && v < n && bal) cbits[v >> 5] |= bal;   // this warp's word
    }
}

__global__ void k_hub_index(uint32_t n, uint32_t rho, const uint32_t* __restrict__ flags,
                            const uint64_t* __restrict__ pos, uint32_t* __restrict__ cidx) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (flags[v]) cidx[v] = rho + (uint32_t)pos[v];
}

// Blocks of the sampling kernel per SM (grid-stride over the edge pairs): 8 leave the other
// lane's union-find kernels some room (Chung-Lu step 7.62 -> 7.56 ms against 16).
constexpr unsigned kEmitBlocksPerSM = 8;

// Sampling and unions of one batch as two kernels (records of live pairs in between).
int launch_sample_split(im_ctx* c, im_ctx::Lane& L, uint32_t r0, uint32_t nb, int key_mode) {
    const unsigned T = 256;
    const uint64_t npairs = (c->m + 1) >> 1;
    const uint4* ep = reinterpret_cast<const uint4*>(c->d_edges);
    const unsigned gs = grid_for(npairs, T, 152u * kEmitBlocksPerSM);
    const double pl = c->smp.eT ? c->mean_p : c->smp.all_live ? 1.0 : c->p;
    const unsigned gu = grid_for((uint64_t)(pl * (double)c->m * nb) + 1, T, 152u * 16u);
    const uint64_t live_cap = im_record_cap(c->live_cap);
    // bucketed records: 8 bytes each, one region per (sketch, sampling block) in the lane's record
    // buffer; counts and the overflow flag in the lane's counter array
    const uint32_t B_ = c->batch_used ? c->batch_used : 1;
    // the bucketed sampler runs 4 blocks per SM: the other lane's union-find kernels then find
    // room beside it (124 against 127 ms per step on R-MAT scale 24 with 16 blocks per SM)
    const unsigned gsb = grid_for(npairs, T, 152u * kBucketBlocksPerSM);
    const uint32_t capr = (uint32_t)std::min<uint64_t>(2 * live_cap / ((uint64_t)B_ * gsb), 0xFFFFFFFFull);
    uint2* buckets = reinterpret_cast<uint2*>(L.live);
    uint32_t* region_n = reinterpret_cast<uint32_t*>(L.live_n) + 8;   // after the flag words
    unsigned int* overflow = reinterpret_cast<unsigned int*>(L.live_n);
    // union blocks: rpb consecutive regions of one sketch, about 32K records per block (fewer,
    // longer blocks: 124 against 137 ms per step on R-MAT scale 24 with one region per block),
    // but at least 8 blocks per SM in all, so that smaller graphs still fill the GPU
    const double per_region = std::max(1.0, pl * (double)c->m / gsb);
    const double rpb_fill = std::floor((double)gsb * nb / (152.0 * 8.0));
    const uint32_t rpb = (uint32_t)std::min({64.0, std::max(1.0, std::round(32768.0 / per_region)),
                                             std::max(1.0, rpb_fill)});
    const unsigned gub = ((gsb + rpb - 1) / rpb) * nb;
#define IM_SE(BB)                                                                                 \
    do {                                                                                          \
        if (c->union_used == IM_UNION_BUCKETS) {                                                  \
            IM_LAUNCH(c, K_SAMPLE_EMIT, k_sample_bucket<BB>, gsb, T, 0, ep, c->m, c->smp, r0, nb,    \
                      buckets, region_n, capr, overflow, L.parent, L.word, c->n, c->d_cidx, key_mode); \
            IM_LAUNCH(c, K_UNION, k_union_bucket<BB>, gub, T, 0, buckets, region_n, gsb, rpb, capr,     \
                      overflow, L.parent, c->n, ep, c->m, c->smp, r0, nb, c->d_live_total);       \
            break;                                                                                \
        }                                                                                         \
        IM_LAUNCH(c, K_SAMPLE_EMIT, k_sample_emit<BB>, gs, T, 0, ep, c->m, c->smp, r0, nb, L.live,   \
                  L.live_n, live_cap, L.parent, L.word, c->n, c->d_cidx, key_mode);                \
        IM_LAUNCH(c, K_UNION, k_union_live<BB>, gu, T, 0, L.live, L.live_n, live_cap, L.parent,    \
                  c->n, ep, c->m, c->smp, r0, nb, c->d_live_total);                               \
    } while (0)
    const uint32_t cap = c->batch_used;
    if (cap <= 1) IM_SE(1);
    else if (cap <= 2) IM_SE(2);
    else if (cap <= 4) IM_SE(4);
    else if (cap <= 8) IM_SE(8);
    else if (cap <= 16) IM_SE(16);
    else IM_SE(32);
#undef IM_SE
    return IM_OK;
}

int launch_sample_fused(im_ctx* c, im_ctx::Lane& L, uint32_t r0, uint32_t nb) {
    const unsigned T = 256;
    const uint64_t npairs = (c->m + 1) >> 1;
    const unsigned grid = grid_for(npairs, T, 152u * 16u);
    const uint4* ep = reinterpret_cast<const uint4*>(c->d_edges);
    IM_LAUNCH(c, K_SAMPLE_UNION, k_sample_union<1>, grid, T, 0, ep, c->m, c->smp, r0, nb, L.parent, c->n);
    return IM_OK;
}

// Sampling and unions of one batch in one kernel (k_sample_unite), after the forest
// initialisation.  The grid is what the SMs hold at once: each warp's queue of live pairs
// lives as long as the warp.
int launch_sample_unite(im_ctx* c, im_ctx::Lane& L, uint32_t r0, uint32_t nb) {
    const uint64_t npairs = (c->m + 1) >> 1;
    const uint4* ep = reinterpret_cast<const uint4*>(c->d_edges);
    const unsigned T = kUniteWarps * 32;
#define IM_SU(BB)                                                                                    \
    do {                                                                                             \
        static int per_sm = 0;                                                                       \
        if (per_sm == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_unite<BB>, T, 0) \
                               != cudaSuccess) per_sm = 4;                                           \
        if (per_sm < 1) per_sm = 1;                                                                  \
        const unsigned g = grid_for(npairs, T, 152u * (unsigned)per_sm);                             \
        IM_LAUNCH(c, K_SAMPLE_UNION, k_sample_unite<BB>, g, T, 0, ep, c->m, c->smp, r0, nb, L.parent, c->n, \
                  c->d_live_total);                                                                  \
    } while (0)
    const uint32_t cap = c->batch_used;
    if (cap <= 1) IM_SU(1);
    else if (cap <= 2) IM_SU(2);
    else if (cap <= 4) IM_SU(4);
    else if (cap <= 8) IM_SU(8);
    else if (cap <= 16) IM_SU(16);
    else IM_SU(32);
#undef IM_SU
    return IM_OK;
}

// init + sampling + unions + compression of sketches r0 .. r0+nb-1 in lane L (on c->cur)
int batch_components(im_ctx* c, im_ctx::Lane& L, uint32_t r0, uint32_t nb, int key_mode) {
    const uint32_t n = c->n;
    const unsigned T = 256;
    const bool sample = (c->smp.eT || c->smp.all_live || c->smp.T != 0) && c->m > 0;
    if (sample && c->union_used == IM_UNION_FUSED && nb <= c->batch_used) {
        IM_LAUNCH(c, K_BATCH_INIT, k_forest_init, dim3(grid_for(n, T, (152u * 16u + nb - 1) / nb), nb), T, 0,
                  L.parent, L.word, n, c->d_cidx, key_mode);
        const int rc = launch_sample_unite(c, L, r0, nb);
        if (rc) return rc;
    } else {
        const bool split = sample && L.live && nb <= c->batch_used;   // the emit kernel initialises
        if (!split)
            IM_LAUNCH(c, K_BATCH_INIT, k_batch_init, grid_for((uint64_t)n * nb, T, 152u * 16u), T, 0,
                      L.parent, L.word, n, nb, c->d_cidx, key_mode);
        if (sample) {
            const int rc = split ? launch_sample_split(c, L, r0, nb, key_mode) : launch_sample_fused(c, L, r0, nb);
            if (rc) return rc;
        }
    }
    // about 8 blocks per SM in all: each block sweeps a stretch of one sketch
    dim3 g(std::max(1u, std::min(grid_for(n, T), (152u * 8u + nb - 1) / nb)), nb);
    // the queued form is faster alone (R-MAT scale 24, one lane: 18.4 -> 12.4 ms per build;
    // Chung-Lu step 8.21 -> 7.73 ms), but beside the bucketed path's sampling on the other lane
    // the step measured slower (125.8 against 123.9 ms), so that path keeps the in-place form
    if (c->union_used == IM_UNION_BUCKETS)
        IM_LAUNCH(c, K_COMPRESS_COUNT, k_compress_count, g, T, 0, L.parent, L.word, n, c->d_cidx, key_mode);
    else
        IM_LAUNCH(c, K_COMPRESS_COUNT, k_compress_queue, g, T, 0, L.parent, L.word, n, c->d_cidx, key_mode);
    return IM_OK;
}

__global__ void k_add_u64(unsigned long long* __restrict__ dst, const unsigned long long* __restrict__ src,
                          uint64_t count, const unsigned int* __restrict__ count_dev) {
    const uint64_t cnt = count_dev ? *count_dev : count;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] += src[i];
}

// Lanes 1.. start after everything queued so far on the context stream ...
int lanes_fork(im_ctx* c, uint32_t lanes) {
    IM_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    for (uint32_t i = 1; i < lanes; ++i) IM_CUDA(c, cudaStreamWaitEvent(c->lane_stream[i], c->ev_fork, 0));
    return IM_OK;
}

// ... and the context stream continues after everything queued on the other lanes.
int lanes_join(im_ctx* c, uint32_t lanes) {
    c->cur = c->stream;
    for (uint32_t i = 1; i < lanes; ++i) {
        IM_CUDA(c, cudaEventRecord(c->ev_join[i], c->lane_stream[i]));
        IM_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join[i], 0));
    }
    return IM_OK;
}

}  // namespace


int im_select_centers(im_ctx* c, uint32_t* d_flags, uint64_t* d_pos) {
    static_assert(sizeof(CenterSel) <= kCenterSelBytes, "center select scratch");
    const uint32_t n = c->n;
    CenterSel* st = reinterpret_cast<CenterSel*>(c->d_csel);
    const uint64_t csalt = mix64(c->seed ^ 0xC3ull);
    const unsigned T = 256;
    IM_LAUNCH(c, K_CENTER_PICK, k_center_init, 1, 256, 0, st, c->rho);
    for (int pass = 0; pass < 8; ++pass)
        IM_LAUNCH(c, K_CENTER_HIST, k_select_pass<false>, grid_for(n, T, 152u * 4u), T, 0, n, csalt,
                  (const uint64_t*)nullptr, (const uint32_t*)nullptr, 0u, st);
    IM_LAUNCH(c, K_CENTER_FLAGS, k_center_flags, grid_for(n, T, 152u * 8u), T, 0, n, csalt, st,
              d_flags, c->d_cbits);
    const int rc = im_scan_u32_to_u64(c, d_flags, d_pos, n);
    if (rc) return rc;
    IM_LAUNCH(c, K_CENTER_INDEX, k_center_index, grid_for(n, T, 152u * 8u), T, 0, n, c->rho, d_flags, d_pos,
              c->d_cidx, c->d_centers);
    IM_CUDA(c, cudaGetLastError());
    return IM_OK;
}

// Hubs after the centers (kernels above); their count goes to the pinned word h_live[2].
int im_select_hubs(im_ctx* c, uint32_t* d_flags, uint64_t* d_pos) {
    const uint32_t n = c->n;
    if (c->hub_rows == 0) {
        c->h_live[2] = 0;
        return IM_OK;
    }
    CenterSel* st = reinterpret_cast<CenterSel*>(c->d_csel);
    const unsigned T = 256;
    const uint32_t md = c->hub_min_deg ? c->hub_min_deg : 1u;
    IM_LAUNCH(c, K_CENTER_PICK, k_center_init, 1, 256, 0, st, c->hub_rows);
    for (int pass = 0; pass < 8; ++pass)
        IM_LAUNCH(c, K_CENTER_HIST, k_select_pass<true>, grid_for(n, T, 152u * 4u), T, 0, n, 0ull, c->d_off,
                  c->d_cidx, md, st);
    IM_LAUNCH(c, K_CENTER_FLAGS, k_hub_flags, grid_for(n, T, 152u * 8u), T, 0, n, c->d_off, c->d_cidx, md, st,
              d_flags, c->d_cbits);
    const int rc = im_scan_u32_to_u64(c, d_flags, d_pos, n);
    if (rc) return rc;
    IM_LAUNCH(c, K_CENTER_INDEX, k_hub_index, grid_for(n, T, 152u * 8u), T, 0, n, c->rho, d_flags, d_pos,
              c->d_cidx);
    IM_CUDA(c, cudaMemcpyAsync(c->h_live + 2, d_pos + n, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               c->stream));
    IM_CUDA(c, cudaGetLastError());
    return IM_OK;
}

// Build all R sketches batch by batch; writes gain0, label, size.  Batch i runs on lane
// i mod lanes; lanes 1.. accumulate their gains (and overlap sums) separately, added at the end.
int im_sketch_batches(im_ctx* c) {
    const uint32_t n = c->n, R = c->R, lanes = c->lanes;
    const unsigned T = 256;
    int rc = lanes_fork(c, lanes);
    if (rc) return rc;
    // lanes 1.. sum their overlaps in buffers of their own
    for (uint32_t li = 1; li < lanes && c->spec_count; ++li)
        IM_CUDA(c, cudaMemsetAsync(c->lane[li].spec_ov, 0, (size_t)c->spec_count * n * sizeof(uint64_t),
                                   c->lane_stream[li]));
    uint32_t i = 0;
    for (uint32_t r0 = 0; r0 < R; r0 += c->batch_used, ++i) {
        const uint32_t nb = R - r0 < c->batch_used ? R - r0 : c->batch_used;
        const uint32_t li = i % lanes;
        im_ctx::Lane& L = c->lane[li];
        c->cur = L.stream;
        rc = batch_components(c, L, r0, nb, c->all_centers ? 0 : 1);
        if (rc) { lanes_join(c, lanes); return rc; }
        uint64_t* gain = li ? L.gain : c->d_gain0;
        const int first = i < lanes ? 1 : 0;
        const uint32_t nspec = i ? c->spec_count : 0;   // candidates are known after batch 0
        // the candidates come from batch 0 (lane 0): another lane's first gain pass waits for them
        if (nspec && li && i < lanes) IM_CUDA(c, cudaStreamWaitEvent(c->cur, c->ev_spec, 0));
#define IM_GAIN(ALL, K)                                                                             \
    if (ALL)                                                                                        \
        IM_LAUNCH(c, K_GAIN_COMPACT, (k_gain_full<K>), grid_for(n, 32, 152u * 8u), kGainWarps * 32, 0, L.parent, \
                  L.word, n, nb, r0, R, gain, first, c->d_label, c->d_size, c->d_spec_ids, nspec,       \
                  L.spec_ov);                                                                       \
    else                                                                                            \
        IM_LAUNCH(c, K_GAIN_COMPACT, (k_gain_compact<false, K>), grid_for(n, T, 152u * 16u), T, 0, L.parent,   \
                  L.word, n, nb, r0, R, gain, first, c->d_cidx, c->d_label, c->d_size, c->d_spec_ids, nspec, \
                  L.spec_ov)
        if (c->all_centers) {
            if (nspec == 0) IM_GAIN(true, 0);
            else if (nspec <= 4) IM_GAIN(true, 4);
            else IM_GAIN(true, 8);
        } else {
            if (nspec == 0) IM_GAIN(false, 0);
            else if (nspec <= 4) IM_GAIN(false, 4);
            else IM_GAIN(false, 8);
        }
#undef IM_GAIN
        if (i == 0 && c->spec_count) {
            // candidate first seeds: the largest gains so far; then this batch's overlap sums
            IM_CUDA(c, cudaMemsetAsync(c->d_spec_keys, 0, kSpecMax * sizeof(uint64_t), c->cur));
            for (uint32_t k = 0; k < c->spec_count; ++k)
                IM_LAUNCH(c, K_CENTER_HIST, k_top_gain, grid_for(n, T, 152u * 8u), T, 0, c->d_gain0, n, c->key_bits,
                          c->d_spec_keys, k, c->d_spec_ids);
            IM_LAUNCH(c, K_CENTER_PICK, k_spec_ids, 1, 32, 0, c->d_spec_keys, c->spec_count, c->key_bits,
                      c->d_spec_ids);
            IM_CUDA(c, cudaEventRecord(c->ev_spec, c->cur));   // the candidates are known
            IM_LAUNCH(c, K_GAIN_COMPACT, k_spec_overlap, grid_for(n, T, 152u * 16u), T, 0, L.parent, L.word, n, nb,
                      c->d_spec_ids, c->spec_count, c->lane[0].spec_ov);
        }
    }
    rc = lanes_join(c, lanes);
    if (rc) return rc;
    for (uint32_t li = 1; li < lanes && li < i; ++li) {   // the lanes that ran a batch
        IM_LAUNCH(c, K_GAIN_COMPACT, k_add_u64, grid_for(n, T, 152u * 8u), T, 0,
                  (unsigned long long*)c->d_gain0, (const unsigned long long*)c->lane[li].gain, (uint64_t)n,
                  (const unsigned int*)nullptr);
        if (c->spec_count)
            IM_LAUNCH(c, K_GAIN_COMPACT, k_add_u64, grid_for((uint64_t)c->spec_count * n, T, 152u * 8u), T, 0,
                      (unsigned long long*)c->lane[0].spec_ov, (const unsigned long long*)c->lane[li].spec_ov,
                      (uint64_t)c->spec_count * n, (const unsigned int*)nullptr);
    }
    IM_CUDA(c, cudaGetLastError());
    return IM_OK;
}

// Min-id labels of one sketch (test hook): the component minimum of lk(v) = v.
int im_labels_min(im_ctx* c, uint32_t r, uint32_t* d_out) {
    const uint32_t n = c->n;
    const unsigned T = 256;
    c->cur = c->stream;
    int rc = batch_components(c, c->lane[0], r, 1, 0);
    if (rc) return rc;
    IM_LAUNCH(c, K_LABELS_OUT, k_labels_out, grid_for(n, T, 152u * 8u), T, 0, c->lane[0].parent,
              c->lane[0].word, n, d_out);
    IM_CUDA(c, cudaGetLastError());
    return IM_OK;
}

// Batched re-evaluation by recomputation: for every batch member x, Marginal(S, x) =
// sum_r [C_r(x) holds no seed] |C_r(x)|, obtained by recomputing each sketch's components
// (Sketch(r) of Alg. 3) instead of one search per (x, r).  Same values as GetCenter; cheaper
// when the batch is a large part of V.  The batch list and its size live on the device.
int im_refresh_eval(im_ctx* c, const uint32_t* d_batch, const unsigned int* d_batch_n,
                    unsigned long long* d_fresh, const uint32_t* d_seeds, const unsigned int* d_nseeds) {
    const uint32_t n = c->n, R = c->R;
    const unsigned T = 256;
    // The member count and the seed count are read on the device, so the launches do not
    // depend on them and the sequence can be captured in the selection graph.  Captured, it
    // stays on the capturing stream (one lane); otherwise the lanes alternate.
    const uint32_t lanes = (c->capturing || c->count_only) ? 1u : c->lanes;
    cudaStream_t s0 = c->cur;
    int rc = IM_OK;
    if (lanes > 1) {
        rc = lanes_fork(c, lanes);
        if (rc) return rc;
        for (uint32_t li = 1; li < lanes; ++li)
            IM_CUDA(c, cudaMemsetAsync(c->lane[li].fresh, 0, (size_t)n * sizeof(uint64_t), c->lane_stream[li]));
    }
    uint32_t i = 0;
    for (uint32_t r0 = 0; r0 < R; r0 += c->batch_used, ++i) {
        const uint32_t nb = R - r0 < c->batch_used ? R - r0 : c->batch_used;
        const uint32_t li = i % lanes;
        im_ctx::Lane& L = c->lane[li];
        c->cur = li ? c->lane_stream[li] : s0;
        rc = batch_components(c, L, r0, nb, 2);
        if (rc) break;
        IM_LAUNCH(c, K_COVER_ROOTS, k_cover_roots, 152u * 4u, T, 0, L.parent, L.word, n, nb, d_seeds,
                  d_nseeds);
        IM_LAUNCH(c, K_REFRESH_GATHER, k_refresh_gather, grid_for(n, T, 152u * 16u), T, 0,
                  L.parent, L.word, n, nb, d_batch, d_batch_n, li ? L.fresh : d_fresh);
    }
    c->cur = s0;
    if (lanes > 1) {
        const int rj = lanes_join(c, lanes);
        if (!rc) rc = rj;
        for (uint32_t li = 1; li < lanes && li < i && !rc; ++li)
            IM_LAUNCH(c, K_REFRESH_GATHER, k_add_u64, grid_for(n, T, 152u * 8u), T, 0, d_fresh,
                      (const unsigned long long*)c->lane[li].fresh, (uint64_t)0, d_batch_n);
    }
    return rc;
}

// Monte-Carlo influence of the seeds d_seeds[0..k): simulation r is the live-edge world of
// sketch index r under the edge hash of `mc_seed` (the sketches' hash reading with another
// seed) and the context's probabilities; *d_total += sum_r |union of the seeds' components|.
// Runs batch by batch on lane 0 with the build's scratch.
int im_mc_run(im_ctx* c, const uint32_t* d_seeds, uint32_t k, uint32_t sims, uint64_t mc_seed,
              unsigned long long* d_total) {
    const Sampler saved = c->smp;
    c->smp.salt = mix64(mc_seed + kGamma);
    c->cur = c->stream;
    int rc = IM_OK;
    for (uint32_t r0 = 0; r0 < sims && !rc; r0 += c->batch_used) {
        const uint32_t nb = sims - r0 < c->batch_used ? sims - r0 : c->batch_used;
        im_ctx::Lane& L = c->lane[0];
        rc = batch_components(c, L, r0, nb, 2);
        if (!rc && k > 0)
            IM_LAUNCH(c, K_COVER_ROOTS, k_mc_cover, grid_for((uint64_t)nb * k, 256, 152u * 4u), 256, 0, L.parent,
                      L.word, c->n, nb, d_seeds, k, d_total);
    }
    c->smp = saved;
    return rc;
}
