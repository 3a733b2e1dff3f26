// im_graph.cu -- graph load: edge packing with validation, CSR build (Sec. 5 stores the
// input as CSR), and the exclusive scan used for CSR offsets and center indices.
#include "im_internal.cuh"

using namespace imk;

namespace {

// Pack (u[e], v[e]) into one 8-byte record; flag ids >= n and self-loops.
__global__ void k_pack_edges(const uint32_t* __restrict__ u, const uint32_t* __restrict__ v,
                             uint64_t m, uint32_t n, uint2* __restrict__ edges,
                             unsigned int* __restrict__ bad) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint32_t a = u[e], b = v[e];
        if (a >= n || b >= n || a == b) {
            // reported, and replaced by the self-loop (0, 0), which every later kernel handles in
            // bounds (a union of 0 with itself does nothing): a graph queued before the host reads
            // the flag (im_batch_run) stays memory-safe, and its instance then fails
            atomicOr(bad, 1u);
            a = b = 0;
        }
        edges[e] = make_uint2(a, b);
    }
}

// Degrees; equal endpoints within a warp share one atomic, so a hub's counter (and edges
// sorted by their first endpoint) do not serialise the whole kernel.
__device__ __forceinline__ void add_degree(bool valid, uint32_t x, uint32_t* __restrict__ deg) {
    const unsigned key = valid ? x : 0xFFFFFFFFu;   // ids are < 2^31
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (valid && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(deg + x, (unsigned)__popc(grp));
}

// Runs before the host has read k_pack_edges' verdict, so edges with an id >= n (which fail
// the build afterwards) are skipped here rather than counted out of bounds.
__global__ void __launch_bounds__(256)
k_csr_degree(const uint2* __restrict__ edges, uint64_t m, uint32_t n, uint32_t* __restrict__ deg) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // the loop bound is uniform over the block, so the warp-wide calls have all lanes
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const uint64_t e = base + threadIdx.x;
        uint2 ed = make_uint2(0, 0);
        if (e < m) ed = edges[e];
        const bool valid = e < m && ed.x < n && ed.y < n;
        add_degree(valid, ed.x, deg);
        add_degree(valid, ed.y, deg);
    }
}

// Every build rewrites the arcs (x -> y) of each edge e: (y | center bit << 31, center index
// of y (kNone if y is no center), key lo, key hi) with the per-edge hash key mix(salt ^ e) (Sec. 2 fusion: the sampling of edge e in
// sketch r is then one more mix of key + (r+1) G) and whether y is a center, so a search
// step needs no other lookup (a search that meets a center reads its label directly).  Inside each adjacency list the arcs to centers come first
// (cursor ccur from the front, ncur from the back): GetCenter stops at the first live center
// it meets, and on a hub it then meets one after ~1/p arcs instead of ~1/(p alpha).  The
// order inside each group is arrival order; no result depends on the order of an adjacency
// list (every center of a component carries the component's label, and a search without a
// center visits the whole component).  Arcs of one source in a warp share one atomic.
__device__ __forceinline__ uint64_t arc_slot(bool valid, uint32_t x, bool to_center,
                                             const uint64_t* __restrict__ off, uint32_t* __restrict__ ccur,
                                             uint32_t* __restrict__ ncur) {
    // x < 2^31, so (x << 1) | c never equals the key of an idle lane
    const unsigned key = valid ? ((x << 1) | (to_center ? 1u : 0u)) : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(grp) - 1;
    const unsigned rank = __popc(grp & ((1u << (threadIdx.x & 31)) - 1u));
    uint32_t base = 0;
    if (valid && (int)(threadIdx.x & 31) == leader)
        base = atomicAdd(to_center ? ccur + x : ncur + x, (unsigned)__popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader) + rank;
    if (!valid) return 0;
    return to_center ? off[x] + base : off[x + 1] - 1 - base;
}

// The static adjacency of a loaded graph (once per graph): every arc's neighbour and edge id
// at a slot of its source's CSR range, and the source itself, so that the per-build fill can
// stream the arcs in CSR order (consecutive arcs share their source).
__global__ void __launch_bounds__(256)
k_adj_fill(const uint2* __restrict__ edges, uint64_t m, const uint64_t* __restrict__ off,
           uint32_t* __restrict__ cur, uint2* __restrict__ adj, uint32_t* __restrict__ src) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // the loop bound is uniform over the block, so every warp-wide call has all lanes
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const uint64_t e = base + threadIdx.x;
        const bool valid = e < m;
        uint2 ed = make_uint2(0, 0);
        if (valid) ed = edges[e];
        const uint64_t pa = arc_slot(valid, ed.x, true, off, cur, cur);
        const uint64_t pb = arc_slot(valid, ed.y, true, off, cur, cur);
        if (valid) {
            adj[pa] = make_uint2(ed.y, (uint32_t)e);
            adj[pb] = make_uint2(ed.x, (uint32_t)e);
            src[pa] = ed.x;
            src[pb] = ed.y;
        }
    }
}

// The static adjacency of a large graph in two passes, so that the scatter into adjacency
// lists stays in L2: k_adj_bin groups the arcs by source range (kAdjBins ranges of width V),
// each range's arcs written to that range's own CSR span [off[b V], off[(b+1) V]) of a
// scratch array (the build's arc array, not yet in use at load time); k_adj_place then takes
// the binned arcs in order, so that the blocks running at any moment place the arcs of one or
// two source ranges, whose cursors, offsets and adjacency slots (tens of MB) stay in L2.  A
// tile of kAdjTileEdges edges per block reserves room per range with one global atomic per
// range (counted in shared memory first).
constexpr uint32_t kAdjBins = 256;
constexpr uint32_t kAdjEdgesPerThread = 4;

__global__ void k_adj_bin_init(const uint64_t* __restrict__ off, uint32_t n, uint32_t V,
                               unsigned long long* __restrict__ bcur) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < kAdjBins) bcur[b] = off[min((uint64_t)b * V, (uint64_t)n)];
}

__global__ void __launch_bounds__(256)
k_adj_bin(const uint2* __restrict__ edges, uint64_t m, uint32_t V, unsigned long long* __restrict__ bcur,
          uint4* __restrict__ binned) {
    __shared__ uint32_t hist[kAdjBins];
    __shared__ unsigned long long base[kAdjBins];
    const uint64_t tile = (uint64_t)blockDim.x * kAdjEdgesPerThread;
    for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < m; t0 += (uint64_t)gridDim.x * tile) {
        for (uint32_t i = threadIdx.x; i < kAdjBins; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        uint2 ed[kAdjEdgesPerThread];
        uint32_t rk[2 * kAdjEdgesPerThread];
#pragma unroll
        for (uint32_t j = 0; j < kAdjEdgesPerThread; ++j) {
            const uint64_t e = t0 + (uint64_t)j * blockDim.x + threadIdx.x;   // coalesced
            ed[j] = e < m ? edges[e] : make_uint2(0, 0);
            if (e < m) {
                rk[2 * j] = atomicAdd(&hist[ed[j].x / V], 1u);
                rk[2 * j + 1] = atomicAdd(&hist[ed[j].y / V], 1u);
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kAdjBins; i += blockDim.x)
            base[i] = hist[i] ? atomicAdd(&bcur[i], (unsigned long long)hist[i]) : 0ull;
        __syncthreads();
#pragma unroll
        for (uint32_t j = 0; j < kAdjEdgesPerThread; ++j) {
            const uint64_t e = t0 + (uint64_t)j * blockDim.x + threadIdx.x;
            if (e < m) {
                const uint32_t x = ed[j].x, y = ed[j].y;
                binned[base[x / V] + rk[2 * j]] = make_uint4(x, y, (uint32_t)e, (uint32_t)(e >> 32));
                binned[base[y / V] + rk[2 * j + 1]] = make_uint4(y, x, (uint32_t)e, (uint32_t)(e >> 32));
            }
        }
        __syncthreads();
    }
}

// Arcs in CSR order of their source ranges; each goes to a slot of its source's list.
__global__ void __launch_bounds__(256)
k_adj_place(const uint4* __restrict__ binned, uint64_t narcs, const uint64_t* __restrict__ off,
            uint32_t* __restrict__ cur, uint2* __restrict__ adj, uint32_t* __restrict__ src) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // the loop bound is uniform over the block, so every warp-wide call has all lanes
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < narcs; base += stride) {
        const uint64_t a = base + threadIdx.x;
        const bool valid = a < narcs;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (valid) r = __ldcs(binned + a);
        const uint64_t pa = arc_slot(valid, r.x, true, off, cur, cur);
        if (valid) {
            adj[pa] = make_uint2(r.y, r.z);
            src[pa] = r.x;
        }
    }
}

// Every build: the arcs of each vertex rewritten with the build's hash keys and center bits,
// arcs to centers first (front cursor), the others from the back.  One thread per arc in CSR
// order: the arcs of a warp mostly share their source, so a hub costs one cursor atomic per
// 32 arcs (arc_slot merges equal (source, side) keys), not one per arc.
__global__ void __launch_bounds__(256)
k_arc_fill(const uint2* __restrict__ adj, const uint32_t* __restrict__ src, uint64_t narcs,
           const uint64_t* __restrict__ off, uint32_t* __restrict__ ccur, uint32_t* __restrict__ ncur,
           uint4* __restrict__ arcs, uint64_t salt, const uint32_t* __restrict__ cbits,
           const uint32_t* __restrict__ cidx, int all_centers, const uint64_t* __restrict__ eT,
           uint64_t* __restrict__ aT) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < narcs; base += stride) {
        const uint64_t a = base + threadIdx.x;
        const bool valid = a < narcs;
        uint2 ye = make_uint2(0, 0);
        uint32_t x = 0;
        if (valid) {
            ye = adj[a];
            x = src[a];
        }
        const uint32_t y = ye.x;
        const bool cy = valid && (all_centers || ((cbits[y >> 5] >> (y & 31)) & 1u));
        const uint64_t p = arc_slot(valid, x, cy, off, ccur, ncur);
        if (valid) {
            const uint64_t key = mix64(salt ^ (uint64_t)ye.y);
            const uint32_t iy = !cy ? kNone : all_centers ? y : cidx[y];
            arcs[p] = make_uint4(y | ((cy ? 1u : 0u) << 31), iy, (uint32_t)key, (uint32_t)(key >> 32));
            if (eT) aT[p] = eT[ye.y];   // per-edge probabilities: each arc carries its edge's threshold
        }
    }
}

// Threshold word of a probability: floor(p 2^64) (exact: ldexp scales by a power of two and
// the conversion truncates), kAllLive for p >= 1, 0 for p <= 0 or NaN.
__device__ __forceinline__ uint64_t prob_T(double p) {
    if (p >= 1.0) return kAllLive;
    if (!(p > 0.0)) return 0;
    return (uint64_t)ldexp(p, 64);
}

__global__ void k_probs_T(const double* __restrict__ p, uint64_t m, uint64_t* __restrict__ eT) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        eT[e] = prob_T(p[e]);
}

// Weighted cascade on an undirected graph: p_e = 2 / (d_u + d_v), the mean of the two
// directions' 1/d (degrees count every edge of the list at both ends).
__global__ void k_wic_T(const uint2* __restrict__ edges, uint64_t m, const uint64_t* __restrict__ off,
                        uint64_t* __restrict__ eT) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 ed = edges[e];
        const double du = (double)(off[ed.x + 1] - off[ed.x]), dv = (double)(off[ed.y + 1] - off[ed.y]);
        eT[e] = prob_T(2.0 / (du + dv));
    }
}

// Sum of the probabilities the thresholds stand for (sizing of the live-record buffers).
__global__ void k_T_sum(const uint64_t* __restrict__ eT, uint64_t m, double* __restrict__ sum) {
    double acc = 0.0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        acc += eT[e] == kAllLive ? 1.0 : (double)eT[e] * 0x1p-64;
#pragma unroll
    for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, acc);
}

// ---- exclusive scan, u32 -> u64 (tiles of 4096: 1024 threads x 4 items) -------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t x, uint64_t* warp_sums,
                                                         uint64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
        uint64_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        warp_sums[lane] = wi - w;          // exclusive prefix of warp totals
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    uint64_t r = warp_sums[wid] + inc - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_partial(const uint32_t* __restrict__ in, uint64_t count, uint64_t* __restrict__ part) {
    __shared__ uint64_t ws[32];
    __shared__ uint64_t tot;
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < count) s += in[base + i];
    block_exclusive_scan(s, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// one block scans all tile totals in place (exclusive), 1024 at a time
__global__ void __launch_bounds__(kScanThreads)
k_scan_top(uint64_t* __restrict__ part, uint64_t nparts) {
    __shared__ uint64_t ws[32];
    __shared__ uint64_t tot;
    uint64_t carry = 0;
    for (uint64_t base = 0; base < nparts; base += kScanThreads) {
        uint64_t i = base + threadIdx.x;
        uint64_t x = i < nparts ? part[i] : 0;
        uint64_t ex = block_exclusive_scan(x, ws, &tot);
        if (i < nparts) part[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const uint32_t* __restrict__ in, uint64_t count, const uint64_t* __restrict__ part,
             uint64_t* __restrict__ out) {
    __shared__ uint64_t ws[32];
    __shared__ uint64_t tot;
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t vals[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        vals[i] = (base + i < count) ? in[base + i] : 0u;
        s += vals[i];
    }
    uint64_t ex = block_exclusive_scan(s, ws, &tot) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < count) out[base + i] = ex;
        ex += vals[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = part[gridDim.x];
}

}  // namespace

// out[0..count] = exclusive prefix sums of in[0..count), out[count] = total.
// Uses c->d_tmp for tile totals (grown on demand).
int im_scan_u32_to_u64(im_ctx* c, const uint32_t* d_in, uint64_t* d_out, uint64_t count) {
    uint64_t tiles = (count + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        IM_CUDA(c, cudaMemsetAsync(d_out, 0, sizeof(uint64_t), c->stream));
        return IM_OK;
    }
    size_t need = (tiles + 1) * sizeof(uint64_t);
    if (need > c->tmp_bytes) {
        if (c->d_tmp) cudaFree(c->d_tmp);
        c->d_tmp = nullptr;
        c->tmp_bytes = 0;
        if (im_dev_malloc(&c->d_tmp, need) != cudaSuccess) return im_fail(c, IM_ENOMEM, "scan scratch");
        c->tmp_bytes = need;
    }
    uint64_t* part = (uint64_t*)c->d_tmp;
    IM_LAUNCH(c, K_SCAN_PARTIAL, k_scan_partial, (unsigned)tiles, kScanThreads, 0, d_in, count, part);
    IM_LAUNCH(c, K_SCAN_TOP, k_scan_top, 1, kScanThreads, 0, part, tiles);
    IM_LAUNCH(c, K_SCAN_APPLY, k_scan_apply, (unsigned)tiles, kScanThreads, 0, d_in, count, part, d_out);
    IM_CUDA(c, cudaGetLastError());
    return IM_OK;
}

// Pack and validate the edge list and build the CSR offsets (u64); the arcs themselves are
// written by every build (im_arc_keys), which knows the centers.
int im_graph_build(im_ctx* c, const uint32_t* d_u, const uint32_t* d_v) {
    const uint32_t n = c->n;
    const uint64_t m = c->m;
    uint64_t m_pad = (m + 1) & ~1ull;
    if (m_pad == 0) m_pad = 2;
    if (!(c->d_edges && n <= c->graph_n_alloc && m <= c->graph_m_alloc)) {
        // larger sizes: new buffers (a captured selection graph points at the old ones), at
        // least the context's reserve
        im_select_graph_free(c);
        cudaFree(c->d_edges); cudaFree(c->d_off); cudaFree(c->d_arcs); cudaFree(c->d_arc_cur);
        cudaFree(c->d_adj); cudaFree(c->d_src);
        c->d_edges = nullptr; c->d_off = nullptr; c->d_arcs = nullptr; c->d_arc_cur = nullptr;
        c->d_adj = nullptr; c->d_src = nullptr;
        c->graph_n_alloc = 0;
        c->graph_m_alloc = 0;
        const uint32_t na = n > c->res_n ? n : c->res_n;
        const uint64_t ma = m > c->res_m ? m : c->res_m;
        const uint64_t ma_pad = ((ma + 1) & ~1ull) + 2;
        if (im_dev_malloc(&c->d_edges, ma_pad * sizeof(uint2)) != cudaSuccess)
            return im_fail(c, IM_ENOMEM, "edge list");
        if (im_dev_malloc(&c->d_off, ((size_t)na + 1) * sizeof(uint64_t)) != cudaSuccess)
            return im_fail(c, IM_ENOMEM, "csr offsets");
        if (im_dev_malloc(&c->d_arcs, (2 * ma + 2) * sizeof(uint4)) != cudaSuccess)
            return im_fail(c, IM_ENOMEM, "csr arcs");
        if (im_dev_malloc(&c->d_adj, (2 * ma + 2) * sizeof(uint2)) != cudaSuccess ||
            im_dev_malloc(&c->d_src, (2 * ma + 2) * sizeof(uint32_t)) != cudaSuccess)
            return im_fail(c, IM_ENOMEM, "static adjacency");
        // two cursors per vertex for the arc fill; the first n + 5 words serve as degree scratch
        if (im_dev_malloc(&c->d_arc_cur, (2 * (size_t)na + 8) * sizeof(uint32_t)) != cudaSuccess)
            return im_fail(c, IM_ENOMEM, "arc cursors");
        c->graph_n_alloc = na;
        c->graph_m_alloc = ma;
    }
    IM_CUDA(c, cudaMemsetAsync(c->d_edges, 0, m_pad * sizeof(uint2), c->stream));
    uint32_t* deg = c->d_arc_cur;
    unsigned int* bad = (unsigned int*)(deg + n + 1);
    int rc = IM_OK;
    do {
        if (cudaMemsetAsync(deg, 0, ((size_t)n + 1) * sizeof(uint32_t) + 16, c->stream) != cudaSuccess) {
            rc = im_fail(c, IM_ECUDA, "memset");
            break;
        }
        const unsigned B = 256;
        if (m > 0) {
            IM_LAUNCH(c, K_PACK_EDGES, k_pack_edges, grid_for(m, B), B, 0, d_u, d_v, m, n, c->d_edges, bad);
            IM_LAUNCH(c, K_CSR_DEGREE, k_csr_degree, grid_for(m, B), B, 0, c->d_edges, m, n, deg);
        }
        if (c->deferred) {
            // queued into a graph: the flag is read after it ran (an invalid edge was skipped by
            // every kernel, so the graph stays memory-safe; the instance then fails)
            c->h_live[3] = 0;
            if (cudaMemcpyAsync(c->h_live + 3, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess) {
                rc = im_cuda_check(c, cudaGetLastError(), "edge validation");
                break;
            }
        } else {
            unsigned int h_bad = 0;
            if (cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess) {
                rc = im_cuda_check(c, cudaGetLastError(), "edge validation");
                break;
            }
            if (h_bad) {
                rc = im_fail(c, IM_EINVAL, "edge list has an id >= n or a self-loop");
                break;
            }
        }
        rc = im_scan_u32_to_u64(c, deg, c->d_off, n);
        if (rc) break;
        if (m > 0) {   // the static adjacency (the cursors start from 0 again)
            if (cudaMemsetAsync(c->d_arc_cur, 0, (size_t)n * sizeof(uint32_t), c->stream) != cudaSuccess) {
                rc = im_fail(c, IM_ECUDA, "memset");
                break;
            }
            if (m >= (1ull << 24) && n >= 4 * kAdjBins && m < (1ull << 32)) {
                // large graphs: binned by source range first (the arc array is the scratch; the
                // range cursors sit in the second half of the cursor array)
                const uint32_t V = (n + kAdjBins - 1) / kAdjBins;
                unsigned long long* bcur = reinterpret_cast<unsigned long long*>(c->d_arc_cur + n + (n & 1u));
                uint4* binned = reinterpret_cast<uint4*>(c->d_arcs);
                IM_LAUNCH(c, K_CSR_FILL, k_adj_bin_init, 1, kAdjBins, 0, c->d_off, n, V, bcur);
                IM_LAUNCH(c, K_CSR_FILL, k_adj_bin, grid_for((m + kAdjEdgesPerThread - 1) / kAdjEdgesPerThread, B,
                                                             152u * 8u), B, 0, c->d_edges, m, V, bcur, binned);
                IM_LAUNCH(c, K_CSR_FILL, k_adj_place, grid_for(2 * m, B, 152u * 16u), B, 0, binned, 2 * m,
                          c->d_off, c->d_arc_cur, c->d_adj, c->d_src);
            } else {
                IM_LAUNCH(c, K_CSR_FILL, k_adj_fill, grid_for(m, B, 152u * 16u), B, 0, c->d_edges, m, c->d_off,
                          c->d_arc_cur, c->d_adj, c->d_src);
            }
        }
        if (!c->deferred) {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = im_cuda_check(c, e, "csr build");
        }
    } while (0);
    return rc;
}

// Scratch of im_scan_u32_to_u64 for `count` elements, allocated ahead (the batch engine queues
// its scans into a graph, where nothing may be allocated).
int im_scan_reserve(im_ctx* c, uint64_t count) {
    const uint64_t tiles = (count + kScanTile - 1) / kScanTile;
    const size_t need = (tiles + 1) * sizeof(uint64_t);
    if (need <= c->tmp_bytes) return IM_OK;
    if (c->d_tmp) cudaFree(c->d_tmp);
    c->d_tmp = nullptr;
    c->tmp_bytes = 0;
    if (im_dev_malloc(&c->d_tmp, need) != cudaSuccess) return im_fail(c, IM_ENOMEM, "scan scratch");
    c->tmp_bytes = need;
    return IM_OK;
}

// Per-edge probabilities: thresholds of every edge (and their mean), on the device.
int im_edge_probs(im_ctx* c, int model, const double* d_p) {
    const uint64_t m = c->m;
    const uint64_t m_pad = (m + 1) & ~1ull;   // k_sample_emit reads them in pairs
    if (!c->d_edgeT) {
        if (im_dev_malloc(&c->d_edgeT, (m_pad + 2) * sizeof(uint64_t)) != cudaSuccess ||
            im_dev_malloc(&c->d_arcT, (2 * m + 2) * sizeof(uint64_t)) != cudaSuccess) {
            cudaFree(c->d_edgeT);   // both or neither (a later call allocates them again)
            cudaFree(c->d_arcT);
            c->d_edgeT = nullptr;
            c->d_arcT = nullptr;
            return im_fail(c, IM_ENOMEM, "edge thresholds");
        }
        c->edgeT_cap = m;
    }
    IM_CUDA(c, cudaMemsetAsync(c->d_edgeT, 0, (m_pad + 2) * sizeof(uint64_t), c->stream));
    if (m > 0) {
        if (model == IM_PROBS_WIC)
            IM_LAUNCH(c, K_ARC_KEYS, k_wic_T, grid_for(m, 256), 256, 0, c->d_edges, m, c->d_off, c->d_edgeT);
        else
            IM_LAUNCH(c, K_ARC_KEYS, k_probs_T, grid_for(m, 256), 256, 0, d_p, m, c->d_edgeT);
    }
    double* d_sum = reinterpret_cast<double*>(c->d_edgeT + m_pad + 1);   // a spare word
    IM_CUDA(c, cudaMemsetAsync(d_sum, 0, sizeof(double), c->stream));
    if (m > 0)
        IM_LAUNCH(c, K_ARC_KEYS, k_T_sum, grid_for(m, 256, 152u * 8u), 256, 0, c->d_edgeT, m, d_sum);
    double sum = 0.0;
    IM_CUDA(c, cudaMemcpyAsync(&sum, d_sum, sizeof sum, cudaMemcpyDeviceToHost, c->stream));
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->mean_p = m ? sum / (double)m : 0.0;
    return IM_OK;
}

int im_arc_keys(im_ctx* c, uint64_t salt) {
    if (c->m > 0) {
        const uint32_t n = c->n;
        IM_CUDA(c, cudaMemsetAsync(c->d_arc_cur, 0, 2 * (size_t)n * sizeof(uint32_t), c->stream));
        IM_LAUNCH(c, K_ARC_KEYS, k_arc_fill, grid_for(2 * c->m, 256, 152u * 16u), 256, 0, c->d_adj, c->d_src,
                  2 * c->m, c->d_off, c->d_arc_cur, c->d_arc_cur + n, c->d_arcs, salt, c->d_cbits, c->d_cidx,
                  (int)c->all_centers, c->smp.eT, c->d_arcT);
    }
    IM_CUDA(c, cudaGetLastError());
    c->arc_salt = salt;
    c->arc_keys_valid = true;
    return IM_OK;
}
