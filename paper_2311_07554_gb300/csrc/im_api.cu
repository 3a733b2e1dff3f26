// im_api.cu -- the C ABI (include/im_gb300.h): context lifetime, argument checks, device
// memory, the build / select / spread flows, statistics and launch profiling.
#include <cmath>
#include <cstring>
#include <algorithm>

#include <atomic>

#include "im_internal.cuh"

using namespace imk;

namespace {

thread_local std::string g_create_error;

const char* const kNames[K_COUNT] = {
    "pack_edges", "csr_degree", "scan_partial", "scan_top", "scan_apply", "csr_fill",
    "center_hist", "center_pick", "center_flags", "center_index",
    "batch_init", "sample_union", "compress_count", "gain_compact", "init_keys",
    "reduce_reset", "reduce", "plan", "sel_hist", "sel_pick", "gather", "eval",
    "fallback", "finalize", "mark_seed", "spread_tasks", "spread_dedup", "labels_min",
    "labels_out", "arc_keys", "sample_emit", "union", "cover_roots", "refresh_gather",
    "count_above", "zero", "select_graph", "sel_begin", "sel_step"};

int bitlen64(uint64_t x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

template <typename T>
bool dalloc(T*& p, size_t count) {
    dfree(p);
    void* q = nullptr;
    if (im_dev_malloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    p = (T*)q;
    return true;
}

void free_sketch_state(im_ctx* c) {
    dfree(c->d_cbits); dfree(c->d_cidx); dfree(c->d_centers);
    dfree(c->d_label); dfree(c->d_size); dfree(c->d_gain0);
    dfree(c->d_key); dfree(c->d_stamp); dfree(c->d_seedflag);
    dfree(c->d_batch); dfree(c->d_fresh); dfree(c->d_seed_list); dfree(c->d_labcache);
    dfree(c->d_pair_undo);
    dfree(c->d_gain_list); dfree(c->d_round_evals);
    im_select_graph_free(c);   // the graph holds pointers to the buffers freed here
    for (auto& L : c->lane) {
        dfree(L.parent); dfree(L.word); dfree(L.live); dfree(L.live_n); dfree(L.gain); dfree(L.fresh);
        dfree(L.spec_ov);
    }
    c->live_cap = 0;
    dfree(c->d_fb_queue); dfree(c->d_fb_bits); dfree(c->d_fb_tasks);
    dfree(c->d_cflags); dfree(c->d_cpos); dfree(c->d_csel);
    c->batch_alloc = 0;
    c->fb_slots = 0;
    c->fb_cap = 0;
    c->compact_cap = 0;
    c->cap_n = 0;
    c->cap_R = 0;
    c->cap_nspec = 0;
    c->built = false;
}

// Every buffer a build's kernels write is allocated (a host-side check before any launch).
bool sketch_buffers_ready(const im_ctx* c, uint32_t nspec) {
    bool ok = c->d_gain0 && c->d_key && c->d_stamp && c->d_seedflag && c->d_batch && c->d_fresh &&
              c->d_seed_list && c->d_labcache && c->d_pair_undo && c->d_gain_list && c->d_round_evals &&
              c->d_label && c->d_size && c->d_live_total;
    for (uint32_t i = 0; i < kMaxLanes && ok; ++i) {
        const im_ctx::Lane& L = c->lane[i];
        ok = L.parent && L.word && (i == 0 || (L.gain && L.fresh)) && (!c->live_cap || (L.live && L.live_n)) &&
             (!nspec || L.spec_ov);
    }
    if (ok && !c->all_centers)
        ok = c->d_cbits && c->d_cidx && c->d_centers && c->d_fb_queue && c->d_fb_bits && c->d_fb_tasks &&
             c->d_cflags && c->d_cpos && c->d_csel;
    if (ok && nspec) ok = c->d_spec_keys && c->d_spec_ids;
    return ok;
}

__global__ void k_mask_covered(uint32_t* p, uint64_t cnt) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (uint64_t)gridDim.x * blockDim.x)
        p[i] &= ~kCovered;
}

__global__ void k_iota(uint32_t* p, uint32_t cnt) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) p[i] = i;
}

void resolve_events(im_ctx* c) {
    if (c->ev_pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (uint32_t i = 1; i < kMaxLanes; ++i)
        if (c->lane_stream[i]) cudaStreamSynchronize(c->lane_stream[i]);
    for (auto& pe : c->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[pe.second.first], c->ev_pool[pe.second.second]) == cudaSuccess)
            c->prof_ms[pe.first] += ms;
    }
    cudaGetLastError();
    c->ev_pending.clear();
}

int next_event(im_ctx* c) {
    size_t used = c->ev_pending.size() * 2;
    if (used + 2 > 8192) { resolve_events(c); used = 0; }
    while (c->ev_pool.size() < used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        c->ev_pool.push_back(e);
    }
    return (int)used;
}

}  // namespace

const char* imk::kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? kNames[id] : "?"; }

void im_prof_begin(im_ctx* c, int kid, int* ev0, bool count_launch) {
    *ev0 = -1;
    if (c->capturing) return;   // a captured launch runs (and is counted) with its graph
    if (count_launch) c->launches++;
    c->prof_launches[kid]++;
    if (!c->prof) return;
    int e = next_event(c);
    if (e < 0) return;
    cudaEventRecord(c->ev_pool[e], c->cur);
    *ev0 = e;
}

void im_prof_end(im_ctx* c, int kid, int ev0) {
    if (!c->prof || ev0 < 0) return;
    cudaEventRecord(c->ev_pool[ev0 + 1], c->cur);
    c->ev_pending.push_back({kid, {ev0, ev0 + 1}});
}

// Failure injection for tests (im_debug_fail_alloc): the number of device allocations still
// to succeed before one fails, or -1 when disarmed.
static std::atomic<int64_t> g_fail_alloc_after{-1};

// Test hook (im_debug_record_cap): the live-pair record capacity the sketch kernels may use, or -1.
static std::atomic<int64_t> g_record_cap{-1};

uint64_t im_record_cap(uint64_t allocated) {
    const int64_t cap = g_record_cap.load();
    return cap < 0 || (uint64_t)cap >= allocated ? allocated : (uint64_t)cap;
}

cudaError_t im_dev_malloc(void** p, size_t bytes) {
    int64_t left = g_fail_alloc_after.load();
    while (left >= 0) {
        if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
            if (left == 0) {   // this allocation is the one that fails; the hook disarms itself
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

int im_fail(im_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

int im_cuda_check(im_ctx* c, cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return im_fail(c, e == cudaErrorMemoryAllocation ? IM_ENOMEM : IM_ECUDA, msg);
}

// Upload (host lists through a staging buffer kept by the context), validate and build the
// CSR of the edge list for c->n, c->m; buffers are reused while n and m are unchanged.
static int load_graph(im_ctx* c, const uint32_t* u, const uint32_t* v, int ptr_kind) {
    c->graph_ok = false;
    const uint64_t m = c->m;
    const uint32_t *pu = u, *pv = v;
    if (ptr_kind == IM_PTR_HOST && m > 0) {
        // page-locked lists that the device can address (the runtime gives a device pointer for
        // them) are read by the packing kernel in place, over the CPU-GPU link: no staging copy
        cudaPointerAttributes au{}, av{};
        const bool mapped = cudaPointerGetAttributes(&au, u) == cudaSuccess && au.type == cudaMemoryTypeHost &&
                            au.devicePointer && cudaPointerGetAttributes(&av, v) == cudaSuccess &&
                            av.type == cudaMemoryTypeHost && av.devicePointer;
        cudaGetLastError();
        if (mapped) {
            const int rc = im_graph_build(c, static_cast<const uint32_t*>(au.devicePointer),
                                          static_cast<const uint32_t*>(av.devicePointer));
            if (rc == IM_OK) c->graph_ok = true;
            return rc;
        }
    }
    if (ptr_kind == IM_PTR_HOST && m > 0) {
        if (c->upload_cap < m) {
            dfree(c->d_upload);
            if (c->h_upload) cudaFreeHost(c->h_upload);
            c->h_upload = nullptr;
            c->upload_cap = 0;
            const uint64_t cap = std::max(m, c->res_m);
            if (!dalloc(c->d_upload, 2 * cap)) return im_fail(c, IM_ENOMEM, "edge upload");
            c->upload_cap = cap;
        }
        // pageable lists go through a pinned buffer, so that the copy engine reads them
        // directly and contexts on other threads do not queue behind the driver's staging
        cudaPointerAttributes at{};
        const bool pinned = cudaPointerGetAttributes(&at, u) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                            cudaPointerGetAttributes(&at, v) == cudaSuccess && at.type == cudaMemoryTypeHost;
        cudaGetLastError();
        const uint32_t *su = u, *sv = v;
        if (!pinned) {
            if (!c->h_upload && cudaMallocHost(&c->h_upload, 2 * c->upload_cap * sizeof(uint32_t)) != cudaSuccess) {
                c->h_upload = nullptr;
                cudaGetLastError();
            }
            if (c->h_upload) {
                memcpy(c->h_upload, u, m * sizeof(uint32_t));
                memcpy(c->h_upload + m, v, m * sizeof(uint32_t));
                su = c->h_upload;
                sv = c->h_upload + m;
            }
        }
        IM_CUDA(c, cudaMemcpyAsync(c->d_upload, su, m * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
        IM_CUDA(c, cudaMemcpyAsync(c->d_upload + m, sv, m * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
        pu = c->d_upload;
        pv = c->d_upload + m;
    }
    const int rc = im_graph_build(c, pu, pv);   // synchronises: the caller's lists may go
    if (rc == IM_OK) c->graph_ok = true;
    return rc;
}

// Spread scratch for k seeds: (component, size) words of every (seed, sketch) and the seed list.
int spread_reserve(im_ctx* c, uint32_t k) {
    const size_t need = (size_t)k * c->R;
    if (need > c->spread_cap) {
        if (!dalloc(c->d_spread_pairs, need)) { c->spread_cap = 0; return im_fail(c, IM_ENOMEM, "spread"); }
        c->spread_cap = need;
    }
    if (!c->d_spread_seeds && !dalloc(c->d_spread_seeds, kSpreadKMax)) return im_fail(c, IM_ENOMEM, "spread");
    return IM_OK;
}

// Buffers for uploading a graph of n vertices and m edges from host memory, reserved ahead of a
// batch graph (nothing may be allocated while it is captured).  The context was created with a
// reserve of at least n and m, so its graph buffers already fit.
int batch_load_reserve(im_ctx* c, uint32_t n, uint64_t m) {
    if (!(c->d_edges && n <= c->graph_n_alloc && m <= c->graph_m_alloc))
        return im_fail(c, IM_ESTATE, "graph buffers not reserved");
    if (m > 0 && c->upload_cap < m) {
        dfree(c->d_upload);
        if (c->h_upload) cudaFreeHost(c->h_upload);
        c->h_upload = nullptr;
        c->upload_cap = 0;
        if (!dalloc(c->d_upload, 2 * m)) return im_fail(c, IM_ENOMEM, "edge upload");
        c->upload_cap = m;
    }
    if (m > 0 && !c->h_upload && cudaMallocHost(&c->h_upload, 2 * c->upload_cap * sizeof(uint32_t)) != cudaSuccess) {
        c->h_upload = nullptr;
        cudaGetLastError();
        return im_fail(c, IM_ENOMEM, "edge staging (pinned host memory)");
    }
    int rc = im_scan_reserve(c, n);
    if (rc) return rc;
    c->n = n;
    c->m = m;
    c->prob_model = IM_PROBS_UNIFORM;
    c->graph_ok = true;   // the graph that is queued next (validated after it ran)
    return IM_OK;
}

// Upload and CSR of the graph queued on the context stream, with no host wait (the batch
// graph captures it); host lists that are not pinned are staged into the context's pinned
// buffer now, on the host.
int batch_load_enqueue(im_ctx* c, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v) {
    if (n != c->n || m != c->m) return im_fail(c, IM_ESTATE, "graph dimensions differ from the reserve");
    c->deferred = true;
    const int rc = load_graph(c, u, v, IM_PTR_HOST);
    c->deferred = false;
    c->graph_ok = rc == IM_OK;
    return rc;
}

// ------------------------------------------------------------------------------------
extern "C" {

int im_create(im_ctx** out, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v,
              int ptr_kind, void* stream) {
    return im_create_reserved(out, n, m, u, v, ptr_kind, stream, nullptr);
}

}  // extern "C"

int im_create_reserved(im_ctx** out, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v, int ptr_kind,
                       void* stream, const ImReserve* res) {
    if (!out) return im_fail(nullptr, IM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n == 0 || n >= 0x80000000u) return im_fail(nullptr, IM_EINVAL, "n must be in [1, 2^31)");
    if (m >= 0xFFFFFFFFull) return im_fail(nullptr, IM_EINVAL, "m must be < 2^32");
    if (ptr_kind != IM_PTR_HOST && ptr_kind != IM_PTR_DEVICE)
        return im_fail(nullptr, IM_EINVAL, "bad ptr_kind");
    if (m > 0 && (!u || !v)) return im_fail(nullptr, IM_EINVAL, "edge arrays are NULL");
    im_ctx* c = new (std::nothrow) im_ctx();
    if (!c) return im_fail(nullptr, IM_ENOMEM, "context");
    c->n = n;
    c->m = m;
    if (res) {
        c->res_n = res->n;
        c->res_R = res->R;
        c->res_m = res->m;
        c->res_nc = res->nc;
        // live-pair records of a batch of 32 sketches at the largest p m (as im_build_sketches)
        const double ex = res->pm * 32.0;
        double cap = ex > 0 ? 1.3 * ex + 16.0 * std::sqrt(ex) + 65536.0 : 0.0;
        if (cap > (double)(1ull << 28)) cap = (double)(1ull << 28);
        c->res_live = (uint64_t)cap;
    }
    cudaGetDevice(&c->device);
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            g_create_error = "cudaStreamCreate failed";
            delete c;
            return IM_ECUDA;
        }
        c->own_stream = true;
    }
    c->cur = c->stream;
    bool made = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&c->ev_spec, cudaEventDisableTiming) == cudaSuccess;
    for (uint32_t i = 1; i < kMaxLanes && made; ++i)
        made = cudaStreamCreateWithFlags(&c->lane_stream[i], cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) == cudaSuccess;

    if (!made) {
        g_create_error = "stream or event creation failed";
        im_destroy(c);
        return IM_ECUDA;
    }
    c->lane[0].stream = c->stream;
    for (uint32_t i = 1; i < kMaxLanes; ++i) c->lane[i].stream = c->lane_stream[i];
    int rc = IM_OK;
    do {
        if (im_dev_malloc(&c->d_sel, sizeof(SelState)) != cudaSuccess ||
            cudaMallocHost(&c->h_sel, sizeof(SelState)) != cudaSuccess ||
            cudaMallocHost(&c->h_live, 4 * sizeof(unsigned long long)) != cudaSuccess) {
            rc = im_fail(c, IM_ENOMEM, "selection state");
            break;
        }
        cudaMemsetAsync(c->d_sel, 0, sizeof(SelState), c->stream);
        memset(c->h_sel, 0, sizeof(SelState));
        if (im_dev_malloc(&c->d_live_total, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMemsetAsync(c->d_live_total, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) {
            rc = im_fail(c, IM_ENOMEM, "counters");
            break;
        }
        if (im_dev_malloc(&c->d_spread_total, sizeof(unsigned long long)) != cudaSuccess) {
            rc = im_fail(c, IM_ENOMEM, "spread total");
            break;
        }
        rc = load_graph(c, u, v, ptr_kind);
    } while (0);
    if (rc != IM_OK) {
        g_create_error = c->err;
        im_destroy(c);
        return rc;
    }
    *out = c;
    return IM_OK;
}

extern "C" {

int im_set_sketch_batch(im_ctx* c, uint32_t batch) {
    if (!c) return IM_EINVAL;
    if (batch != 0 && (batch > 32 || (batch & (batch - 1)) != 0))
        return im_fail(c, IM_EINVAL, "sketch batch must be 0 or a power of two <= 32");
    c->batch_req = batch;
    return IM_OK;
}

int im_set_seed_speculation(im_ctx* c, uint32_t candidates) {
    if (!c) return IM_EINVAL;
    if (candidates > kSpecMax) return im_fail(c, IM_EINVAL, "at most 8 candidate first seeds");
    c->spec_req = candidates;
    return IM_OK;
}

int im_set_hubs(im_ctx* c, uint32_t cap, uint32_t min_degree) {
    if (!c) return IM_EINVAL;
    c->hub_cap = cap;
    c->hub_min_deg = min_degree ? min_degree : 1u;
    return IM_OK;
}

int im_set_graph(im_ctx* c, int on) {
    if (!c) return IM_EINVAL;
    c->use_graph = on != 0;
    return IM_OK;
}

int im_set_pipeline(im_ctx* c, uint32_t lanes) {
    if (!c) return IM_EINVAL;
    if (lanes < 1 || lanes > kMaxLanes) return im_fail(c, IM_EINVAL, "lanes must be 1 or 2");
    c->lanes = lanes;
    return IM_OK;
}

int im_set_union_path(im_ctx* c, int path) {
    if (!c) return IM_EINVAL;
    if (path != IM_UNION_FUSED && path != IM_UNION_RECORDS && path != IM_UNION_BUCKETS && path != IM_UNION_AUTO)
        return im_fail(c, IM_EINVAL,
                       "union path must be IM_UNION_FUSED, IM_UNION_RECORDS, IM_UNION_BUCKETS or IM_UNION_AUTO");
    c->union_path = path;
    return IM_OK;
}

int im_set_refresh_threshold(im_ctx* c, uint64_t min_batch) {
    if (!c) return IM_EINVAL;
    c->refresh_req = min_batch;
    if (c->built) c->refresh_min = min_batch ? min_batch : std::max<uint64_t>(16384, c->n / 4);
    return IM_OK;
}

int im_load_graph(im_ctx* c, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v, int ptr_kind) {
    if (!c) return IM_EINVAL;
    if (c->serving) return im_fail(c, IM_ESTATE, "a serving loop owns the context (im_serve_finish first)");
    if (n == 0 || n >= 0x80000000u) return im_fail(c, IM_EINVAL, "n must be in [1, 2^31)");
    if (m >= 0xFFFFFFFFull) return im_fail(c, IM_EINVAL, "m must be < 2^32");
    if (ptr_kind != IM_PTR_HOST && ptr_kind != IM_PTR_DEVICE) return im_fail(c, IM_EINVAL, "bad ptr_kind");
    if (m > 0 && (!u || !v)) return im_fail(c, IM_EINVAL, "edge arrays are NULL");
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (n > c->cap_n) free_sketch_state(c);   // the per-vertex buffers are too small
    if (n != c->n || m != c->m) im_select_graph_free(c);   // it captured n and m
    if (m > c->edgeT_cap) { dfree(c->d_edgeT); dfree(c->d_arcT); c->edgeT_cap = 0; }
    c->prob_model = IM_PROBS_UNIFORM;      // probabilities belong to the old edge list
    c->built = false;
    c->seeds.clear();
    c->seed_gains.clear();
    c->round_evals.clear();
    c->n = n;
    c->m = m;
    return load_graph(c, u, v, ptr_kind);
}

int im_set_edge_probs(im_ctx* c, int model, const double* p, int ptr_kind) {
    if (!c) return IM_EINVAL;
    if (c->serving) return im_fail(c, IM_ESTATE, "a serving loop owns the context (im_serve_finish first)");
    if (!c->graph_ok) return im_fail(c, IM_ESTATE, "no valid graph is loaded");
    if (model != IM_PROBS_UNIFORM && model != IM_PROBS_ARRAY && model != IM_PROBS_WIC)
        return im_fail(c, IM_EINVAL, "unknown probability model");
    if (model == IM_PROBS_ARRAY && c->m > 0) {
        if (!p) return im_fail(c, IM_EINVAL, "p is NULL");
        if (ptr_kind != IM_PTR_HOST && ptr_kind != IM_PTR_DEVICE) return im_fail(c, IM_EINVAL, "bad ptr_kind");
    }
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->built = false;   // the sketches belong to the old probabilities
    c->seeds.clear();
    c->seed_gains.clear();
    c->round_evals.clear();
    c->prob_model = IM_PROBS_UNIFORM;   // (the next build re-captures the selection graph if the
                                        // sampler it carries changed)
    if (model == IM_PROBS_UNIFORM) return IM_OK;
    const double* dp = p;
    double* tmp = nullptr;
    if (model == IM_PROBS_ARRAY && ptr_kind == IM_PTR_HOST && c->m > 0) {
        if (!dalloc(tmp, c->m)) return im_fail(c, IM_ENOMEM, "probabilities");
        if (cudaMemcpyAsync(tmp, p, c->m * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            dfree(tmp);
            return im_fail(c, IM_ECUDA, "probabilities");
        }
        dp = tmp;
    }
    const int rc = im_edge_probs(c, model, dp);
    dfree(tmp);
    if (rc) return rc;
    c->prob_model = model;
    return IM_OK;
}

}  // extern "C"

// Sketch construction in three parts, so that the batch engine can capture the middle one into
// a graph: build_prepare validates the arguments, sets the build's parameters and reserves every
// buffer (no kernel); build_enqueue queues the kernels on the context stream (no host
// synchronisation, no allocation); build_finish waits for them and records the results.
int build_prepare(im_ctx* c, uint32_t R, uint64_t seed, double p, double alpha) {
    if (!c) return IM_EINVAL;
    if (c->serving) return im_fail(c, IM_ESTATE, "a serving loop owns the context (im_serve_finish first)");
    if (!c->graph_ok) return im_fail(c, IM_ESTATE, "no valid graph is loaded");
    if (R == 0 || R > 65536) return im_fail(c, IM_EINVAL, "R must be in [1, 65536]");
    if (!(alpha > 0.0) || alpha > 1.0) return im_fail(c, IM_EINVAL, "alpha must be in (0, 1]");
    if (std::isnan(p)) return im_fail(c, IM_EINVAL, "p is NaN");
    const uint32_t n = c->n;
    const int bits = bitlen64(n);
    if (bits + bitlen64((uint64_t)R * n) > 64)
        return im_fail(c, IM_EINVAL, "R * n too large for 64-bit packed gain keys");
    double rr = std::ceil(alpha * (double)n);
    uint32_t rho = rr >= (double)n ? n : (uint32_t)rr;
    if (rho == 0) rho = 1;
    const uint32_t all = rho == n ? 1u : 0u;

    // sampler (Sec. 2 fusion; threshold T = floor(p 2^64), exact)
    Sampler smp{};
    smp.salt = mix64(seed + kGamma);
    smp.all_live = 0;
    smp.T = 0;
    if (p >= 1.0) smp.all_live = 1;
    else if (p > 0.0) smp.T = (uint64_t)std::ldexp(p, 64);
    smp.eT = c->prob_model != IM_PROBS_UNIFORM ? c->d_edgeT : nullptr;
    smp.aT = c->prob_model != IM_PROBS_UNIFORM ? c->d_arcT : nullptr;

    // sketches per edge pass: union-find launches are bound by their critical path, not by
    // their size, so fewer, larger batches win; memory is 12 bytes per vertex per sketch
    uint32_t B = c->batch_req;
    if (B == 0) {
        const uint64_t per = (uint64_t)n * 12;
        B = 32;
        while (B > 1 && (uint64_t)B * per > (8ull << 30)) B /= 2;
    }
    uint32_t rp2 = 1;
    while (rp2 < R) rp2 <<= 1;
    if (B > rp2) B = rp2;

    // IM_UNION_AUTO: bucketed records once a batch's parent arrays (4 n B bytes) are well beyond
    // L2, where taking the sketches one after the other keeps the climbed parents there
    const int upath = c->union_path != IM_UNION_AUTO ? c->union_path
                      : (uint64_t)n * B * 4 > (256ull << 20) ? IM_UNION_BUCKETS : IM_UNION_RECORDS;
    // live-pair records of one batch: expected p m B, with a generous margin; a batch that
    // still overflows falls back to the fused sample+union loop on the device
    uint64_t live_cap = 0;
    if (upath != IM_UNION_FUSED && c->m > 0 && (smp.eT || smp.all_live || smp.T != 0)) {
        const double pe = smp.eT ? c->mean_p : smp.all_live ? 1.0 : p;
        const double ex = pe * (double)c->m * B;
        double cap = 1.3 * ex + 16.0 * std::sqrt(ex) + 65536.0;
        if (cap > (double)(1ull << 28)) cap = (double)(1ull << 28);
        live_cap = (uint64_t)cap;
    }
    // hubs (im_select_hubs): label / size rows after the rho compact rows
    uint32_t hub_rows = 0;
    if (!all) {
        const uint32_t cap = c->hub_cap == imk::kHubsAuto ? std::max<uint32_t>(1024, n / 64) : c->hub_cap;
        hub_rows = std::min<uint32_t>(cap, n - rho);
    }
    const size_t nc = ((size_t)rho + hub_rows) * R;
    // candidate first seeds (chosen after the first batch; a second lane waits for them)
    const uint32_t nspec = std::min<uint32_t>(c->spec_req, n);
    // A build that fits the device buffers reuses them (cudaMalloc / cudaFree synchronise the
    // device, stalling every stream, other contexts' included); the selection graph, which
    // captured the shapes and the sampler, is kept only while both are unchanged.
    const bool fits = c->batch_alloc > 0 && n <= c->cap_n && B <= c->batch_alloc && R <= c->cap_R &&
                      nc <= c->compact_cap && live_cap <= c->live_cap && nspec <= c->cap_nspec &&
                      (all || c->d_cidx != nullptr);
    const bool same_shape = c->R == R && c->rho == rho && c->hub_rows == hub_rows && c->batch_used == B &&
                            c->all_centers == all && c->spec_count == nspec && c->union_used == upath;
    if (!fits) {
        free_sketch_state(c);
    } else if (!same_shape || c->smp.salt != smp.salt || c->smp.T != smp.T || c->smp.all_live != smp.all_live ||
               c->smp.eT != smp.eT || c->smp.aT != smp.aT) {
        im_select_graph_free(c);   // the captured kernels carry the shapes and the sampler
    }
    c->built = false;
    c->R = R; c->seed = seed; c->p = p; c->alpha = alpha; c->rho = rho; c->all_centers = all;
    c->hub_rows = hub_rows;
    c->key_bits = (uint32_t)bits;
    c->smp = smp;
    c->batch_used = B;
    c->union_used = upath;
    c->spec_count = nspec;
    if (!fits) {
        // at least the context's reserve (im_create_reserved), so that later builds fit
        const uint32_t na = std::max(n, c->res_n), Ra = std::max(R, c->res_R);
        const size_t nca = std::max<size_t>(nc, c->res_nc);
        const uint64_t livea = upath != IM_UNION_FUSED ? std::max(live_cap, c->res_live) : live_cap;
        const uint32_t nsa = std::min(std::max(nspec, c->res_n ? std::min<uint32_t>(c->spec_req, kSpecMax) : 0u),
                                      kSpecMax);
        const bool compact = !all || c->res_n > 0;   // a reserved context may serve compact builds
        bool ok = dalloc(c->d_gain0, na) && dalloc(c->d_key, na) && dalloc(c->d_stamp, na) &&
                  dalloc(c->d_seedflag, na) && dalloc(c->d_batch, na) && dalloc(c->d_fresh, na) &&
                  dalloc(c->d_seed_list, na) && dalloc(c->d_labcache, (size_t)kLabSlots * Ra) &&
                  dalloc(c->d_pair_undo, Ra) &&
                  dalloc(c->d_gain_list, na) && dalloc(c->d_round_evals, na) &&
                  dalloc(c->d_label, nca) && dalloc(c->d_size, nca) &&
                  dalloc(c->lane[0].parent, (size_t)B * na) && dalloc(c->lane[0].word, (size_t)B * na);
        for (uint32_t i = 1; i < kMaxLanes && ok; ++i)
            ok = dalloc(c->lane[i].parent, (size_t)B * na) && dalloc(c->lane[i].word, (size_t)B * na) &&
                 dalloc(c->lane[i].gain, na) && dalloc(c->lane[i].fresh, na);
        for (uint32_t i = 0; i < kMaxLanes && ok && nsa; ++i) ok = dalloc(c->lane[i].spec_ov, (size_t)nsa * na);
        if (ok && livea) {
            c->live_cap = livea;
            for (uint32_t i = 0; i < kMaxLanes && ok; ++i)
                ok = dalloc(c->lane[i].live, c->live_cap) && dalloc(c->lane[i].live_n, kLiveCounters);
        }
        if (ok && compact) {
            const size_t nw = ((size_t)na + 31) / 32;
            c->fb_slots = 8;
            c->fb_cap = 1u << 22;
            ok = dalloc(c->d_cbits, nw) && dalloc(c->d_cidx, na) && dalloc(c->d_centers, na) &&
                 dalloc(c->d_fb_queue, (size_t)c->fb_slots * na) &&
                 dalloc(c->d_fb_bits, (size_t)c->fb_slots * nw) && dalloc(c->d_fb_tasks, c->fb_cap) &&
                 dalloc(c->d_cflags, na) && dalloc(c->d_cpos, (size_t)na + 1) &&
                 dalloc(c->d_csel, kCenterSelBytes);
            if (ok) ok = cudaMemsetAsync(c->d_fb_bits, 0, (size_t)c->fb_slots * nw * 4, c->stream) == cudaSuccess;
        }
        if (!ok) {
            free_sketch_state(c);
            return im_fail(c, IM_ENOMEM, "sketch memory");
        }
        c->batch_alloc = B;
        c->compact_cap = nca;
        c->cap_n = na;
        c->cap_R = Ra;
        c->cap_nspec = nsa;
    }
    c->refresh_min = c->refresh_req ? c->refresh_req : std::max<uint64_t>(16384, n / 4);
    int rc = IM_OK;
    if (nspec && (!c->d_spec_keys || !c->d_spec_ids)) {
        // both or neither: a build after a failed one allocates them again
        if (!dalloc(c->d_spec_keys, kSpecMax) || !dalloc(c->d_spec_ids, kSpecMax)) {
            dfree(c->d_spec_keys);
            dfree(c->d_spec_ids);
            rc = im_fail(c, IM_ENOMEM, "first seed candidates");
        }
    }
    if (!rc && !sketch_buffers_ready(c, nspec))
        rc = im_fail(c, IM_ESTATE, "sketch buffers missing after allocation");
    if (rc) { free_sketch_state(c); return rc; }
    return IM_OK;
}

int build_enqueue(im_ctx* c) {
    const uint32_t all = c->all_centers;
    int rc = IM_OK;
    // live pairs before the build, read with the build's final synchronisation
    IM_CUDA(c, cudaMemcpyAsync(c->h_live, c->d_live_total, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               c->stream));
    if (!all) {
        rc = im_select_centers(c, c->d_cflags, c->d_cpos);
        if (!rc) rc = im_select_hubs(c, c->d_cflags, c->d_cpos);
    }
    if (!rc) rc = im_arc_keys(c, c->smp.salt);
    // record counters of the lanes start at zero (each union kernel resets its lane's after use)
    for (uint32_t i = 0; i < kMaxLanes && !rc; ++i)
        if (c->lane[i].live_n &&
            cudaMemsetAsync(c->lane[i].live_n, 0, kLiveCounters * sizeof(unsigned long long), c->stream) != cudaSuccess)
            rc = im_fail(c, IM_ECUDA, "record counter reset");
    if (!rc) rc = im_sketch_batches(c);
    if (!rc) rc = im_selection_init(c, true);   // the build wrote every size entry
    if (!rc) {
        const cudaError_t e = cudaMemcpyAsync(c->h_live + 1, c->d_live_total, sizeof(unsigned long long),
                                              cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) rc = im_cuda_check(c, e, "sketch construction");
    }
    return rc;
}

int build_finish(im_ctx* c) {
    int rc = IM_OK;
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = im_cuda_check(c, e, "sketch construction");
    c->build_live_pairs = c->h_live[1] - c->h_live[0];
    c->hubs = (uint32_t)c->h_live[2];
    if (rc) { free_sketch_state(c); return rc; }
    c->built = true;
    return IM_OK;
}

extern "C" {

int im_build_sketches(im_ctx* c, uint32_t R, uint64_t seed, double p, double alpha) {
    int rc = build_prepare(c, R, seed, p, alpha);
    if (rc) return rc;
    c->h_live[2] = 0;
    rc = build_enqueue(c);
    if (rc) { free_sketch_state(c); return rc; }
    return build_finish(c);
}

int im_select_seeds(im_ctx* c, uint32_t k, uint32_t* seeds_out, uint64_t* gains_out) {
    if (!c) return IM_EINVAL;
    if (c->serving) return im_fail(c, IM_ESTATE, "a serving loop owns the context (im_serve_finish first)");
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    if (k == 0 || k > c->n) return im_fail(c, IM_EINVAL, "k must be in [1, n]");
    if (!seeds_out) return im_fail(c, IM_EINVAL, "seeds_out is NULL");
    if (c->seeds.size() < k) {
        const int rc = im_select_run(c, k);
        if (rc) return rc;
    }
    memcpy(seeds_out, c->seeds.data(), k * sizeof(uint32_t));
    if (gains_out) memcpy(gains_out, c->seed_gains.data(), k * sizeof(uint64_t));
    return IM_OK;
}

int im_reset_selection(im_ctx* c) {
    if (!c) return IM_EINVAL;
    if (c->serving) return im_fail(c, IM_ESTATE, "a serving loop owns the context (im_serve_finish first)");
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    int rc = im_selection_init(c, false);
    if (rc) return rc;
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    return IM_OK;
}

int im_spread(im_ctx* c, const uint32_t* seeds, uint32_t k, uint64_t* spread_out) {
    if (!c) return IM_EINVAL;
    if (c->serving) return im_fail(c, IM_ESTATE, "a serving loop owns the context (im_serve_finish first)");
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    if (!spread_out) return im_fail(c, IM_EINVAL, "spread_out is NULL");
    if (k > kSpreadKMax) return im_fail(c, IM_EINVAL, "k exceeds 16384");
    if (k > 0 && !seeds) return im_fail(c, IM_EINVAL, "seeds is NULL");
    for (uint32_t i = 0; i < k; ++i)
        if (seeds[i] >= c->n) return im_fail(c, IM_EINVAL, "seed id >= n");
    const int rs = spread_reserve(c, k);
    if (rs) return rs;
    if (k > 0)
        IM_CUDA(c, cudaMemcpyAsync(c->d_spread_seeds, seeds, k * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                   c->stream));
    return im_spread_run(c, k, spread_out);
}

int im_mc_spread(im_ctx* c, const uint32_t* seeds, uint32_t k, uint32_t sims, uint64_t mc_seed, uint64_t* out) {
    if (!c) return IM_EINVAL;
    if (c->serving) return im_fail(c, IM_ESTATE, "a serving loop owns the context (im_serve_finish first)");
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    if (!out) return im_fail(c, IM_EINVAL, "out is NULL");
    if (k > kSpreadKMax) return im_fail(c, IM_EINVAL, "k exceeds 16384");
    if (k > 0 && !seeds) return im_fail(c, IM_EINVAL, "seeds is NULL");
    for (uint32_t i = 0; i < k; ++i)
        if (seeds[i] >= c->n) return im_fail(c, IM_EINVAL, "seed id >= n");
    if (!c->d_spread_seeds && !dalloc(c->d_spread_seeds, kSpreadKMax))
        return im_fail(c, IM_ENOMEM, "spread seeds");
    if (k > 0)
        IM_CUDA(c, cudaMemcpyAsync(c->d_spread_seeds, seeds, k * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                   c->stream));
    IM_CUDA(c, cudaMemsetAsync(c->d_spread_total, 0, sizeof(unsigned long long), c->stream));
    int rc = im_mc_run(c, c->d_spread_seeds, k, sims, mc_seed, c->d_spread_total);
    if (rc) return rc;
    unsigned long long h = 0;
    IM_CUDA(c, cudaMemcpyAsync(&h, c->d_spread_total, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = h;
    return IM_OK;
}

int im_get_labels(im_ctx* c, uint32_t r, uint32_t* out, int ptr_kind) {
    if (!c) return IM_EINVAL;
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    if (r >= c->R) return im_fail(c, IM_EINVAL, "r >= R");
    if (!out || (ptr_kind != IM_PTR_HOST && ptr_kind != IM_PTR_DEVICE)) return im_fail(c, IM_EINVAL, "out");
    uint32_t* d = out;
    if (ptr_kind == IM_PTR_HOST) {
        d = nullptr;
        if (!dalloc(d, c->n)) return im_fail(c, IM_ENOMEM, "labels");
    }
    int rc = im_labels_min(c, r, d);
    if (!rc && ptr_kind == IM_PTR_HOST) {
        cudaError_t e = cudaMemcpyAsync(out, d, (size_t)c->n * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = im_cuda_check(c, e, "labels copy");
    } else if (!rc) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = im_cuda_check(c, e, "labels");
    }
    if (ptr_kind == IM_PTR_HOST) dfree(d);
    return rc;
}

static int copy_out(im_ctx* c, void* dst, const void* src, size_t bytes, int ptr_kind) {
    if (!dst || (ptr_kind != IM_PTR_HOST && ptr_kind != IM_PTR_DEVICE)) return im_fail(c, IM_EINVAL, "out");
    IM_CUDA(c, cudaMemcpyAsync(dst, src, bytes,
                               ptr_kind == IM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                               c->stream));
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    return IM_OK;
}

int im_get_gains(im_ctx* c, uint64_t* out, int ptr_kind) {
    if (!c) return IM_EINVAL;
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    return copy_out(c, out, c->d_gain0, (size_t)c->n * 8, ptr_kind);
}

int im_get_centers(im_ctx* c, uint32_t* out, uint32_t* rho_out, int ptr_kind) {
    if (!c) return IM_EINVAL;
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    if (rho_out) *rho_out = c->rho;
    if (!out) return IM_OK;
    if (!c->all_centers) return copy_out(c, out, c->d_centers, (size_t)c->rho * 4, ptr_kind);
    if (ptr_kind == IM_PTR_HOST) {
        for (uint32_t i = 0; i < c->rho; ++i) out[i] = i;
        return IM_OK;
    }
    if (ptr_kind != IM_PTR_DEVICE) return im_fail(c, IM_EINVAL, "ptr_kind");
    k_iota<<<grid_for(c->rho, 256), 256, 0, c->stream>>>(out, c->rho);
    IM_CUDA(c, cudaGetLastError());
    IM_CUDA(c, cudaStreamSynchronize(c->stream));
    return IM_OK;
}

int im_get_compact(im_ctx* c, uint32_t* label, uint32_t* size, int ptr_kind) {
    if (!c) return IM_EINVAL;
    if (!c->built) return im_fail(c, IM_ESTATE, "im_build_sketches has not run");
    const size_t cnt = (size_t)c->rho * c->R;
    if (label) {
        int rc = copy_out(c, label, c->d_label, cnt * 4, ptr_kind);
        if (rc) return rc;
    }
    if (size) {
        int rc = copy_out(c, size, c->d_size, cnt * 4, ptr_kind);
        if (rc) return rc;
        if (ptr_kind == IM_PTR_HOST) {
            for (size_t i = 0; i < cnt; ++i) size[i] &= ~kCovered;
        } else {
            k_mask_covered<<<grid_for(cnt, 256), 256, 0, c->stream>>>(size, cnt);
            IM_CUDA(c, cudaGetLastError());
            IM_CUDA(c, cudaStreamSynchronize(c->stream));
        }
    }
    return IM_OK;
}

int im_get_stats(im_ctx* c, im_stats* out) {
    if (!c || !out) return IM_EINVAL;
    memset(out, 0, sizeof *out);
    out->n = c->n; out->m = c->m; out->R = c->R; out->rho = c->rho;
    out->rounds = (uint32_t)c->seeds.size();
    out->launches = c->launches;

    out->sketch_batch = c->batch_used;
    out->union_path = (uint32_t)c->union_used;
    uint64_t ev = 0;
    for (auto x : c->round_evals) ev += x;
    out->evaluations = ev;
    if (c->h_sel) {
        cudaMemcpyAsync(c->h_sel, c->d_sel, sizeof(SelState), cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        out->bfs_fallbacks = c->h_sel->fb_total;
        out->hop1_arcs = c->h_sel->hop1_arcs;
        out->hop2_searches = c->h_sel->hop2_calls;
        out->hop2_chunks = c->h_sel->hop2_chunks;
        out->refresh_batches = c->h_sel->refresh_batches;
        out->batches = c->h_sel->batches;
        out->spec_batches = c->h_sel->spec_batches;
        out->hubs = c->hubs;
        unsigned long long lt = 0;
        cudaMemcpy(&lt, c->d_live_total, sizeof lt, cudaMemcpyDeviceToHost);
        out->live_pairs = lt;
        out->build_live_pairs = c->build_live_pairs;
    }
    return IM_OK;
}

int im_get_round_evals(im_ctx* c, uint64_t* out, uint32_t count) {
    if (!c || (!out && count)) return IM_EINVAL;
    for (uint32_t i = 0; i < count && i < c->round_evals.size(); ++i) out[i] = c->round_evals[i];
    return IM_OK;
}

int im_profile_enable(im_ctx* c, int on) {
    if (!c) return IM_EINVAL;
    resolve_events(c);
    c->prof = on != 0;
    return IM_OK;
}

int im_profile_reset(im_ctx* c) {
    if (!c) return IM_EINVAL;
    resolve_events(c);
    for (int i = 0; i < K_COUNT; ++i) { c->prof_ms[i] = 0; c->prof_launches[i] = 0; }
    c->launches = 0;
    return IM_OK;
}

int im_profile_get(im_ctx* c, int kernel_id, double* total_ms, uint64_t* launches) {
    if (!c || kernel_id < 0 || kernel_id >= K_COUNT) return IM_EINVAL;
    resolve_events(c);
    if (total_ms) *total_ms = c->prof_ms[kernel_id];
    if (launches) *launches = c->prof_launches[kernel_id];
    return IM_OK;
}

int im_kernel_count(void) { return K_COUNT; }

const char* im_kernel_name(int kernel_id) { return kernel_name(kernel_id); }

int im_debug_fail_alloc(int64_t after) {
    g_fail_alloc_after.store(after < 0 ? -1 : after);
    return IM_OK;
}

int im_debug_record_cap(int64_t records) {
    g_record_cap.store(records < 0 ? -1 : records);
    return IM_OK;
}

void* im_stream(im_ctx* c) { return c ? (void*)c->stream : nullptr; }

const char* im_last_error(const im_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void im_destroy(im_ctx* c) {
    if (!c) return;
    im_serve_stop(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_sketch_state(c);
    dfree(c->d_edges); dfree(c->d_off); dfree(c->d_arcs); dfree(c->d_arc_cur); dfree(c->d_upload);
    dfree(c->d_adj); dfree(c->d_src);
    if (c->h_upload) cudaFreeHost(c->h_upload);
    dfree(c->d_edgeT); dfree(c->d_arcT);
    dfree(c->d_spread_pairs); dfree(c->d_spread_seeds); dfree(c->d_spread_total); dfree(c->d_live_total);
    dfree(c->d_topb);
    if (c->d_sel) cudaFree(c->d_sel);
    if (c->h_sel) cudaFreeHost(c->h_sel);
    if (c->h_live) cudaFreeHost(c->h_live);
    if (c->d_tmp) cudaFree(c->d_tmp);
    dfree(c->d_spec_keys);
    dfree(c->d_spec_ids);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (uint32_t i = 1; i < kMaxLanes; ++i) {
        if (c->lane_stream[i]) { cudaStreamSynchronize(c->lane_stream[i]); cudaStreamDestroy(c->lane_stream[i]); }
        if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_spec) cudaEventDestroy(c->ev_spec);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
