// im_batch.cu -- many independent IM instances on one device (Alg. 1 per instance: sketches,
// lazy greedy, spread), run by a pool of host workers, each owning one context and its own
// stream, so that the instances' kernels overlap on the GPU.  A worker keeps its context
// across instances: im_load_graph and im_build_sketches reuse the buffers while an instance
// fits them (no cudaMalloc / cudaFree, which would synchronise the whole device and stall
// the other workers), so instances are handed out largest first.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "im_internal.cuh"

namespace {

struct BatchShared {
    im_instance* inst = nullptr;
    std::vector<uint32_t> order;    // largest first
    std::atomic<uint32_t> next{0};
    int device = 0;
    ImReserve res{};                // every dimension's largest value over the batch
};

void run_worker(BatchShared* sh) {
    cudaSetDevice(sh->device);
    im_ctx* c = nullptr;
    for (;;) {
        const uint32_t i = sh->next.fetch_add(1);
        if (i >= sh->order.size()) break;
        im_instance& in = sh->inst[sh->order[i]];
        int rc;
        if (!c) rc = im_create_reserved(&c, in.n, in.m, in.u, in.v, IM_PTR_HOST, nullptr, &sh->res);
        else rc = im_load_graph(c, in.n, in.m, in.u, in.v, IM_PTR_HOST);
        if (!rc) rc = im_build_sketches(c, in.R, in.seed, in.p, in.alpha);
        if (!rc) rc = im_select_seeds(c, in.k, in.seeds_out, in.gains_out);
        if (!rc) rc = im_spread(c, in.seeds_out, in.k, in.spread_out);
        in.status = rc;
        if (rc == IM_ECUDA || rc == IM_ENOMEM) {   // start the next instance from a fresh context
            if (c) im_destroy(c);
            c = nullptr;
        }
    }
    if (c) im_destroy(c);
}

}  // namespace

extern "C" int im_run_batch(im_instance* inst, uint32_t count, uint32_t workers) {
    if (count > 0 && !inst) return IM_EINVAL;
    if (workers == 0) return IM_EINVAL;
    for (uint32_t i = 0; i < count; ++i) {
        const im_instance& in = inst[i];
        if (!in.seeds_out || !in.gains_out || !in.spread_out || (in.m > 0 && (!in.u || !in.v)))
            return IM_EINVAL;
    }
    BatchShared sh;
    sh.inst = inst;
    cudaGetDevice(&sh.device);
    sh.order.resize(count);
    for (uint32_t i = 0; i < count; ++i) sh.order[i] = i;
    // work of an instance: its sketches' edge-sketch pairs, then its vertex-sketch pairs
    std::stable_sort(sh.order.begin(), sh.order.end(), [&](uint32_t a, uint32_t b) {
        const double wa = (double)inst[a].m * inst[a].R + (double)inst[a].n * inst[a].R;
        const double wb = (double)inst[b].m * inst[b].R + (double)inst[b].n * inst[b].R;
        return wa > wb;
    });
    for (uint32_t i = 0; i < count; ++i) {
        const im_instance& in = inst[i];
        sh.res.n = std::max(sh.res.n, in.n);
        sh.res.R = std::max(sh.res.R, in.R);
        sh.res.m = std::max(sh.res.m, in.m);
        sh.res.nc = std::max(sh.res.nc, (uint64_t)in.n * in.R);   // centers and hubs: at most n rows
        const double pe = in.p >= 1.0 ? 1.0 : (in.p > 0.0 ? in.p : 0.0);
        sh.res.pm = std::max(sh.res.pm, pe * (double)in.m);
    }
    const uint32_t w = std::min(workers, std::max(count, 1u));
    std::vector<std::thread> pool;
    pool.reserve(w);
    for (uint32_t t = 0; t < w; ++t) pool.emplace_back(run_worker, &sh);
    for (auto& th : pool) th.join();
    for (uint32_t i = 0; i < count; ++i)
        if (inst[i].status != IM_OK) return inst[i].status;
    return IM_OK;
}

// ---- the batch as one CUDA graph ----------------------------------------------------------
// im_batch_create plans a batch: one context per instance, every buffer reserved, and one CUDA
// graph that holds every instance's whole path -- upload, CSR, sketch construction (Alg. 1 step
// 1, two lanes), the lazy-greedy loop (Alg. 2 / Alg. 4, conditional nodes set by the device),
// the spread and the copies of the results to pinned host memory.  Instances form `branches`
// chains (largest first, dealt round-robin) that the graph runs side by side.  im_batch_run
// launches that graph once and hands out the results: the instances run with no host step
// between their kernels and no launch from the host but one.
struct im_batch {
    int device = 0;
    im_instance* inst = nullptr;
    uint32_t count = 0;
    std::vector<im_ctx*> ctx;
    std::vector<size_t> off;          // per instance: offset of its results in `pinned`
    char* pinned = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

struct Slot {   // an instance's results in pinned memory, written by the graph
    imk::SelState sel;
    unsigned long long spread;
};

size_t slot_bytes(uint32_t k) {
    return ((sizeof(Slot) + (size_t)k * 8 + (size_t)k * 4) + 255) & ~(size_t)255;
}

void batch_free(im_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (im_ctx* c : b->ctx)
        if (c) im_destroy(c);
    if (b->pinned) cudaFreeHost(b->pinned);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// The single node a stream's capture ends at (an empty node joins several).
int capture_frontier(im_ctx* c, cudaGraph_t g, cudaGraphNode_t* out) {
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    IM_CUDA(c, cudaStreamGetCaptureInfo(c->stream, &status, nullptr, nullptr, &deps, nullptr, &ndeps));
    if (status != cudaStreamCaptureStatusActive || ndeps == 0) return im_fail(c, IM_ECUDA, "batch graph capture");
    if (ndeps == 1) {
        *out = deps[0];
        return IM_OK;
    }
    std::vector<cudaGraphNode_t> d(deps, deps + ndeps);
    IM_CUDA(c, cudaGraphAddEmptyNode(out, g, d.data(), d.size()));
    return IM_OK;
}

// Everything of instance i appended to the graph after `after` (or at its root); *last receives
// the node its chain continues from.
int append_instance(im_batch* b, uint32_t i, cudaGraphNode_t after, cudaGraphNode_t* last) {
    im_ctx* c = b->ctx[i];
    const im_instance& in = b->inst[i];
    Slot* slot = reinterpret_cast<Slot*>(b->pinned + b->off[i]);
    uint64_t* h_gains = reinterpret_cast<uint64_t*>(slot + 1);
    uint32_t* h_seeds = reinterpret_cast<uint32_t*>(h_gains + in.k);
    c->cur = c->stream;
    c->capturing = true;
    int rc = IM_OK;
    cudaGraph_t cg = nullptr;
    IM_CUDA(c, cudaStreamBeginCaptureToGraph(c->stream, b->graph, after ? &after : nullptr, nullptr, after ? 1 : 0,
                                             cudaStreamCaptureModeRelaxed));
    rc = batch_load_enqueue(c, in.n, in.m, in.u, in.v);
    if (!rc) {
        c->h_live[2] = 0;
        rc = build_enqueue(c);
    }
    cudaGraphNode_t built = nullptr;
    if (!rc) rc = capture_frontier(c, b->graph, &built);
    cudaError_t e = cudaStreamEndCapture(c->stream, &cg);
    if (!rc && e != cudaSuccess) rc = im_cuda_check(c, e, "batch graph capture");
    cudaGraphNode_t selected = nullptr;
    if (!rc) rc = im_select_graph_append(c, b->graph, built, in.k, &selected);
    if (!rc) {
        IM_CUDA(c, cudaStreamBeginCaptureToGraph(c->stream, b->graph, &selected, nullptr, 1,
                                                 cudaStreamCaptureModeRelaxed));
        if (cudaMemcpyAsync(h_seeds, c->d_seed_list, (size_t)in.k * 4, cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(h_gains, c->d_gain_list, (size_t)in.k * 8, cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(&slot->sel, c->d_sel, sizeof(imk::SelState), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess)
            rc = im_cuda_check(c, cudaGetLastError(), "batch result copies");
        if (!rc) rc = im_spread_enqueue(c, in.k, &slot->spread);
        if (!rc) rc = capture_frontier(c, b->graph, last);
        e = cudaStreamEndCapture(c->stream, &cg);
        if (!rc && e != cudaSuccess) rc = im_cuda_check(c, e, "batch graph capture");
    }
    c->capturing = false;
    c->cur = c->stream;
    return rc;
}

}  // namespace

extern "C" int im_batch_create(im_instance* inst, uint32_t count, const im_batch_schedule* sched, im_batch** out) {
    if (!out || (count > 0 && !inst)) return IM_EINVAL;
    *out = nullptr;
    for (uint32_t i = 0; i < count; ++i) {
        const im_instance& in = inst[i];
        if (!in.seeds_out || !in.gains_out || !in.spread_out || (in.m > 0 && (!in.u || !in.v)) || in.n == 0 ||
            in.k == 0 || in.k > in.n || in.k > 16384 || in.R == 0 || !(in.alpha > 0.0) || in.alpha > 1.0)
            return IM_EINVAL;
    }
    if (sched && sched->classes > 4) return IM_EINVAL;
    im_batch* b = new (std::nothrow) im_batch();
    if (!b) return IM_ENOMEM;
    b->inst = inst;
    b->count = count;
    cudaGetDevice(&b->device);
    b->ctx.assign(count, nullptr);
    b->off.assign(count, 0);
    size_t bytes = 0;
    for (uint32_t i = 0; i < count; ++i) {
        b->off[i] = bytes;
        bytes += slot_bytes(inst[i].k);
    }
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&b->pinned), bytes + 256, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        b->pinned = nullptr;
        batch_free(b);
        return IM_ENOMEM;
    }
    int rc = IM_OK;
    // one context per instance, every buffer reserved for it
    for (uint32_t i = 0; i < count && !rc; ++i) {
        const im_instance& in = inst[i];
        ImReserve res{};
        res.n = in.n;
        res.R = in.R;
        res.m = in.m;
        res.nc = 0;
        res.pm = 0.0;
        im_ctx* c = nullptr;
        rc = im_create_reserved(&c, in.n, 0, nullptr, nullptr, IM_PTR_HOST, nullptr, &res);
        if (rc) break;
        b->ctx[i] = c;
        if (sched && sched->classes) {   // the knobs of the instance's size class
            const double pairs = (double)in.m * in.R;
            uint32_t cl = sched->classes - 1;
            for (uint32_t j = 0; j + 1 < sched->classes; ++j)
                if (pairs <= (double)sched->class_pairs[j]) { cl = j; break; }
            rc = im_set_sketch_batch(c, sched->sketch_batch[cl]);
            if (!rc) rc = im_set_pipeline(c, sched->lanes[cl] ? sched->lanes[cl] : 2);
            if (!rc) rc = im_set_union_path(c, (int)sched->union_path[cl]);
        }
        if (!rc) rc = batch_load_reserve(c, in.n, in.m);
        if (!rc) rc = build_prepare(c, in.R, in.seed, in.p, in.alpha);
        if (!rc) rc = im_select_prepare(c, in.k);
    }
    // the graph: chains of instances, largest first, dealt round-robin
    std::vector<uint32_t> order(count);
    for (uint32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c2) {
        return (double)inst[a].m * inst[a].R + (double)inst[a].n * inst[a].R >
               (double)inst[c2].m * inst[c2].R + (double)inst[c2].n * inst[c2].R;
    });
    uint32_t branches = sched && sched->branches ? sched->branches : 8u;
    branches = std::max(1u, std::min(branches, std::max(count, 1u)));
    if (!rc && cudaGraphCreate(&b->graph, 0) != cudaSuccess) rc = IM_ECUDA;
    std::vector<cudaGraphNode_t> last(branches, nullptr);
    for (uint32_t j = 0; j < count && !rc; ++j) {
        const uint32_t i = order[j];
        rc = append_instance(b, i, last[j % branches], &last[j % branches]);
    }
    if (!rc && count > 0 && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = IM_ECUDA;
    if (rc) {
        cudaGetLastError();
        batch_free(b);
        return rc;
    }
    *out = b;
    return IM_OK;
}

extern "C" int im_batch_run(im_batch* b) {
    if (!b) return IM_EINVAL;
    if (b->count == 0) return IM_OK;
    cudaSetDevice(b->device);
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        for (uint32_t i = 0; i < b->count; ++i) b->inst[i].status = IM_ECUDA;
        return IM_ECUDA;
    }
    int first = IM_OK;
    for (uint32_t i = 0; i < b->count; ++i) {
        im_instance& in = b->inst[i];
        const Slot* slot = reinterpret_cast<const Slot*>(b->pinned + b->off[i]);
        const uint64_t* h_gains = reinterpret_cast<const uint64_t*>(slot + 1);
        const uint32_t* h_seeds = reinterpret_cast<const uint32_t*>(h_gains + in.k);
        int st = IM_OK;
        if (b->ctx[i]->h_live[3]) st = IM_EINVAL;   // an edge id >= n or a self-loop
        else if (slot->sel.err || slot->sel.fb_overflow || slot->sel.round < in.k) st = IM_EDEVICE;
        if (!st) {
            memcpy(in.seeds_out, h_seeds, (size_t)in.k * 4);
            memcpy(in.gains_out, h_gains, (size_t)in.k * 8);
            *in.spread_out = slot->spread;
        }
        in.status = st;
        if (st && !first) first = st;
    }
    return first;
}

extern "C" int im_batch_destroy(im_batch* b) {
    if (!b) return IM_EINVAL;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    return IM_OK;
}

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Build + selection of one instance with the given union path, timed (the context holds its graph).
double time_union_path(im_ctx* c, const im_instance& in, int path) {
    if (im_set_union_path(c, path)) return 1e30;
    double best = 1e30;
    for (int rep = 0; rep < 2; ++rep) {
        const double t0 = now_ms();
        int rc = im_build_sketches(c, in.R, in.seed, in.p, in.alpha);
        std::vector<uint32_t> sd(in.k);
        if (!rc) rc = im_select_seeds(c, in.k, sd.data(), nullptr);
        if (rc) return 1e30;
        if (rep) best = std::min(best, now_ms() - t0);
    }
    return best;
}

}  // namespace

extern "C" int im_batch_tune(im_instance* inst, uint32_t count, im_batch_schedule* out) {
    if (!out || (count > 0 && !inst)) return IM_EINVAL;
    im_batch_schedule s{};
    s.classes = 3;
    s.class_pairs[0] = 1ull << 28;   // small instances: latency-bound rounds
    s.class_pairs[1] = 1ull << 31;
    int rc = IM_OK;
    for (uint32_t cl = 0; cl < s.classes && !rc; ++cl) {
        // the class's largest instance (by m R)
        int pick = -1;
        for (uint32_t i = 0; i < count; ++i) {
            const double pairs = (double)inst[i].m * inst[i].R;
            uint32_t c2 = s.classes - 1;
            for (uint32_t j = 0; j + 1 < s.classes; ++j)
                if (pairs <= (double)s.class_pairs[j]) { c2 = j; break; }
            if (c2 == cl && (pick < 0 || pairs > (double)inst[pick].m * inst[pick].R)) pick = (int)i;
        }
        if (pick < 0) continue;
        const im_instance& in = inst[pick];
        im_ctx* c = nullptr;
        rc = im_create(&c, in.n, in.m, in.u, in.v, IM_PTR_HOST, nullptr);
        if (rc) break;
        im_tuning t{};
        rc = im_autotune(c, in.R, in.seed, in.p, in.alpha, in.k, 1, &t);
        if (!rc) {
            s.sketch_batch[cl] = t.sketch_batch;
            s.lanes[cl] = t.lanes;
            im_set_sketch_batch(c, t.sketch_batch);
            im_set_pipeline(c, t.lanes);
            im_set_hubs(c, t.hub_cap, 32);
            double best_t = 1e30;
            for (int path : {IM_UNION_RECORDS, IM_UNION_BUCKETS, IM_UNION_FUSED}) {
                const double t_path = time_union_path(c, in, path);
                if (t_path < best_t) { best_t = t_path; s.union_path[cl] = (uint32_t)path; }
            }
        }
        im_destroy(c);
    }
    if (rc) return rc;
    // branches: whole batches, each run twice (the second timed)
    double best = 1e30;
    uint32_t best_b = 8;
    for (uint32_t br : {4u, 8u, 16u}) {
        s.branches = br;
        im_batch* b = nullptr;
        rc = im_batch_create(inst, count, &s, &b);
        if (rc) return rc;
        rc = im_batch_run(b);
        const double t0 = now_ms();
        if (!rc) rc = im_batch_run(b);
        const double dt = now_ms() - t0;
        im_batch_destroy(b);
        if (rc) return rc;
        if (dt < best) { best = dt; best_b = br; }
    }
    s.branches = best_b;
    s.run_ms = best;
    *out = s;
    return IM_OK;
}
