// im_batch.cu -- many independent IM instances on one device (Alg. 1 per instance: sketches,
// lazy greedy, spread), run by a pool of host workers, each owning one context and its own
// stream, so that the instances' kernels overlap on the GPU.  A worker keeps its context
// across instances: im_load_graph and im_build_sketches reuse the buffers while an instance
// fits them (no cudaMalloc / cudaFree, which would synchronise the whole device and stall
// the other workers), so instances are handed out largest first.
#include <algorithm>
#include <atomic>
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
