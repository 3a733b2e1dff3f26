// im_server.cu -- a serving engine over resident sketch sets.  A model is one graph with its
// IC probability, R, seed and alpha; its sketches are built once, when it is admitted, and
// stay in HBM.  A request asks a model for k seeds.  Greedy selection is a sequence (Alg. 1
// picks one seed per round), so the answer to k is the first k seeds of the model's sequence
// and its spread estimate the sum of their marginal gains (telescoping); the engine extends
// a model's sequence only as far as the largest k asked so far.  Every model has a host
// thread that takes all of its pending requests at once (continuous batching: one selection
// run to their largest k answers them all) and runs on the model's own stream, so requests on
// different models overlap on the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "im_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Model {
    im_ctx* ctx = nullptr;
    uint32_t n = 0;
    uint64_t footprint = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<im_request*> q;
    bool stop = false;
    std::vector<uint32_t> seeds;   // the greedy sequence chosen so far
    std::vector<uint64_t> gains;
};

}  // namespace

struct im_server {
    int device = 0;
    std::vector<Model*> models;
    uint64_t admitted_bytes = 0;
    Clock::time_point t0;
    std::mutex done_mu;
    std::condition_variable done_cv;
    uint32_t outstanding = 0;
};

namespace {

uint64_t now_ns(const im_server* s) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - s->t0).count();
}

// Device bytes a model will hold: the graph (edge list, arcs with their keys, offsets, arc
// cursors, upload staging), the per-vertex selection arrays, two lanes of union-find scratch
// for B sketches, their live-pair records, the compact (and hub) rows and the fallback queues
// (as im_graph_build and im_build_sketches size them).
uint64_t footprint_estimate(uint32_t n, uint64_t m, uint32_t R, double p, double alpha) {
    uint64_t B = 32;
    while (B > 1 && B * (uint64_t)n * 12 > (8ull << 30)) B /= 2;
    uint64_t rp2 = 1;
    while (rp2 < R) rp2 <<= 1;
    if (B > rp2) B = rp2;
    const double rho = std::min<double>(n, std::ceil(alpha * n));
    const double hubs = rho >= n ? 0.0 : std::min<double>(std::max<double>(1024.0, n / 64.0), n - rho);
    const double pe = p >= 1.0 ? 1.0 : (p > 0.0 ? p : 0.0);
    const double ex = pe * (double)m * B;
    const double live = ex > 0 ? std::min(1.3 * ex + 16.0 * std::sqrt(ex) + 65536.0, (double)(1ull << 28)) : 0.0;
    const double graph = 8.0 * m + 32.0 * m + 8.0 * n + 8.0 * n + 8.0 * m;
    const double vertex = 80.0 * n + 8.0 * 4 * n + 8.0 * (n / 32.0) * 4 + 40.0 * n;
    const double lanes = 2.0 * B * n * 12.0 + 2.0 * live * 16.0;
    const double compact = 8.0 * (rho + hubs) * R + 8.0 * 256.0 * R;
    return (uint64_t)(graph + vertex + lanes + compact) + (64ull << 20);
}

void model_loop(im_server* s, Model* md) {
    cudaSetDevice(s->device);
    std::vector<im_request*> batch;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(md->mu);
            md->cv.wait(lk, [&] { return md->stop || !md->q.empty(); });
            if (md->q.empty() && md->stop) return;
            batch.assign(md->q.begin(), md->q.end());   // every request pending now
            md->q.clear();
        }
        uint32_t kmax = 0;
        for (im_request* r : batch) kmax = std::max(kmax, r->k);
        int rc = IM_OK;
        if (kmax > md->seeds.size()) {
            md->seeds.resize(kmax);
            md->gains.resize(kmax);
            rc = im_select_seeds(md->ctx, kmax, md->seeds.data(), md->gains.data());
            if (rc) {
                md->seeds.resize(md->ctx->seeds.size());
                md->gains.resize(md->ctx->seed_gains.size());
            }
        }
        for (im_request* r : batch) {
            if (r->k <= md->seeds.size()) {
                uint64_t sp = 0;
                for (uint32_t i = 0; i < r->k; ++i) {
                    if (r->seeds_out) r->seeds_out[i] = md->seeds[i];
                    if (r->gains_out) r->gains_out[i] = md->gains[i];
                    sp += md->gains[i];
                }
                if (r->spread_out) *r->spread_out = sp;
                r->status = IM_OK;
            } else {
                r->status = rc ? rc : IM_EDEVICE;
            }
            r->done_ns = now_ns(s);
        }
        {
            std::lock_guard<std::mutex> lk(s->done_mu);
            s->outstanding -= (uint32_t)batch.size();
        }
        s->done_cv.notify_all();
        batch.clear();
    }
}

}  // namespace

extern "C" {

int im_server_create(im_server** out) {
    if (!out) return IM_EINVAL;
    im_server* s = new (std::nothrow) im_server();
    if (!s) return IM_ENOMEM;
    cudaGetDevice(&s->device);
    s->t0 = Clock::now();
    *out = s;
    return IM_OK;
}

int im_server_add_model(im_server* s, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v, uint32_t R,
                        uint64_t seed, double p, double alpha, uint32_t* model_out, uint64_t* footprint_out) {
    if (!s || !model_out) return IM_EINVAL;
    const uint64_t need = footprint_estimate(n, m, R, p, alpha);
    if (footprint_out) *footprint_out = need;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return IM_ECUDA;
    if (need + (2ull << 30) > free_b) return IM_ENOMEM;   // admission: keep 2 GiB free
    Model* md = new (std::nothrow) Model();
    if (!md) return IM_ENOMEM;
    int rc = im_create(&md->ctx, n, m, u, v, IM_PTR_HOST, nullptr);
    if (!rc) rc = im_build_sketches(md->ctx, R, seed, p, alpha);
    if (rc) {
        if (md->ctx) im_destroy(md->ctx);
        delete md;
        return rc;
    }
    md->n = n;
    md->footprint = need;
    s->admitted_bytes += need;
    *model_out = (uint32_t)s->models.size();
    s->models.push_back(md);
    md->th = std::thread(model_loop, s, md);
    return IM_OK;
}

int im_server_replay(im_server* s, im_request* req, uint32_t count) {
    if (!s || (count > 0 && !req)) return IM_EINVAL;
    for (uint32_t i = 0; i < count; ++i) {
        if (req[i].model >= s->models.size()) return IM_EINVAL;
        if (req[i].k == 0 || req[i].k > s->models[req[i].model]->n) return IM_EINVAL;
    }
    std::vector<uint32_t> order(count);
    for (uint32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return req[a].arrival_ns < req[b].arrival_ns; });
    {
        std::lock_guard<std::mutex> lk(s->done_mu);
        s->outstanding += count;
    }
    const Clock::time_point start = Clock::now();
    const uint64_t base = now_ns(s);
    for (uint32_t i : order) {
        im_request* r = &req[i];
        std::this_thread::sleep_until(start + std::chrono::nanoseconds(r->arrival_ns));
        r->submit_ns = now_ns(s) - base;
        r->status = IM_EDEVICE;
        Model* md = s->models[r->model];
        {
            std::lock_guard<std::mutex> lk(md->mu);
            md->q.push_back(r);
        }
        md->cv.notify_one();
    }
    {
        std::unique_lock<std::mutex> lk(s->done_mu);
        s->done_cv.wait(lk, [&] { return s->outstanding == 0; });
    }
    for (uint32_t i = 0; i < count; ++i) req[i].done_ns -= base;
    for (uint32_t i = 0; i < count; ++i)
        if (req[i].status != IM_OK) return req[i].status;
    return IM_OK;
}

int im_server_destroy(im_server* s) {
    if (!s) return IM_EINVAL;
    for (Model* md : s->models) {
        {
            std::lock_guard<std::mutex> lk(md->mu);
            md->stop = true;
        }
        md->cv.notify_one();
    }
    for (Model* md : s->models) {
        if (md->th.joinable()) md->th.join();
        im_destroy(md->ctx);
        delete md;
    }
    delete s;
    return IM_OK;
}

}  // extern "C"
