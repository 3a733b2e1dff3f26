// im_server.cu -- a serving engine over sketch sets held in HBM under a memory budget.
//
// A model is one graph with its IC probability, R, seed and alpha.  A request asks a model for
// k seeds.  Greedy selection is a sequence (Alg. 1 picks one seed per round), so the answer to
// k is the first k seeds of the model's sequence and its spread estimate the sum of their
// marginal gains (telescoping).  The engine keeps every model's sequence found so far on the
// host and extends it on the device only as far as the largest k asked.
//
// Residency: a model's sketches occupy its estimated footprint of the engine's budget while it
// is resident.  A request for a model that is not resident waits for admission: if its
// footprint fits under the budget it is built; otherwise the least recently used resident
// model that is idle (no request pending or running) is evicted -- its context and sketches
// freed, its sequence kept on the host -- and admission is tried again; if no model can be
// evicted the request waits until one finishes.  A request that the host prefix already
// answers needs no residency at all.  Rebuilt sketches are bit-identical (the sampling is a
// fixed hash), so every answer equals the one the model gives alone.
//
// Serving on the device: each resident model has a mailbox and a device-resident request
// loop (im_serve_launch).  The model's host thread takes all of its pending requests at once,
// pushes the largest k into the mailbox, launches the loop only if none is running, and waits
// for the seeds to be published; the loop stays on the device for idle_us after its last
// request, so a model under load answers request after request with no new launch.  Requests
// on different models run on their own contexts and streams and overlap on the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "im_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Model {
    // registration (host copies of the edge lists, for builds after an eviction)
    uint32_t n = 0;
    uint64_t m = 0;
    std::vector<uint32_t> u, v;
    uint32_t R = 0;
    uint64_t seed = 0;
    double p = 0.0, alpha = 1.0;
    uint64_t footprint = 0;
    // residency (guarded by the server's mutex)
    im_ctx* ctx = nullptr;
    im_mailbox* mb = nullptr;
    bool resident = false;   // its footprint is counted in the budget
    bool busy = false;       // its thread is building or serving
    uint64_t last_use = 0;
    uint32_t builds = 0, evictions = 0;
    // requests
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<im_request*> q;
    bool stop = false;
    std::vector<uint32_t> seeds;   // the greedy sequence known so far (kept across evictions)
    std::vector<uint64_t> gains;
};

// A model's device loop waits this long for its next request.  A waiting loop holds one block on
// an SM, and the selection's step kernels are sized to fill every SM once, so loops left waiting
// on other models push those kernels into a second wave: with 50 ms the serving workload's p99
// was 139 ms, with 1-5 ms 53 ms.
constexpr uint32_t kLoopIdleUs = 2000;
constexpr uint32_t kWaitUs = 120000000;   // a request's answer, at most (two minutes)

}  // namespace

struct im_server {
    int device = 0;
    std::vector<Model*> models;
    uint64_t budget = 0;
    uint64_t used = 0;
    uint64_t tick = 0;
    std::mutex mu;                    // residency of every model
    std::condition_variable freed;    // a model became idle or was evicted
    Clock::time_point t0;
    std::mutex done_mu;
    std::condition_variable done_cv;
    uint32_t outstanding = 0;
};

namespace {

uint64_t now_ns(const im_server* s) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - s->t0).count();
}

// Device bytes a model holds when resident: the graph (edge list, 16-byte arcs, static
// adjacency and sources, offsets, arc cursors, upload staging), the per-vertex selection
// arrays, two lanes of union-find scratch for B sketches with their live-pair records, the
// compact (and hub) rows, the fallback queues and fixed scratch -- as im_create and
// im_build_sketches size them.
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
    const double graph = 8.0 * m + 32.0 * m + 16.0 * m + 8.0 * m + 8.0 * n + 8.0 * n;
    const double vertex = 80.0 * n + 8.0 * 4 * n + 8.0 * (n / 32.0) * 4 + 48.0 * n;
    const double lanes = 2.0 * B * n * 12.0 + 2.0 * live * 16.0 + 2.0 * 8.0 * 8.0 * n;
    const double compact = 8.0 * (rho + hubs) * R + 8.0 * 256.0 * R;
    return (uint64_t)(graph + vertex + lanes + compact) + (96ull << 20);
}

// Frees a resident model's device state (the caller holds the server's mutex; the model is idle).
void evict(im_server* s, Model* md) {
    if (md->mb) {
        im_serve_finish(md->mb, nullptr);   // its loop may still be waiting on the device
        im_mailbox_destroy(md->mb);
        md->mb = nullptr;
    }
    if (md->ctx) im_destroy(md->ctx);
    md->ctx = nullptr;
    md->resident = false;
    s->used -= md->footprint;
    md->evictions++;
}

// Admission: wait until the model's footprint fits under the budget, evicting idle models
// (least recently used first).  Returns IM_ENOMEM if it can never fit.
int admit(im_server* s, Model* md) {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (md->resident) break;
        if (md->footprint > s->budget) return IM_ENOMEM;
        if (s->used + md->footprint <= s->budget) {
            s->used += md->footprint;
            md->resident = true;
            break;
        }
        Model* victim = nullptr;
        for (Model* o : s->models) {
            if (o == md || !o->resident || o->busy) continue;
            {
                std::lock_guard<std::mutex> ql(o->mu);
                if (!o->q.empty()) continue;
            }
            if (!victim || o->last_use < victim->last_use) victim = o;
        }
        if (victim) {
            evict(s, victim);
            continue;
        }
        s->freed.wait(lk);   // every resident model is busy: wait until one is done
    }
    md->busy = true;
    return IM_OK;
}

void release(im_server* s, Model* md) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        md->busy = false;
        md->last_use = ++s->tick;
    }
    s->freed.notify_all();
}

// Builds the model's sketches if it has none (after admission), with its mailbox.
int ensure_built(im_server* s, Model* md) {
    if (md->ctx) return IM_OK;
    cudaSetDevice(s->device);
    int rc = im_create(&md->ctx, md->n, md->m, md->u.data(), md->v.data(), IM_PTR_HOST, nullptr);
    if (!rc) rc = im_build_sketches(md->ctx, md->R, md->seed, md->p, md->alpha);
    if (!rc) rc = im_mailbox_create(md->ctx, 64, md->n, &md->mb);
    if (rc) {
        if (md->ctx) im_destroy(md->ctx);
        md->ctx = nullptr;
        md->mb = nullptr;
        std::lock_guard<std::mutex> lk(s->mu);
        md->resident = false;
        s->used -= md->footprint;
        return rc;
    }
    md->builds++;
    return IM_OK;
}

// Extends the model's sequence to kmax seeds through its device loop.
int extend(Model* md, uint32_t kmax) {
    int rc = im_mailbox_push(md->mb, kmax);
    if (rc) return rc;
    uint32_t running = 0;
    im_mailbox_state(md->mb, &running, nullptr, nullptr);
    if (!running) rc = im_serve_launch(md->mb, kLoopIdleUs);
    if (!rc) {
        md->seeds.resize(kmax);
        md->gains.resize(kmax);
        rc = im_mailbox_wait(md->mb, kmax, kWaitUs, md->seeds.data(), md->gains.data());
        if (rc == IM_ESTATE) {   // the loop idled out just before the push: start another
            rc = im_serve_launch(md->mb, kLoopIdleUs);
            if (!rc) rc = im_mailbox_wait(md->mb, kmax, kWaitUs, md->seeds.data(), md->gains.data());
        }
    }
    return rc;
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
        if (kmax > md->seeds.size()) {   // the host prefix does not answer them all
            const size_t have = md->seeds.size();
            rc = admit(s, md);
            if (!rc) {
                rc = ensure_built(s, md);
                if (!rc) rc = extend(md, kmax);
                if (rc) {
                    md->seeds.resize(have);
                    md->gains.resize(have);
                }
                release(s, md);
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

int im_footprint_estimate(uint32_t n, uint64_t m, uint32_t R, double p, double alpha, uint64_t* bytes_out) {
    if (!bytes_out || n == 0 || R == 0 || !(alpha > 0.0) || alpha > 1.0) return IM_EINVAL;
    *bytes_out = footprint_estimate(n, m, R, p, alpha);
    return IM_OK;
}

int im_server_create(im_server** out) {
    if (!out) return IM_EINVAL;
    im_server* s = new (std::nothrow) im_server();
    if (!s) return IM_ENOMEM;
    cudaGetDevice(&s->device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return IM_ECUDA;
    }
    s->budget = free_b > (2ull << 30) ? free_b - (2ull << 30) : 0;   // keep 2 GiB of the device free
    s->t0 = Clock::now();
    *out = s;
    return IM_OK;
}

int im_server_set_budget(im_server* s, uint64_t bytes) {
    if (!s) return IM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (bytes < s->used) return IM_ESTATE;   // resident models already hold more
    s->budget = bytes;
    return IM_OK;
}

int im_server_add_model(im_server* s, uint32_t n, uint64_t m, const uint32_t* u, const uint32_t* v, uint32_t R,
                        uint64_t seed, double p, double alpha, uint32_t* model_out, uint64_t* footprint_out) {
    if (!s || !model_out || n == 0 || R == 0 || (m > 0 && (!u || !v))) return IM_EINVAL;
    if (!(alpha > 0.0) || alpha > 1.0 || std::isnan(p)) return IM_EINVAL;
    for (uint64_t e = 0; e < m; ++e)
        if (u[e] >= n || v[e] >= n || u[e] == v[e]) return IM_EINVAL;
    const uint64_t need = footprint_estimate(n, m, R, p, alpha);
    if (footprint_out) *footprint_out = need;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (need > s->budget) return IM_ENOMEM;   // can never be resident: refused, nothing allocated
    }
    Model* md = new (std::nothrow) Model();
    if (!md) return IM_ENOMEM;
    md->n = n;
    md->m = m;
    md->u.assign(u, u + m);
    md->v.assign(v, v + m);
    md->R = R;
    md->seed = seed;
    md->p = p;
    md->alpha = alpha;
    md->footprint = need;
    // built now if it fits without evicting anyone; otherwise at its first request
    bool now = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->used + need <= s->budget) {
            s->used += need;
            md->resident = true;
            md->busy = true;
            now = true;
        }
    }
    if (now) {
        const int rc = ensure_built(s, md);
        if (rc) {
            delete md;
            return rc;
        }
        release(s, md);
    }
    *model_out = (uint32_t)s->models.size();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->models.push_back(md);
    }
    md->th = std::thread(model_loop, s, md);
    return IM_OK;
}

int im_server_stats(im_server* s, uint32_t model, im_model_stats* out) {
    if (!s || !out) return IM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (model >= s->models.size()) return IM_EINVAL;
    const Model* md = s->models[model];
    out->footprint = md->footprint;
    out->builds = md->builds;
    out->evictions = md->evictions;
    out->resident = md->resident ? 1u : 0u;
    out->known_seeds = (uint32_t)md->seeds.size();
    out->budget = s->budget;
    out->used = s->used;
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
        if (md->mb) {
            im_serve_finish(md->mb, nullptr);
            im_mailbox_destroy(md->mb);
        }
        if (md->ctx) im_destroy(md->ctx);
        delete md;
    }
    delete s;
    return IM_OK;
}

}  // extern "C"
