// im_tune.cu -- measured choice of the knobs that change the speed of the sketch build and the
// selection but none of their results: sketches per edge pass, sketch batches in flight and
// (compact sketches) hubs.  Host code over the public calls; every combination is checked to
// give the same seeds.
#include <chrono>
#include <cstring>
#include <vector>

#include "im_internal.cuh"

namespace {

struct Knobs {
    uint32_t batch, lanes, hubs;
};

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" int im_autotune(im_ctx* c, uint32_t R, uint64_t seed, double p, double alpha, uint32_t k, uint32_t reps,
                           im_tuning* out) {
    if (!c) return IM_EINVAL;
    if (!out) return im_fail(c, IM_EINVAL, "out is NULL");
    if (reps == 0) return im_fail(c, IM_EINVAL, "reps must be at least 1");
    if (k == 0 || k > c->n) return im_fail(c, IM_EINVAL, "k must be in [1, n]");
    memset(out, 0, sizeof(*out));
    const uint32_t min_deg = c->hub_min_deg;
    std::vector<Knobs> grid;
    for (uint32_t hubs : {(uint32_t)IM_HUBS_AUTO, 0u}) {
        if (hubs == 0 && alpha >= 1.0) continue;   // every vertex is a center: no hubs to choose
        for (uint32_t lanes : {2u, 1u})
            for (uint32_t batch : {0u, 16u, 8u}) grid.push_back({batch, lanes, hubs});
    }
    std::vector<uint32_t> first, seeds(k);
    double best = 0.0;
    for (size_t i = 0; i < grid.size(); ++i) {
        const Knobs& kn = grid[i];
        int rc = im_set_sketch_batch(c, kn.batch);
        if (!rc) rc = im_set_pipeline(c, kn.lanes);
        if (!rc) rc = im_set_hubs(c, kn.hubs, min_deg);
        double tb = 0.0, ts = 0.0;
        for (uint32_t rep = 0; !rc && rep <= reps; ++rep) {
            const auto t0 = std::chrono::steady_clock::now();
            rc = im_build_sketches(c, R, seed, p, alpha);
            const double b = ms_since(t0);
            if (rc) break;
            const auto t1 = std::chrono::steady_clock::now();
            rc = im_select_seeds(c, k, seeds.data(), nullptr);
            const double s = ms_since(t1);
            if (rc) break;
            if (rep == 1 || (rep > 1 && b + s < tb + ts)) {   // rep 0 warms up
                tb = b;
                ts = s;
            }
        }
        if (rc) return rc;
        if (first.empty()) {
            first = seeds;
            out->default_build_ms = tb;
            out->default_select_ms = ts;
        } else if (seeds != first) {
            return im_fail(c, IM_EDEVICE, "autotuning: a combination of knobs changed the seeds");
        }
        out->tried = (uint32_t)(i + 1);
        if (i == 0 || tb + ts < best) {
            best = tb + ts;
            out->sketch_batch = kn.batch;
            out->lanes = kn.lanes;
            out->hub_cap = kn.hubs;
            out->build_ms = tb;
            out->select_ms = ts;
        }
    }
    int rc = im_set_sketch_batch(c, out->sketch_batch);
    if (!rc) rc = im_set_pipeline(c, out->lanes);
    if (!rc) rc = im_set_hubs(c, out->hub_cap, min_deg);
    if (!rc) rc = im_build_sketches(c, R, seed, p, alpha);
    return rc;
}
