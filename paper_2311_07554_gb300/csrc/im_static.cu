// im_static.cu -- im_sketch_static: the components of one sketch without any allocation.
//
// Same arithmetic as the batched build (hash sampling, union-find with smallest-id hooking,
// compression, component histogram) for a single sketch, but its union-find scratch lives in
// one file-scope device array of fixed size instead of memory obtained from cudaMalloc.
// Host code must not pass the array's name to a kernel (on the host it is only a stand-in
// symbol); its device address comes from cudaGetSymbolAddress in the current context.
#include <cmath>
#include <mutex>

#include "im_internal.cuh"
#include "im_uf.cuh"

using namespace imk;

namespace {

// [0, IM_STATIC_MAX_N): parent, [IM_STATIC_MAX_N, 2*IM_STATIC_MAX_N): component counts,
// then one status word (bad edge ids).
constexpr size_t kStaticWords = 2 * (size_t)IM_STATIC_MAX_N + 64;
static __device__ __align__(256) uint32_t g_static_scratch[kStaticWords];

constexpr int kMaxDevices = 256;
std::mutex g_static_mu;
uint32_t* g_static_ptr[kMaxDevices] = {};

__global__ void k_static_init(uint32_t* __restrict__ P, uint32_t* __restrict__ C,
                              uint32_t* __restrict__ status, uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        P[v] = v;
        C[v] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

// one edge per thread; edges with an id >= n or a self-loop are skipped and reported
__global__ void k_static_sample_union(const uint32_t* __restrict__ u, const uint32_t* __restrict__ v,
                                      uint64_t m, uint32_t n, Sampler smp, uint32_t r,
                                      uint32_t* __restrict__ P, uint32_t* __restrict__ status) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t a = u[e], b = v[e];
        if (a >= n || b >= n || a == b) {
            atomicOr(status, 1u);
            continue;
        }
        if (edge_live(smp, edge_key(smp, e), r)) unite_min(P, a, b);
    }
}

__global__ void k_static_compress(uint32_t* __restrict__ P, uint32_t* __restrict__ C, uint32_t n) {
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        const bool act = v < n;
        uint32_t root = 0;
        if (act) root = compress_to_root(P, v);
        const unsigned am = __ballot_sync(0xffffffffu, act);
        if (act) {
            const unsigned grp = __match_any_sync(am, root);
            if ((threadIdx.x & 31) == (unsigned)(__ffs(grp) - 1)) atomicAdd(C + root, __popc(grp));
        }
    }
}

__global__ void k_static_write(const uint32_t* __restrict__ P, const uint32_t* __restrict__ C,
                               uint32_t n, uint32_t* __restrict__ labels,
                               uint32_t* __restrict__ sizes) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint32_t root = P[v];
        if (labels) labels[v] = root;
        if (sizes) sizes[v] = C[root];
    }
}

// Device address of the static scratch in the current context.  Outside stream capture it is
// looked up on every call (cudaGetSymbolAddress allocates nothing), so a context created
// after a cudaDeviceReset, or a non-primary context made current, gets its own address; the
// last address found on each device is kept for calls made while `st` is being captured,
// which must not make runtime calls that are not stream operations.
cudaError_t static_scratch(cudaStream_t st, uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = (uint32_t*)p;
    } else if (!g_static_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

// failures are reported through im_last_error(NULL), like those of im_create
int static_fail(int code, const std::string& msg) { return im_fail(nullptr, code, msg); }

}  // namespace

extern "C" int im_sketch_static(uint32_t n, uint64_t m, const uint32_t* d_u, const uint32_t* d_v,
                                uint64_t seed, double p, uint32_t r, uint32_t* d_labels,
                                uint32_t* d_sizes, void* stream) {
    if (n == 0 || n > IM_STATIC_MAX_N)
        return static_fail(IM_EINVAL, "n must be in [1, IM_STATIC_MAX_N]");
    if (m >= 0xFFFFFFFFull) return static_fail(IM_EINVAL, "m must be < 2^32");
    if (m > 0 && (!d_u || !d_v)) return static_fail(IM_EINVAL, "edge arrays are NULL");
    if (!d_labels && !d_sizes) return static_fail(IM_EINVAL, "no output requested");
    if (p != p) return static_fail(IM_EINVAL, "p is NaN");
    uint32_t* base = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = static_scratch(st, &base);
    if (e != cudaSuccess) return static_fail(IM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    uint32_t* P = base;
    uint32_t* C = base + IM_STATIC_MAX_N;
    uint32_t* status = base + 2 * (size_t)IM_STATIC_MAX_N;
    Sampler smp{};   // one p for every edge: no per-edge thresholds
    smp.salt = mix64(seed + kGamma);
    smp.all_live = p >= 1.0 ? 1u : 0u;
    smp.T = (p > 0.0 && p < 1.0) ? (uint64_t)std::ldexp(p, 64) : 0ull;
    const unsigned T = 256;
    k_static_init<<<grid_for(n, T, 152u * 8u), T, 0, st>>>(P, C, status, n);
    if (m > 0) k_static_sample_union<<<grid_for(m, T, 152u * 16u), T, 0, st>>>(d_u, d_v, m, n, smp, r, P, status);
    k_static_compress<<<grid_for(n, T, 152u * 8u), T, 0, st>>>(P, C, n);
    k_static_write<<<grid_for(n, T, 152u * 8u), T, 0, st>>>(P, C, n, d_labels, d_sizes);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(IM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    uint32_t bad = 0;
    e = cudaMemcpyAsync(&bad, status, sizeof bad, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_fail(IM_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
    if (bad) return static_fail(IM_EINVAL, "edge list has an id >= n or a self-loop");
    return IM_OK;
}
