// im_peak.cu -- the compute ceiling of the sampling kernel, measured: the candidate test of
// k_sample_emit (64-bit add, the hash's high word, compare, live-mask update) on register
// values only, so that its rate bounds what the sampling can reach with no memory traffic.
#include "im_internal.cuh"

using namespace imk;

namespace {

// Each thread tests `iters` consecutive sketches for 2 independent keys (as k_sample_emit
// does for its two edges), 32 sketches per unrolled step.
__global__ void __launch_bounds__(256)
k_hash_peak(uint64_t salt, uint32_t th1, uint32_t iters, unsigned int* __restrict__ sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x0 = mix64(salt ^ (2 * tid)) + kGamma, x1 = mix64(salt ^ (2 * tid + 1)) + kGamma;
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; it += 32) {
        uint32_t live0 = 0, live1 = 0;
#pragma unroll
        for (int b = 0; b < 32; ++b) {
            if (mix64_hi_raw(x0) <= th1) live0 |= 1u << b;
            if (mix64_hi_raw(x1) <= th1) live1 |= 1u << b;
            x0 += kGamma;
            x1 += kGamma;
        }
        acc += __popc(live0) + __popc(live1);
    }
    if (acc == 0xFFFFFFFFu) sink[0] = acc;   // keeps the work observable; never taken in practice
}

}  // namespace

extern "C" int im_hash_peak(uint32_t iters, double* pairs_per_s) {
    if (!pairs_per_s || iters == 0 || iters % 32) return IM_EINVAL;
    const unsigned blocks = 152u * 8u, threads = 256u;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    unsigned int* sink = nullptr;
    int rc = IM_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(unsigned int)) != cudaSuccess) {
        rc = IM_ECUDA;
    } else {
        const uint32_t th1 = (uint32_t)(0.02 * 4294967296.0) + 1u;   // p = 0.02, as on the bench
        k_hash_peak<<<blocks, threads, 0, s>>>(0x1234u, th1, 32, sink);   // warm-up
        cudaEventRecord(e0, s);
        k_hash_peak<<<blocks, threads, 0, s>>>(0x5678u, th1, iters, sink);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            ms <= 0.f) {
            rc = IM_ECUDA;
        } else {
            *pairs_per_s = 2.0 * iters * (double)blocks * threads / (ms * 1e-3);
        }
    }
    cudaGetLastError();
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return rc;
}
