// im_uf.cuh -- union-find primitives shared by the sketch kernels (internal).
#pragma once

#include "im_internal.cuh"

namespace imk {

// ---- union-find ---------------------------------------------------------------------
// Reads go through L2 (__ldcg) so that a spin over a root another SM has just hooked
// always sees the new parent.

template <bool kAll>
__device__ __forceinline__ bool uf_before(const uint32_t* __restrict__ cbits, uint32_t a, uint32_t b) {
    if (kAll) return a < b;
    uint32_t ca = (__ldg(cbits + (a >> 5)) >> (a & 31)) & 1u;
    uint32_t cb = (__ldg(cbits + (b >> 5)) >> (b & 31)) & 1u;
    return ca != cb ? ca > cb : a < b;
}

__device__ __forceinline__ uint32_t find_root(uint32_t* P, uint32_t x) {
    for (;;) {
        uint32_t p = __ldcg(P + x);
        if (p == x) return x;
        uint32_t gp = __ldcg(P + p);
        if (gp == p) return p;
        __stcg(P + x, gp);   // path halving: gp is an ancestor of x
        x = gp;
    }
}

template <bool kAll>
__device__ __forceinline__ void unite(uint32_t* P, const uint32_t* cbits, uint32_t a, uint32_t b) {
    for (;;) {
        a = find_root(P, a);
        b = find_root(P, b);
        if (a == b) return;
        if (uf_before<kAll>(cbits, b, a)) { uint32_t t = a; a = b; b = t; }
        // hook the later root b under the earlier root a
        uint32_t old = atomicCAS(P + b, b, a);
        if (old == b) return;
        b = old;
    }
}

// Full compression once no union runs any more: walk to the (final) root without writing,
// then store that root along the path.  Only the root is ever written, so a concurrent
// compression of an overlapping path cannot leave an intermediate ancestor behind.
__device__ __forceinline__ uint32_t compress_to_root(uint32_t* P, uint32_t v) {
    uint32_t root = v;
    for (uint32_t p = __ldcg(P + root); p != root; p = __ldcg(P + root)) root = p;
    for (uint32_t x = v; x != root;) {
        const uint32_t nx = __ldcg(P + x);
        if (nx != root) __stcg(P + x, root);
        x = nx;
    }
    return root;
}

}  // namespace imk
