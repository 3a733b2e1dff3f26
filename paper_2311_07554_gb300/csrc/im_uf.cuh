// im_uf.cuh -- union-find primitives shared by the sketch kernels (internal).
//
// Parent pointers only ever move to an ancestor and a vertex that stops being a root never
// becomes one again, so a stale parent read from L1 is still an ancestor: climbing it is
// correct, and a stale "is a root" answer is caught by the atomicCAS that hooks it.  Climbs
// therefore read through L1 (__ldca): every climb in a giant component ends at the same root
// entry, which would otherwise be one hot L2 sector for the whole GPU.
#pragma once

#include "im_internal.cuh"

namespace imk {

__device__ __forceinline__ uint32_t find_root(uint32_t* P, uint32_t x) {
    for (;;) {
        uint32_t p = __ldca(P + x);
        if (p == x) return x;
        uint32_t gp = __ldca(P + p);
        if (gp == p) return p;
        __stcg(P + x, gp);   // path halving: gp is an ancestor of x
        x = gp;
    }
}

// Link priority: a fixed random permutation of the ids (the "lowbias32" integer mixer of
// C. Wellons, a bijection of 32-bit words).  Hooking the root of larger priority under the
// other gives trees of expected logarithmic depth whatever order the edges arrive in, where
// hooking by id lets a subtree be re-rooted again and again.
__device__ __forceinline__ uint32_t link_prio(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Union with randomized linking; the root is not a canonical label (labels are computed
// afterwards as a per-component minimum).
__device__ __forceinline__ void unite_rand(uint32_t* P, uint32_t a, uint32_t b) {
    for (;;) {
        a = find_root(P, a);
        b = find_root(P, b);
        if (a == b) return;
        if (link_prio(b) < link_prio(a)) { uint32_t t = a; a = b; b = t; }
        const uint32_t old = atomicCAS(P + b, b, a);   // hook b under a
        if (old == b) return;
        b = old;
    }
}

// Union with smallest-id hooking: the root of every tree is its smallest id.
__device__ __forceinline__ void unite_min(uint32_t* P, uint32_t a, uint32_t b) {
    for (;;) {
        a = find_root(P, a);
        b = find_root(P, b);
        if (a == b) return;
        if (b < a) { uint32_t t = a; a = b; b = t; }
        const uint32_t old = atomicCAS(P + b, b, a);
        if (old == b) return;
        b = old;
    }
}

// Full compression once no union runs any more: walk to the (final) root without writing,
// then store that root along the path.  Only the root is ever written, so a concurrent
// compression of an overlapping path cannot leave an intermediate ancestor behind.
__device__ __forceinline__ uint32_t compress_to_root(uint32_t* P, uint32_t v) {
    uint32_t root = v;
    for (uint32_t p = __ldca(P + root); p != root; p = __ldca(P + root)) root = p;
    for (uint32_t x = v; x != root;) {
        const uint32_t nx = __ldca(P + x);
        if (nx != root) __stcg(P + x, root);
        x = nx;
    }
    return root;
}

}  // namespace imk
