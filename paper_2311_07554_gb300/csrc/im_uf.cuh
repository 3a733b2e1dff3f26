// im_uf.cuh -- union-find primitives shared by the sketch kernels (internal).
//
// Parent ids only ever decrease and a vertex that stops being a root never becomes one again,
// so a stale parent read from L1 is a former parent in the same set: climbing it is correct,
// and a stale "is a root" answer is caught by the atomicCAS that hooks it.  Climbs therefore
// read through L1 (__ldca): every climb in a giant component ends at the same root entry,
// which would otherwise be one hot L2 sector for the whole GPU.
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

// Rem's union with splicing (Patwary, Blair, Manne, "Experiments on union-find algorithms for
// the disjoint-set data structure", 2010), in the concurrent form with compare-and-swap used
// by ConnectIt (Dhulipala, Hong, Shun, 2020).  Invariant: a parent has a smaller id than its
// child, so roots are component minima.  Both endpoints climb in one loop: each step moves
// the side whose parent is larger, either hooking it (a root) under the other side's parent
// or splicing it there (P[rx] := py) and continuing from its old parent.  The two parent
// loads of a step are independent, and the climb ends where the paths meet, not at the root.
// Every write joins the two sets being united, and each step lowers rx, so stale (L1) reads
// cost extra steps but neither correctness nor termination.
__device__ __forceinline__ void unite_rem(uint32_t* P, uint32_t x, uint32_t y) {
    uint32_t rx = x, ry = y;
    uint32_t px = __ldca(P + rx), py = __ldca(P + ry);
    while (px != py) {
        if (px < py) {
            uint32_t t = rx; rx = ry; ry = t;
            t = px; px = py; py = t;
        }
        // now py < px <= rx
        if (rx == px) {
            const uint32_t old = atomicCAS(P + rx, rx, py);   // hook the root rx under py
            if (old == rx) return;
            px = old;                                         // rx got a parent meanwhile
            continue;
        }
        atomicCAS(P + rx, px, py);                            // splice
        rx = px;
        px = __ldca(P + rx);
    }
}

// Full compression once no union runs any more: walk to the (final) root without writing,
// then store that root along the path.  Only the root is ever written, so a concurrent
// compression of an overlapping path cannot leave an intermediate ancestor behind.  A root's
// own entry may carry kRootFlag (set by the counting pass: the root has members), which the
// walk ignores.
__device__ __forceinline__ uint32_t compress_to_root(uint32_t* P, uint32_t v) {
    uint32_t root = v;
    for (uint32_t p = __ldca(P + root) & kIdMask; p != root; p = __ldca(P + root) & kIdMask) root = p;
    for (uint32_t x = v; x != root;) {
        const uint32_t nx = __ldca(P + x) & kIdMask;
        if (nx != root) __stcg(P + x, root);
        x = nx;
    }
    return root;
}

}  // namespace imk
