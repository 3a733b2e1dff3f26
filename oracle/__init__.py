"""CPU oracle for sketch-based influence maximisation (PaC-IM) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
leg may import this package.  It wraps ``im_oracle.c`` (plain C, integer arithmetic,
OpenMP only across independent sketches) through ctypes and shares no code with the GPU
library.  Each function names the passage of the paper it follows; the C source has the
details.

Parity status: every function here is pinned by ``tests/test_oracle.py`` (brute-force
live-edge worlds, closed forms, library routines and invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "im_oracle.c"
_LIB = _HERE / "liboracle.so"
_lib = None

MODE_HASH = 0     # Alg. 3 Sample(e, r): hash rule, one probability p for every edge
MODE_WORLDS = 1   # sketch r = the live-edge world whose live set is the bit set of r
MODE_EDGE = 2     # hash rule with each edge's own probability (Graph.set_probs / set_wic)


def build(force: bool = False) -> Path:
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               str(_SRC), "-o", str(tmp), "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


U32P = ctypes.POINTER(ctypes.c_uint32)
U64P = ctypes.POINTER(ctypes.c_uint64)
U8P = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(str(_LIB))
    c = ctypes
    lib.or_mix.argtypes = [c.c_uint64]; lib.or_mix.restype = c.c_uint64
    lib.or_edge_key.argtypes = [c.c_uint64, c.c_uint64]; lib.or_edge_key.restype = c.c_uint64
    lib.or_edge_hash.argtypes = [c.c_uint64, c.c_uint64, c.c_uint32]
    lib.or_edge_hash.restype = c.c_uint64
    lib.or_threshold.argtypes = [c.c_double, U64P, c.POINTER(c.c_int)]
    lib.or_graph_new.argtypes = [c.c_uint32, c.c_uint64, U32P, U32P]
    lib.or_graph_new.restype = c.c_void_p
    lib.or_graph_free.argtypes = [c.c_void_p]
    lib.or_graph_set_probs.argtypes = [c.c_void_p, c.POINTER(c.c_double)]
    lib.or_graph_set_wic.argtypes = [c.c_void_p, c.POINTER(c.c_double)]
    lib.or_labels.argtypes = [c.c_void_p, c.c_int, c.c_uint64, c.c_double, c.c_uint32,
                              c.c_uint32, U32P, c.c_int]
    lib.or_gains.argtypes = [c.c_uint32, c.c_uint32, U32P, U64P]
    lib.or_num_centers.argtypes = [c.c_uint32, c.c_double]; lib.or_num_centers.restype = c.c_uint32
    lib.or_center_key.argtypes = [c.c_uint64, c.c_uint32]; lib.or_center_key.restype = c.c_uint64
    lib.or_centers.argtypes = [c.c_uint32, c.c_uint64, c.c_double, U32P, U32P]
    lib.or_compact.argtypes = [c.c_uint32, c.c_uint32, U32P, U32P, c.c_uint32, U32P, U32P]
    lib.or_greedy.argtypes = [c.c_uint32, c.c_uint32, U32P, c.c_uint32, c.c_int, U32P, U64P]
    lib.or_celf.argtypes = [c.c_uint32, c.c_uint32, U32P, c.c_uint32, U32P, U64P, U64P]
    lib.or_spread.argtypes = [c.c_uint32, c.c_uint32, U32P, U32P, c.c_uint32, U64P]
    lib.or_compact_greedy.argtypes = [c.c_void_p, c.c_int, c.c_uint64, c.c_double, c.c_uint32,
                                      U32P, c.c_uint32, U32P, U32P, c.c_uint32, U32P, U64P]
    lib.or_compact_marginal.argtypes = [c.c_void_p, c.c_int, c.c_uint64, c.c_double, c.c_uint32,
                                        U32P, U32P, U32P, U8P, c.c_uint32, U64P]
    lib.or_max_threads.restype = c.c_int
    for name in ("or_labels", "or_gains", "or_centers", "or_compact", "or_greedy", "or_celf",
                 "or_spread", "or_compact_greedy", "or_compact_marginal"):
        getattr(lib, name).restype = c.c_int
    _lib = lib
    return lib


def _p32(a):
    return a.ctypes.data_as(U32P)


def _p64(a):
    return a.ctypes.data_as(U64P)


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle.{what} failed with code {rc}")


def max_threads() -> int:
    return int(_load().or_max_threads())


# ---- hash and threshold (Sec. 2 fusion sampling, Alg. 3 Sample) -------------
def mix(x: int) -> int:
    return int(_load().or_mix(x & (2**64 - 1)))


def edge_hash(seed: int, e: int, r: int) -> int:
    return int(_load().or_edge_hash(seed, e, r))


def threshold(p: float):
    T = ctypes.c_uint64(0)
    a = ctypes.c_int(0)
    _load().or_threshold(p, ctypes.byref(T), ctypes.byref(a))
    return int(T.value), bool(a.value)


def center_key(seed: int, v: int) -> int:
    return int(_load().or_center_key(seed, v))


class Graph:
    """CSR view of a canonical undirected edge list, owned by the C oracle."""

    def __init__(self, n: int, u: np.ndarray, v: np.ndarray):
        self.n = int(n)
        self.u = np.ascontiguousarray(u, dtype=np.uint32)
        self.v = np.ascontiguousarray(v, dtype=np.uint32)
        self.m = int(self.u.shape[0])
        self._h = _load().or_graph_new(self.n, self.m, _p32(self.u), _p32(self.v))
        if not self._h:
            raise ValueError("oracle: invalid edge list (endpoint >= n or self-loop)")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_graph_free(self._h)
            self._h = None

    # per-edge IC probabilities (Sec. 2: the IC model gives every edge its own p_e)
    def set_probs(self, p: np.ndarray) -> None:
        """p[e] for every edge of the input list; used by mode=MODE_EDGE."""
        pa = np.ascontiguousarray(p, np.float64)
        if pa.shape != (self.m,):
            raise ValueError("one probability per edge")
        _ok(_load().or_graph_set_probs(self._h, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
            "set_probs")

    def set_wic(self) -> np.ndarray:
        """Weighted cascade p_e = 2 / (d_u + d_v); returns the probabilities."""
        out = np.empty(self.m, np.float64)
        _ok(_load().or_graph_set_wic(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
            "set_wic")
        return out

    # per-sketch connected components (Sec. 3 "Sketch Construction")
    def labels(self, seed: int, p: float, R: int, r0: int = 0, mode: int = MODE_HASH,
               threads: int | None = None) -> np.ndarray:
        L = np.empty((R, self.n), np.uint32)
        th = threads if threads else max_threads()
        _ok(_load().or_labels(self._h, mode, seed, p, r0, R, _p32(L), th), "labels")
        return L

    def compact_greedy(self, seed, p, R, centers, label, size, k, mode=MODE_HASH):
        seeds = np.empty(k, np.uint32)
        gains = np.empty(k, np.uint64)
        c = np.ascontiguousarray(centers, np.uint32)
        lab = np.ascontiguousarray(label, np.uint32)
        sz = np.ascontiguousarray(size, np.uint32)
        _ok(_load().or_compact_greedy(self._h, mode, seed, p, R, _p32(c), len(c), _p32(lab),
                                      _p32(sz), k, _p32(seeds), _p64(gains)), "compact_greedy")
        return seeds, gains

    def compact_marginal(self, seed, p, R, cidx, label, size, in_s, v, mode=MODE_HASH) -> int:
        out = ctypes.c_uint64(0)
        ci = np.ascontiguousarray(cidx, np.uint32)
        lab = np.ascontiguousarray(label, np.uint32)
        sz = np.ascontiguousarray(size, np.uint32)
        s = np.ascontiguousarray(in_s, np.uint8)
        _ok(_load().or_compact_marginal(self._h, mode, seed, p, R, _p32(ci), _p32(lab), _p32(sz),
                                        s.ctypes.data_as(U8P), v, ctypes.byref(out)),
            "compact_marginal")
        return int(out.value)


def gains(L: np.ndarray) -> np.ndarray:
    """Initial scores: gain[v] = sum_r |C_r(v)| (memoised components, Sec. 2)."""
    R, n = L.shape
    g = np.empty(n, np.uint64)
    _ok(_load().or_gains(n, R, _p32(np.ascontiguousarray(L)), _p64(g)), "gains")
    return g


def num_centers(n: int, alpha: float) -> int:
    return int(_load().or_num_centers(n, alpha))


def centers(n: int, seed: int, alpha: float) -> np.ndarray:
    """Centers (Sec. 3): ceil(alpha n) vertices, sorted by vertex id (= center index)."""
    out = np.empty(max(n, 1), np.uint32)
    rho = ctypes.c_uint32(0)
    _ok(_load().or_centers(n, seed, alpha, _p32(out), ctypes.byref(rho)), "centers")
    return out[: rho.value].copy()


def compact(L: np.ndarray, ctr: np.ndarray):
    """Compact sketches (Alg. 3): label, size as [rho, R] (center-major) arrays."""
    R, n = L.shape
    rho = len(ctr)
    lab = np.empty((rho, R), np.uint32)
    sz = np.empty((rho, R), np.uint32)
    c = np.ascontiguousarray(ctr, np.uint32)
    _ok(_load().or_compact(n, R, _p32(np.ascontiguousarray(L)), _p32(c), rho, _p32(lab), _p32(sz)),
        "compact")
    return lab, sz


def greedy(L: np.ndarray, k: int, variant: int = 1):
    """Plain greedy, ties to the smallest id (variant 0 recompute, 1 exact decrement)."""
    R, n = L.shape
    seeds = np.empty(k, np.uint32)
    g = np.empty(k, np.uint64)
    _ok(_load().or_greedy(n, R, _p32(np.ascontiguousarray(L)), k, variant, _p32(seeds), _p64(g)),
        "greedy")
    return seeds, g


def celf(L: np.ndarray, k: int):
    """Sequential CELF (Alg. 2): seeds, gains and evaluations per round."""
    R, n = L.shape
    seeds = np.empty(k, np.uint32)
    g = np.empty(k, np.uint64)
    ev = np.empty(k, np.uint64)
    _ok(_load().or_celf(n, R, _p32(np.ascontiguousarray(L)), k, _p32(seeds), _p64(g), _p64(ev)),
        "celf")
    return seeds, g, ev


def spread(L: np.ndarray, seeds) -> int:
    """sum_r |union_{s in S} C_r(s)| (an integer; sigma(S) times R)."""
    R, n = L.shape
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint32))
    out = ctypes.c_uint64(0)
    _ok(_load().or_spread(n, R, _p32(np.ascontiguousarray(L)), _p32(s), len(s), ctypes.byref(out)),
        "spread")
    return int(out.value)


def cidx_of(n: int, ctr: np.ndarray) -> np.ndarray:
    ci = np.full(n, 0xFFFFFFFF, np.uint32)
    ci[np.asarray(ctr, dtype=np.int64)] = np.arange(len(ctr), dtype=np.uint32)
    return ci


def solve(n, u, v, seed, p, R, alpha, k, threads=None):
    """The whole path on the CPU: labels, gains, compact sketches, greedy seeds, spread."""
    G = Graph(n, u, v)
    L = G.labels(seed, p, R, threads=threads)
    g0 = gains(L)
    ctr = centers(n, seed, alpha)
    lab, sz = compact(L, ctr)
    seeds, sg = greedy(L, k, variant=1)
    sp = spread(L, seeds)
    return dict(labels=L, gains=g0, centers=ctr, label=lab, size=sz, seeds=seeds,
                seed_gains=sg, spread=sp)
