"""Seeded synthetic graphs shared by the CPU oracle and the GPU library.

Every generator returns ``(n, u, v)`` with ``u, v`` uint32 numpy arrays of equal length m:
distinct undirected edges, ``u[e] < v[e]``, sorted by ``(u, v)`` so that the edge id ``e``
is the rank of the pair.  The edge set is the first m distinct pairs of a splitmix64
counter stream (see ``graphgen.c``).  This module synthesises inputs only; it contains
none of the influence-maximisation arithmetic.

The workload presets follow the paper's experimental setup (Sec. 5): scale-free graphs
with a constant IC probability, R = 256 sketches.  The paper's own datasets (SNAP,
WebGraph, road and k-NN graphs) are replaced by Erdos-Renyi, Chung-Lu power-law and
R-MAT graphs of matching shape.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "graphgen.c"
_LIB = _HERE / "libgraphgen.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile libgraphgen.so next to its source (gcc, OpenMP)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.check_call([
            "gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
            str(_SRC), "-o", str(tmp), "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        P = ctypes.POINTER(ctypes.c_uint32)
        lib.gg_erdos_renyi.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, P, P]
        lib.gg_erdos_renyi.restype = ctypes.c_int64
        lib.gg_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, P, P]
        lib.gg_chung_lu.restype = ctypes.c_int64
        lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, P, P]
        lib.gg_rmat.restype = ctypes.c_int64
        lib.gg_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _cache_dir():
    d = os.environ.get("IM_GRAPH_CACHE")
    return Path(d) if d else None


def _cached(tag: str, fn):
    d = _cache_dir()
    if d is None:
        return fn()
    d.mkdir(parents=True, exist_ok=True)
    h = hashlib.sha1(tag.encode()).hexdigest()[:16]
    f = d / f"g_{h}.npz"
    if f.exists():
        z = np.load(f)
        return int(z["n"]), z["u"], z["v"]
    n, u, v = fn()
    tmp = d / f"g_{h}.{os.getpid()}.tmp.npz"
    np.savez(tmp, n=np.int64(n), u=u, v=v)
    os.replace(tmp, f)
    return n, u, v


def _check(ret: int, m: int, what: str):
    if ret != m:
        raise RuntimeError(f"graphgen.{what} failed (code {ret})")


def erdos_renyi(n: int, m: int, seed: int):
    """G(n, m): uniform endpoints, self-loops and duplicates rejected."""
    def gen():
        u = np.empty(m, np.uint32)
        v = np.empty(m, np.uint32)
        _check(_load().gg_erdos_renyi(n, m, seed, _ptr(u), _ptr(v)), m, "erdos_renyi")
        return n, u, v
    return _cached(f"er:{n}:{m}:{seed}", gen)


def chung_lu(n: int, m: int, exponent: float, max_deg: float, seed: int):
    """Chung-Lu expected-degree graph with power-law weights (i+1)^(-1/(exponent-1))."""
    def gen():
        u = np.empty(m, np.uint32)
        v = np.empty(m, np.uint32)
        _check(_load().gg_chung_lu(n, m, exponent, max_deg, seed, _ptr(u), _ptr(v)), m, "chung_lu")
        return n, u, v
    return _cached(f"cl:{n}:{m}:{exponent!r}:{max_deg!r}:{seed}", gen)


def rmat(scale: int, m: int, a: float, b: float, c: float, seed: int):
    """R-MAT (no noise), symmetrised and de-duplicated until m distinct edges."""
    def gen():
        u = np.empty(m, np.uint32)
        v = np.empty(m, np.uint32)
        _check(_load().gg_rmat(scale, m, a, b, c, seed, _ptr(u), _ptr(v)), m, "rmat")
        return 1 << scale, u, v
    return _cached(f"rmat:{scale}:{m}:{a!r}:{b!r}:{c!r}:{seed}", gen)


# ---- workload presets -------------------------------------------------------
# Each entry: graph recipe + method parameters (p, R, alpha, k, hash seed).
WORKLOADS = {
    "er_n2000_m10000": dict(
        graph=lambda: erdos_renyi(2000, 10_000, 1), p=0.05, R=256, alpha=1.0, k=10, seed=42),
    "chunglu_n1M_m10M": dict(
        graph=lambda: chung_lu(1_000_000, 10_000_000, 2.1, 50_000.0, 2), p=0.02, R=256,
        alpha=0.1, k=100, seed=42),
    "rmat_s24_m256M": dict(
        graph=lambda: rmat(24, 1 << 28, 0.57, 0.19, 0.19, 3), p=0.01, R=256, alpha=0.05,
        k=200, seed=42),
    # the same recipe at scale 21 (n = 2^21, 2^25 edges): small enough for the profiler's
    # multi-pass captures, still larger than L2 per sketch batch
    "rmat_s21_m32M": dict(
        graph=lambda: rmat(21, 1 << 25, 0.57, 0.19, 0.19, 3), p=0.01, R=256, alpha=0.05,
        k=200, seed=42),
}


def c4_instances(count: int = 64, first_seed: int = 1000, n_range=(1e4, 2e6)):
    """The batched workload: `count` independent Chung-Lu instances.  Instance i takes the seed
    first_seed + i for its parameter draws and its graph: n log-uniform in n_range, average
    degree U(4, 32) (m = n deg / 2), exponent 2.1, maximum expected degree min(50,000, n/4),
    p from {.01, .02, .05, .1}, R from {64, 128, 256}, k from {10, 50, 100}; every vertex a
    center (alpha = 1); the hash seed is the instance seed."""
    out = []
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    for i in range(count):
        s = first_seed + i
        rng = np.random.default_rng(s)
        n = int(round(float(np.exp(rng.uniform(lo, hi)))))
        deg = float(rng.uniform(4.0, 32.0))
        m = int(round(n * deg / 2))
        p = float(rng.choice([0.01, 0.02, 0.05, 0.1]))
        R = int(rng.choice([64, 128, 256]))
        k = int(rng.choice([10, 50, 100]))
        n_, u, v = chung_lu(n, m, 2.1, min(50_000.0, n / 4), s)
        out.append(dict(n=n_, u=u, v=v, p=p, R=R, k=min(k, n_), seed=s, alpha=1.0))
    return out


def c5_requests(models: int, rate: float, duration: float, seed: int = 2311):
    """The serving workload's request trace: Poisson arrivals at `rate` per second for
    `duration` seconds, each asking a uniform model for k ~ U{5..200} seeds.  Returns
    (model, k, arrival_ns) tuples in arrival order."""
    rng = np.random.default_rng(seed)
    nreq = int(rate * duration)
    arrivals = np.cumsum(rng.exponential(1e9 / rate, nreq))
    return [(int(rng.integers(0, models)), int(rng.integers(5, 201)), int(t)) for t in arrivals]


def workload(name: str):
    """Return (n, u, v, params) for a named workload."""
    w = WORKLOADS[name]
    n, u, v = w["graph"]()
    params = {k: w[k] for k in ("p", "R", "alpha", "k", "seed")}
    return n, u, v, params


def num_threads() -> int:
    return int(_load().gg_num_threads())
