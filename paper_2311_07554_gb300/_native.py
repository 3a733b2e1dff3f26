"""ctypes binding of ``libim_gb300.so`` (the C ABI in include/im_gb300.h).

Argument marshalling only: every step of the path runs in the library's CUDA kernels.
There is no CPU fallback; a missing or unloadable library raises at first use.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "libim_gb300.so"

IM_OK, IM_EINVAL, IM_ENOMEM, IM_ECUDA, IM_ESTATE, IM_ETIMEOUT, IM_EDEVICE = 0, -1, -2, -3, -4, -5, -6
IM_PTR_HOST, IM_PTR_DEVICE = 0, 1
ERROR_NAMES = {0: "IM_OK", -1: "IM_EINVAL", -2: "IM_ENOMEM", -3: "IM_ECUDA", -4: "IM_ESTATE",
               -5: "IM_ETIMEOUT", -6: "IM_EDEVICE"}

_lib = None


class IMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class im_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("R", ctypes.c_uint32), ("rho", ctypes.c_uint32),
                ("rounds", ctypes.c_uint32), ("m", ctypes.c_uint64),
                ("evaluations", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("bfs_fallbacks", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("sketch_batch", ctypes.c_uint32), ("hop1_arcs", ctypes.c_uint64),
                ("hop2_searches", ctypes.c_uint64), ("hop2_chunks", ctypes.c_uint64),
                ("refresh_batches", ctypes.c_uint64), ("live_pairs", ctypes.c_uint64),
                ("build_live_pairs", ctypes.c_uint64), ("spec_batches", ctypes.c_uint64),
                ("hubs", ctypes.c_uint64), ("union_path", ctypes.c_uint32)]


class im_instance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("m", ctypes.c_uint64),
                ("u", ctypes.POINTER(ctypes.c_uint32)), ("v", ctypes.POINTER(ctypes.c_uint32)),
                ("R", ctypes.c_uint32), ("k", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("p", ctypes.c_double), ("alpha", ctypes.c_double),
                ("seeds_out", ctypes.POINTER(ctypes.c_uint32)), ("gains_out", ctypes.POINTER(ctypes.c_uint64)),
                ("spread_out", ctypes.POINTER(ctypes.c_uint64)), ("status", ctypes.c_int)]


class im_request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_uint32), ("k", ctypes.c_uint32), ("arrival_ns", ctypes.c_uint64),
                ("seeds_out", ctypes.POINTER(ctypes.c_uint32)), ("gains_out", ctypes.POINTER(ctypes.c_uint64)),
                ("spread_out", ctypes.POINTER(ctypes.c_uint64)), ("submit_ns", ctypes.c_uint64),
                ("done_ns", ctypes.c_uint64), ("status", ctypes.c_int)]


class im_model_stats(ctypes.Structure):
    _fields_ = [("footprint", ctypes.c_uint64), ("builds", ctypes.c_uint32), ("evictions", ctypes.c_uint32),
                ("resident", ctypes.c_uint32), ("known_seeds", ctypes.c_uint32), ("budget", ctypes.c_uint64),
                ("used", ctypes.c_uint64)]


class im_batch_schedule(ctypes.Structure):
    _fields_ = [("branches", ctypes.c_uint32), ("classes", ctypes.c_uint32), ("class_pairs", ctypes.c_uint64 * 4),
                ("sketch_batch", ctypes.c_uint32 * 4), ("lanes", ctypes.c_uint32 * 4),
                ("union_path", ctypes.c_uint32 * 4), ("run_ms", ctypes.c_double)]


class im_tuning(ctypes.Structure):
    _fields_ = [("sketch_batch", ctypes.c_uint32), ("lanes", ctypes.c_uint32), ("hub_cap", ctypes.c_uint32),
                ("tried", ctypes.c_uint32), ("build_ms", ctypes.c_double), ("select_ms", ctypes.c_double),
                ("default_build_ms", ctypes.c_double), ("default_select_ms", ctypes.c_double)]


def lib():
    """Load the library (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                          "(or python -m paper_2311_07554_gb300.build)")
    L = ctypes.CDLL(str(LIB_PATH))
    c = ctypes
    vp, u32, u64, i32, dbl = c.c_void_p, c.c_uint32, c.c_uint64, c.c_int, c.c_double
    sig = {
        "im_create": ([c.POINTER(vp), u32, u64, vp, vp, i32, vp], i32),
        "im_build_sketches": ([vp, u32, u64, dbl, dbl], i32),
        "im_load_graph": ([vp, u32, u64, vp, vp, i32], i32),
        "im_set_edge_probs": ([vp, i32, vp, i32], i32),
        "im_select_seeds": ([vp, u32, vp, vp], i32),
        "im_spread": ([vp, vp, u32, c.POINTER(u64)], i32),
        "im_reset_selection": ([vp], i32),
        "im_get_labels": ([vp, u32, vp, i32], i32),
        "im_get_gains": ([vp, vp, i32], i32),
        "im_get_centers": ([vp, vp, c.POINTER(u32), i32], i32),
        "im_get_compact": ([vp, vp, vp, i32], i32),
        "im_get_stats": ([vp, c.POINTER(im_stats)], i32),
        "im_get_round_evals": ([vp, vp, u32], i32),
        "im_profile_enable": ([vp, i32], i32),
        "im_profile_reset": ([vp], i32),
        "im_profile_get": ([vp, i32, c.POINTER(dbl), c.POINTER(u64)], i32),
        "im_kernel_count": ([], i32),
        "im_kernel_name": ([i32], c.c_char_p),
        "im_set_sketch_batch": ([vp, u32], i32),
        "im_set_refresh_threshold": ([vp, u64], i32),
        "im_set_pipeline": ([vp, u32], i32),
        "im_set_union_path": ([vp, i32], i32),
        "im_debug_fail_alloc": ([c.c_int64], i32),
        "im_debug_record_cap": ([c.c_int64], i32),
        "im_mailbox_create": ([vp, u32, u32, c.POINTER(vp)], i32),
        "im_server_set_budget": ([vp, u64], i32),
        "im_batch_create": ([vp, u32, vp, c.POINTER(vp)], i32),
        "im_batch_run": ([vp], i32),
        "im_batch_destroy": ([vp], i32),
        "im_batch_tune": ([vp, u32, vp], i32),
        "im_server_stats": ([vp, u32, c.POINTER(im_model_stats)], i32),
        "im_footprint_estimate": ([u32, u64, u32, dbl, dbl, c.POINTER(u64)], i32),
        "im_mailbox_push": ([vp, u32], i32),
        "im_serve_launch": ([vp, u32], i32),
        "im_mailbox_wait": ([vp, u32, u32, vp, vp], i32),
        "im_mailbox_state": ([vp, c.POINTER(u32), c.POINTER(c.c_int32), c.POINTER(u32)], i32),
        "im_serve_finish": ([vp, c.POINTER(c.c_int32)], i32),
        "im_mailbox_destroy": ([vp], i32),
        "im_set_graph": ([vp, i32], i32),
        "im_hash_peak": ([u32, c.POINTER(dbl)], i32),
        "im_set_seed_speculation": ([vp, u32], i32),
        "im_set_hubs": ([vp, u32, u32], i32),
        "im_autotune": ([vp, u32, u64, dbl, dbl, u32, u32, c.POINTER(im_tuning)], i32),
        "im_run_batch": ([c.POINTER(im_instance), u32, u32], i32),
        "im_server_create": ([c.POINTER(vp)], i32),
        "im_server_add_model": ([vp, u32, u64, vp, vp, u32, u64, dbl, dbl, c.POINTER(u32), c.POINTER(u64)], i32),
        "im_server_replay": ([vp, c.POINTER(im_request), u32], i32),
        "im_server_destroy": ([vp], i32),
        "im_mc_spread": ([vp, ctypes.POINTER(ctypes.c_uint32), u32, u32, u64, ctypes.POINTER(ctypes.c_uint64)], i32),
        "im_stream": ([vp], vp),
        "im_sketch_static": ([u32, u64, vp, vp, u64, dbl, u32, vp, vp, vp], i32),
        "im_last_error": ([vp], c.c_char_p),
        "im_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(ctx, rc: int):
    if rc != IM_OK:
        msg = lib().im_last_error(ctx)
        raise IMError(rc, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, ptr_kind) of a numpy array or a torch tensor (CUDA -> device pointer)."""
    if a is None:
        return None, IM_PTR_HOST
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), (IM_PTR_DEVICE if a.is_cuda else IM_PTR_HOST)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), IM_PTR_HOST


# ---- the C calls, same names ------------------------------------------------------------
def im_create(n: int, u, v, stream=None):
    """Returns an opaque context handle (int).  u, v: uint32 numpy arrays or CUDA tensors."""
    pu, ku = _ptr(u)
    pv, kv = _ptr(v)
    if ku != kv:
        raise ValueError("u and v must both be host or both be device buffers")
    m = int(len(u))
    if len(v) != m:
        raise ValueError("u and v differ in length")
    h = ctypes.c_void_p()
    rc = lib().im_create(ctypes.byref(h), n, m, pu, pv, ku, ctypes.c_void_p(stream) if stream else None)
    if rc != IM_OK:
        msg = lib().im_last_error(None)
        raise IMError(rc, msg.decode() if msg else "")
    return h.value


def im_load_graph(ctx, n: int, u, v):
    """Replace the context's graph (same argument conventions as im_create)."""
    pu, ku = _ptr(u)
    pv, kv = _ptr(v)
    if ku != kv:
        raise ValueError("u and v must both be host or both be device buffers")
    m = int(len(u))
    if len(v) != m:
        raise ValueError("u and v differ in length")
    _check(ctx, lib().im_load_graph(ctx, n, m, pu, pv, ku))


IM_PROBS_UNIFORM, IM_PROBS_ARRAY, IM_PROBS_WIC = 0, 1, 2


def im_set_edge_probs(ctx, model: int, p=None):
    """model IM_PROBS_UNIFORM / IM_PROBS_WIC (p ignored) or IM_PROBS_ARRAY with p: one float64
    per edge (numpy array or CUDA tensor)."""
    pp, kind = (None, IM_PTR_HOST)
    if model == IM_PROBS_ARRAY:
        if hasattr(p, "dtype") and str(p.dtype) not in ("float64", "torch.float64"):
            raise ValueError("probabilities must be float64")
        pp, kind = _ptr(p)
    _check(ctx, lib().im_set_edge_probs(ctx, model, pp, kind))


def im_build_sketches(ctx, R: int, seed: int, p: float, alpha: float):
    _check(ctx, lib().im_build_sketches(ctx, R, seed, p, alpha))


def im_select_seeds(ctx, k: int):
    seeds = np.empty(k, np.uint32)
    gains = np.empty(k, np.uint64)
    _check(ctx, lib().im_select_seeds(ctx, k, seeds.ctypes.data, gains.ctypes.data))
    return seeds, gains


def im_spread(ctx, seeds) -> int:
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint32))
    out = ctypes.c_uint64(0)
    _check(ctx, lib().im_spread(ctx, s.ctypes.data if len(s) else None, len(s), ctypes.byref(out)))
    return int(out.value)


def im_reset_selection(ctx):
    _check(ctx, lib().im_reset_selection(ctx))


def im_get_labels(ctx, r: int, out=None, n: int | None = None):
    if out is None:
        out = np.empty(n if n is not None else im_get_stats(ctx)["n"], np.uint32)
    p, kind = _ptr(out)
    _check(ctx, lib().im_get_labels(ctx, r, p, kind))
    return out


def im_get_gains(ctx, out=None):
    if out is None:
        out = np.empty(im_get_stats(ctx)["n"], np.uint64)
    p, kind = _ptr(out)
    _check(ctx, lib().im_get_gains(ctx, p, kind))
    return out


def im_get_centers(ctx, out=None):
    rho = ctypes.c_uint32(0)
    _check(ctx, lib().im_get_centers(ctx, None, ctypes.byref(rho), IM_PTR_HOST))
    if out is None:
        out = np.empty(rho.value, np.uint32)
    p, kind = _ptr(out)
    _check(ctx, lib().im_get_centers(ctx, p, ctypes.byref(rho), kind))
    return out


def im_get_compact(ctx):
    st = im_get_stats(ctx)
    lab = np.empty((st["rho"], st["R"]), np.uint32)
    sz = np.empty((st["rho"], st["R"]), np.uint32)
    _check(ctx, lib().im_get_compact(ctx, lab.ctypes.data, sz.ctypes.data, IM_PTR_HOST))
    return lab, sz


def im_get_stats(ctx) -> dict:
    s = im_stats()
    _check(ctx, lib().im_get_stats(ctx, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in im_stats._fields_}


def im_get_round_evals(ctx, count: int):
    out = np.zeros(count, np.uint64)
    _check(ctx, lib().im_get_round_evals(ctx, out.ctypes.data, count))
    return out


def im_profile_enable(ctx, on: bool = True):
    _check(ctx, lib().im_profile_enable(ctx, 1 if on else 0))


def im_profile_reset(ctx):
    _check(ctx, lib().im_profile_reset(ctx))


def im_profile_get(ctx) -> dict:
    """{kernel name: (total device ms, launches)} for kernels launched since the reset."""
    res = {}
    for kid in range(lib().im_kernel_count()):
        ms = ctypes.c_double(0)
        nl = ctypes.c_uint64(0)
        _check(ctx, lib().im_profile_get(ctx, kid, ctypes.byref(ms), ctypes.byref(nl)))
        if nl.value:
            res[lib().im_kernel_name(kid).decode()] = (ms.value, int(nl.value))
    return res


def im_set_sketch_batch(ctx, batch: int):
    _check(ctx, lib().im_set_sketch_batch(ctx, batch))


def im_set_refresh_threshold(ctx, min_batch: int):
    _check(ctx, lib().im_set_refresh_threshold(ctx, min_batch))


def im_set_pipeline(ctx, lanes: int):
    _check(ctx, lib().im_set_pipeline(ctx, lanes))


def im_debug_fail_alloc(after: int):
    """Test hook: the device allocation after `after` more successful ones fails (IM_ENOMEM);
    negative disarms."""
    lib().im_debug_fail_alloc(int(after))


def im_debug_record_cap(records: int):
    """Test hook: cap the live-pair records the sketch kernels use (negative restores)."""
    lib().im_debug_record_cap(int(records))


IM_UNION_FUSED = 0
IM_UNION_RECORDS = 1
IM_UNION_BUCKETS = 2
IM_UNION_AUTO = 3


def im_set_union_path(ctx, path: int):
    """IM_UNION_FUSED: hashing and unions in one kernel; IM_UNION_RECORDS: live-pair records
    united by a second kernel; IM_UNION_BUCKETS: records grouped by sketch, united sketch after
    sketch; IM_UNION_AUTO (default): buckets when a batch's parent arrays exceed 256 MiB."""
    _check(ctx, lib().im_set_union_path(ctx, path))


def im_set_graph(ctx, on: bool):
    _check(ctx, lib().im_set_graph(ctx, 1 if on else 0))


def im_set_seed_speculation(ctx, candidates: int):
    _check(ctx, lib().im_set_seed_speculation(ctx, candidates))


def im_mc_spread(ctx, seeds, sims: int, mc_seed: int) -> int:
    """Sum over `sims` Monte-Carlo simulations (live-edge worlds of hash seed `mc_seed`) of the
    number of vertices reachable from the seeds; the estimate of sigma(S) is the result / sims."""
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint32))
    out = ctypes.c_uint64(0)
    _check(ctx, lib().im_mc_spread(ctx, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), len(s), sims, mc_seed,
                                   ctypes.byref(out)))
    return int(out.value)


def im_run_batch(instances, workers: int = 8):
    """Run independent instances concurrently (one context and stream per worker thread).

    `instances`: dicts with n, u, v (host uint32 arrays), R, k, seed, p, alpha.  Returns a list of
    (seeds, gains, spread) in input order; raises IMError with the first failing status."""
    keep = []
    arr = (im_instance * len(instances))()
    outs = []
    for i, d in enumerate(instances):
        u = np.ascontiguousarray(np.asarray(d["u"], dtype=np.uint32))
        v = np.ascontiguousarray(np.asarray(d["v"], dtype=np.uint32))
        k = int(d["k"])
        sd = np.zeros(k, np.uint32)
        gn = np.zeros(k, np.uint64)
        sp = np.zeros(1, np.uint64)
        keep += [u, v]
        outs.append((sd, gn, sp))
        P32, P64 = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
        arr[i] = im_instance(int(d["n"]), len(u), u.ctypes.data_as(P32), v.ctypes.data_as(P32), int(d["R"]), k,
                             int(d["seed"]), float(d["p"]), float(d["alpha"]), sd.ctypes.data_as(P32),
                             gn.ctypes.data_as(P64), sp.ctypes.data_as(P64), 0)
    rc = lib().im_run_batch(arr, len(instances), workers)
    if rc != IM_OK:
        bad = next(i for i in range(len(instances)) if arr[i].status != IM_OK)
        raise IMError(rc, f"instance {bad} failed with status {arr[bad].status}")
    return [(sd, gn, int(sp[0])) for sd, gn, sp in outs]


def _instances(instances):
    """ctypes array of im_instance for dicts with n, u, v, R, k, seed, p, alpha, with output arrays;
    returns (array, outputs, arrays to keep alive)."""
    keep = []
    arr = (im_instance * len(instances))()
    outs = []
    P32, P64 = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
    for i, d in enumerate(instances):
        u = d["u"] if isinstance(d["u"], np.ndarray) and d["u"].dtype == np.uint32 and d["u"].flags["C_CONTIGUOUS"] \
            else np.ascontiguousarray(np.asarray(d["u"], dtype=np.uint32))
        v = d["v"] if isinstance(d["v"], np.ndarray) and d["v"].dtype == np.uint32 and d["v"].flags["C_CONTIGUOUS"] \
            else np.ascontiguousarray(np.asarray(d["v"], dtype=np.uint32))
        k = int(d["k"])
        sd, gn, sp = np.zeros(k, np.uint32), np.zeros(k, np.uint64), np.zeros(1, np.uint64)
        keep += [u, v]
        outs.append((sd, gn, sp))
        arr[i] = im_instance(int(d["n"]), len(u), u.ctypes.data_as(P32), v.ctypes.data_as(P32), int(d["R"]), k,
                             int(d["seed"]), float(d["p"]), float(d["alpha"]), sd.ctypes.data_as(P32),
                             gn.ctypes.data_as(P64), sp.ctypes.data_as(P64), 0)
    return arr, outs, keep


class Batch:
    """A batch of instances planned as one CUDA graph (im_batch_create); run() launches it."""

    def __init__(self, instances, schedule=None):
        self._arr, self._outs, self._keep = _instances(instances)
        self._sched = schedule
        h = ctypes.c_void_p()
        rc = lib().im_batch_create(self._arr, len(instances), ctypes.byref(schedule) if schedule is not None else None,
                                   ctypes.byref(h))
        if rc != IM_OK:
            raise IMError(rc, lib().im_last_error(None).decode())
        self.h = h

    def run(self):
        rc = lib().im_batch_run(self.h)
        if rc != IM_OK:
            bad = next(i for i in range(len(self._outs)) if self._arr[i].status != IM_OK)
            raise IMError(rc, f"instance {bad} failed with status {self._arr[bad].status}")
        return [(sd.copy(), gn.copy(), int(sp[0])) for sd, gn, sp in self._outs]

    def statuses(self):
        return [int(self._arr[i].status) for i in range(len(self._outs))]

    def close(self):
        if self.h:
            lib().im_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def im_batch_tune(instances):
    """The schedule (size-class knobs and branches) im_batch_tune picks for these instances."""
    arr, outs, keep = _instances(instances)
    sched = im_batch_schedule()
    rc = lib().im_batch_tune(arr, len(instances), ctypes.byref(sched))
    if rc != IM_OK:
        raise IMError(rc, "im_batch_tune")
    return sched


class IMServer:
    """Resident models answering requests for k seeds (im_server_*)."""

    def __init__(self):
        h = ctypes.c_void_p()
        rc = lib().im_server_create(ctypes.byref(h))
        if rc != IM_OK:
            raise IMError(rc, "im_server_create")
        self.h = h
        self._keep = []

    def add_model(self, n, u, v, R, seed, p, alpha):
        """Admit a model; returns (model id, estimated device bytes)."""
        u = np.ascontiguousarray(np.asarray(u, dtype=np.uint32))
        v = np.ascontiguousarray(np.asarray(v, dtype=np.uint32))
        mid = ctypes.c_uint32(0)
        fp = ctypes.c_uint64(0)
        rc = lib().im_server_add_model(self.h, n, len(u), u.ctypes.data, v.ctypes.data, R, seed, p, alpha,
                                       ctypes.byref(mid), ctypes.byref(fp))
        if rc != IM_OK:
            raise IMError(rc, f"im_server_add_model (estimated {fp.value} bytes)")
        return int(mid.value), int(fp.value)

    def set_budget(self, nbytes: int):
        rc = lib().im_server_set_budget(self.h, int(nbytes))
        if rc != IM_OK:
            raise IMError(rc, "im_server_set_budget")

    def stats(self, model: int) -> dict:
        out = im_model_stats()
        rc = lib().im_server_stats(self.h, model, ctypes.byref(out))
        if rc != IM_OK:
            raise IMError(rc, "im_server_stats")
        return {f: getattr(out, f) for f, _ in im_model_stats._fields_}

    def replay(self, requests):
        """requests: (model, k, arrival_ns) tuples.  Returns dicts with seeds, gains, spread,
        submit_ns, done_ns, in input order."""
        arr = (im_request * len(requests))()
        outs = []
        P32, P64 = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
        for i, (model, k, t) in enumerate(requests):
            sd = np.zeros(k, np.uint32)
            gn = np.zeros(k, np.uint64)
            sp = np.zeros(1, np.uint64)
            outs.append((sd, gn, sp))
            arr[i] = im_request(model, k, int(t), sd.ctypes.data_as(P32), gn.ctypes.data_as(P64),
                                sp.ctypes.data_as(P64), 0, 0, 0)
        rc = lib().im_server_replay(self.h, arr, len(requests))
        if rc != IM_OK:
            raise IMError(rc, "im_server_replay")
        return [dict(seeds=sd, gains=gn, spread=int(sp[0]), submit_ns=int(arr[i].submit_ns),
                     done_ns=int(arr[i].done_ns)) for i, (sd, gn, sp) in enumerate(outs)]

    def close(self):
        if self.h:
            lib().im_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


IM_HUBS_AUTO = 0xFFFFFFFF


def im_set_hubs(ctx, cap: int = IM_HUBS_AUTO, min_degree: int = 32):
    _check(ctx, lib().im_set_hubs(ctx, cap, min_degree))


def im_autotune(ctx, R: int, seed: int, p: float, alpha: float, k: int, reps: int = 1) -> dict:
    """Times every combination of sketch batch, lanes and hubs on (R, seed, p, alpha, k), sets the
    fastest and builds the sketches with it; returns the chosen knobs and their times."""
    out = im_tuning()
    _check(ctx, lib().im_autotune(ctx, R, seed, p, alpha, k, reps, ctypes.byref(out)))
    return {f: getattr(out, f) for f, _ in im_tuning._fields_}


def im_footprint_estimate(n: int, m: int, R: int, p: float, alpha: float) -> int:
    """Estimated device bytes of a context holding that graph and its sketches."""
    out = ctypes.c_uint64(0)
    rc = lib().im_footprint_estimate(n, m, R, p, alpha, ctypes.byref(out))
    if rc != IM_OK:
        raise IMError(rc, "im_footprint_estimate")
    return int(out.value)


def im_hash_peak(iters: int = 4096) -> float:
    """Pairs per second of the sampling kernel's per-pair compute on registers only."""
    out = ctypes.c_double(0)
    rc = lib().im_hash_peak(iters, ctypes.byref(out))
    if rc != IM_OK:
        raise IMError(rc, "im_hash_peak failed")
    return out.value


def im_stream(ctx) -> int:
    return int(lib().im_stream(ctx) or 0)


def im_sketch_static(n: int, d_u, d_v, seed: int, p: float, r: int, d_labels=None, d_sizes=None,
                     stream=None):
    """Labels / component sizes of sketch r without any device allocation (device buffers)."""
    for t in (d_u, d_v, d_labels, d_sizes):
        if t is not None and not getattr(t, "is_cuda", False):
            raise ValueError("im_sketch_static takes device tensors only")
    rc = lib().im_sketch_static(n, int(len(d_u)), ctypes.c_void_p(d_u.data_ptr()),
                                ctypes.c_void_p(d_v.data_ptr()), seed, p, r,
                                ctypes.c_void_p(d_labels.data_ptr()) if d_labels is not None else None,
                                ctypes.c_void_p(d_sizes.data_ptr()) if d_sizes is not None else None,
                                ctypes.c_void_p(stream) if stream else None)
    if rc != IM_OK:
        msg = lib().im_last_error(None)
        raise IMError(rc, msg.decode() if msg else "")


def im_destroy(ctx):
    if ctx:
        lib().im_destroy(ctx)


class IMContext:
    """Owning wrapper around an ``im_ctx``; methods map one-to-one onto the C calls."""

    def __init__(self, n: int, u, v, stream=None):
        self.n = int(n)
        self.h = im_create(n, u, v, stream)

    def load_graph(self, n, u, v):
        im_load_graph(self.h, n, u, v)
        self.n = int(n)
        return self

    def set_edge_probs(self, model, p=None):
        im_set_edge_probs(self.h, model, p)
        return self

    def build_sketches(self, R, seed, p, alpha):
        im_build_sketches(self.h, R, seed, p, alpha)
        return self

    def select_seeds(self, k):
        return im_select_seeds(self.h, k)

    def spread(self, seeds):
        return im_spread(self.h, seeds)

    def mc_spread(self, seeds, sims, mc_seed):
        return im_mc_spread(self.h, seeds, sims, mc_seed)

    def autotune(self, R, seed, p, alpha, k, reps=1):
        return im_autotune(self.h, R, seed, p, alpha, k, reps)

    def reset_selection(self):
        im_reset_selection(self.h)

    def labels(self, r, out=None):
        return im_get_labels(self.h, r, out, self.n)

    def gains(self, out=None):
        return im_get_gains(self.h, out)

    def centers(self):
        return im_get_centers(self.h)

    def compact(self):
        return im_get_compact(self.h)

    def stats(self):
        return im_get_stats(self.h)

    def round_evals(self):
        return im_get_round_evals(self.h, self.stats()["rounds"])

    def close(self):
        if self.h:
            im_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

class Mailbox:
    """A device-resident request loop's mailbox on a context (im_mailbox_* / im_serve_*)."""

    def __init__(self, ctx, ring: int = 64, kcap: int | None = None):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(ctx.h, lib().im_mailbox_create(ctx.h, ring, kcap if kcap else ctx.n, ctypes.byref(h)))
        self.h = h

    def push(self, k: int):
        _check(self.ctx.h, lib().im_mailbox_push(self.h, k))

    def launch(self, idle_us: int = 20000):
        _check(self.ctx.h, lib().im_serve_launch(self.h, idle_us))

    def wait(self, k: int, timeout_us: int = 30_000_000):
        seeds = np.zeros(k, np.uint32)
        gains = np.zeros(k, np.uint64)
        _check(self.ctx.h, lib().im_mailbox_wait(self.h, k, timeout_us, seeds.ctypes.data_as(ctypes.c_void_p),
                                                 gains.ctypes.data_as(ctypes.c_void_p)))
        return seeds, gains

    def state(self):
        r, st, a = ctypes.c_uint32(0), ctypes.c_int32(0), ctypes.c_uint32(0)
        _check(self.ctx.h, lib().im_mailbox_state(self.h, ctypes.byref(r), ctypes.byref(st), ctypes.byref(a)))
        return {"running": int(r.value), "status": int(st.value), "answered": int(a.value)}

    def finish(self) -> int:
        st = ctypes.c_int32(0)
        _check(self.ctx.h, lib().im_serve_finish(self.h, ctypes.byref(st)))
        return int(st.value)

    def close(self):
        """Ends a loop still serving the mailbox (im_serve_finish), then frees it."""
        if self.h:
            st = ctypes.c_int32(0)
            lib().im_serve_finish(self.h, ctypes.byref(st))
            _check(self.ctx.h, lib().im_mailbox_destroy(self.h))
            self.h = None

