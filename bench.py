"""Benchmark: sampled edge-sketch pairs/s of the whole hot path on one GB300.

One step = one pass of the whole path over the resident graph: build R sketches
(hash sampling, batched union-find, compression, component histograms, initial gains,
compact sketches), select k seeds with the device lazy greedy, and the spread of those seeds.
value = m * R (sampled edge-sketch pairs) per step / step time, summed over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rmat_s24_m256M] [--no-extras]

The default workload is the R-MAT graph of scale 24 with 2^28 edges (p = 0.01, R = 256,
alpha = 0.05, k = 200), the largest configuration of the paper's kind that one GPU holds.
The same JSON line carries, unless --no-extras, three more measurements of the same run:
"secondary" (the Chung-Lu n = 10^6, m = 10^7 workload, timed the same way), "batched" (64
independent Chung-Lu instances: one at a time against the batched engine, outputs compared)
and "serving" (Poisson requests against resident R-MAT models: queries/s, p50/p99 latency,
answers compared with the same requests run alone).

Under torchrun every rank runs an independent replica of the workload (the path needs no
exchange); rank 0 prints the JSON line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import graphgen  # noqa: E402

METRIC = "sampled edge-sketch pairs/s"
DEFAULT_WORKLOAD = "rmat_s24_m256M"
SECONDARY_WORKLOAD = "chunglu_n1M_m10M"
PROFILES = ROOT / "profiles"
SRC = ROOT / "paper_2311_07554_gb300" / "csrc"


# ------------------------------------------------------------------------------ helpers
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, dist, device):
    """Each value's maximum over the ranks (the slowest replica decides the job's time);
    unchanged without a process group."""
    if dist is None:
        return [float(x) for x in values]
    import torch
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_rank, ranks, seconds):
    """Whole-job throughput of `ranks` replicas that each processed units_per_rank in at most
    `seconds` (the max over ranks)."""
    return units_per_rank * ranks / seconds


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = Path(os.environ.get("TMPDIR", "/tmp")) / f"im_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.path.read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        try:
            self.path.unlink()
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    f = ROOT / "MEASURED_PEAKS.json"
    if f.exists():
        d = json.loads(f.read_text())
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _kernel_digest(name: str, fn: str) -> str:
    """sha1 of a kernel's own source text (its name through its closing brace) in csrc/name:
    the ncu counters of a kernel stay valid while that text is unchanged."""
    text = (SRC / name).read_text()
    i = text.find("\n" + fn + "(")
    if i < 0:
        return ""
    depth, k = 0, text.index("{", i)
    for k in range(k, len(text)):
        depth += {"{": 1, "}": -1}.get(text[k], 0)
        if depth == 0:
            break
    return hashlib.sha1(text[i + 1:k + 1].encode()).hexdigest()[:12]


def _traffic(kernel: str, units_per_launch: float, path: str = "records"):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current source.
    An entry "name@path" (the bucketed path's own sampling, union and compression kernels)
    takes precedence over "name" for builds on that union path."""
    f = PROFILES / "dram_traffic.json"
    if not f.exists():
        return None
    try:
        table = json.loads(f.read_text())
        d = table.get(f"{kernel}@{path}") or table.get(kernel)
        if not d or d.get("kernel_sha1") != _kernel_digest(d["source"], d["function"]):
            return None
        return d["bytes_per_unit"] * units_per_launch
    except Exception:
        return None


# Algorithmic work per unit:
#   sample_emit  one hash per (edge, sketch) pair: its candidate test as written, counted in
#                32-bit operations of the integer ALU pipe -- 64-bit add (2), xor with the shift by
#                30 (a funnel shift and a shift, two xors: 4), xor with the shift by 27 (4), the
#                compare (1) and the live-mask update (1): 12 per pair (its six 32-bit multiplies
#                run on the FMA pipe and are not counted) -> bound "alu"; the peak is the ALU pipe
#                of the GPU: 152 SMs x 4 sub-partitions x 16 lanes per clock at the SM clock (ncu
#                counts 13.4 ALU-pipe operations per pair in this kernel, 75% pipe utilisation)
#   union        one live (edge, sketch) pair: its record read (16 bytes; 8 on the bucketed
#                path) plus two random 32-byte sector reads for the endpoints' parents -> 80
#                (72) bytes, bound "hbm"
#   compress     one (vertex, sketch): parent read + write, root word update -> 16 bytes, "hbm"
ALU_OPS_PER_PAIR = 12.0
ALU_LANES_PER_SM = 64          # integer ALU pipe: 16 lanes per SM sub-partition, 4 sub-partitions
UNION_BYTES_PER_PAIR = {"records": 80.0, "buckets": 72.0, "fused": 64.0}
COMPRESS_BYTES_PER_VERTEX = 16.0


def kernel_rooflines(prof, live_build, n, m, R, steps, peaks, peak_src, clk, hash_peak, path="records"):
    """Rooflines of the sketch kernels launched by the builds of the timed steps.

    The refresh passes of the selection run inside the selection graph, whose time is one
    entry ("select_graph"); the per-kernel events therefore cover exactly one sketch pass
    over all R sketches per step, and live_build counts that pass's live pairs."""
    out = {}
    total_ms = sum(x[0] for x in prof.values()) or 1.0
    passes = steps                                      # sketch passes over all R sketches
    mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = 152 * ALU_LANES_PER_SM * mhz * 1e6 / 1e12   # Tops/s: the integer ALU pipe of 152 SMs
    hash_ceiling = ALU_OPS_PER_PAIR * hash_peak / 1e12     # the same hash on registers alone
    hbm = peaks.get("hbm_gbs", 6800.0)

    def entry(name, bound, units, per_unit, unit, peak, psrc):
        ms, nl = prof[name]
        avg_s = ms / nl / 1e3
        per_launch = units / nl
        ach = per_launch * per_unit / avg_s / (1e12 if unit == "Tops/s" else 1e9)
        return {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                "frac": ach / peak, "traffic": _traffic(name, per_launch, path),
                "units_per_launch": per_launch, "avg_launch_ms": avg_s * 1e3,
                "share_of_device_time": ms / total_ms, "peak_source": psrc}

    if "sample_emit" in prof:
        out["sample_emit"] = entry("sample_emit", "alu", float(m) * R * passes, ALU_OPS_PER_PAIR,
                                   "Tops/s", alu_peak,
                                   f"derived: 152 SMs x {ALU_LANES_PER_SM} integer ALU lanes x {mhz:.0f} MHz "
                                   f"(sm_max_mhz of MEASURED_PEAKS.json)")
        out["sample_emit"]["hash_ceiling"] = hash_ceiling
        out["sample_emit"]["hash_ceiling_source"] = (
            f"measured: im_hash_peak, the same per-pair compute on registers alone "
            f"({hash_peak:.3e} pairs/s x {ALU_OPS_PER_PAIR:.0f} ops)")
    live = live_build
    if "union" in prof and live > 0:
        out["union"] = entry("union", "hbm", float(live), UNION_BYTES_PER_PAIR[path], "GB/s", hbm,
                             f"hbm_gbs of MEASURED_PEAKS.json ({peak_src})")
    if "compress_count" in prof:
        out["compress_count"] = entry("compress_count", "hbm", float(n) * R * passes,
                                      COMPRESS_BYTES_PER_VERTEX, "GB/s", hbm,
                                      f"hbm_gbs of MEASURED_PEAKS.json ({peak_src})")
    return out


def sketch_roofline(prof, n, m, R, B, p_mean, alpha, steps, sketch_ms, peaks, hash_peak, live_build,
                    path="records"):
    """Sketch construction (one im_build_sketches) against the HBM roofline, as the modelled
    bytes of a build: per sketch 8m/B (edge stream shared by B sketches) + 2 p m 32 (random
    parent sectors of the live pairs) + 20 n (initialisation, compression, histogram, gain
    gather, label reads) + 8 rho (compact output), plus 8 n once (gains).  Beside it the ALU
    floor of the hashing (m R pairs at the measured per-pair rate) and the DRAM bytes ncu
    measured for the four sketch kernels (null if any of them changed since)."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    rho = min(n, int(np.ceil(alpha * n)))
    per_sketch = 8.0 * m / B + 2.0 * p_mean * m * 32.0 + 20.0 * n + 8.0 * rho
    model_bytes = R * per_sketch + 8.0 * n
    hbm_floor_ms = model_bytes / (hbm * 1e9) * 1e3
    alu_floor_ms = float(m) * R / hash_peak * 1e3
    units = {"sample_emit": float(m) * R * steps, "union": float(live_build),
             "compress_count": float(n) * R * steps, "gain_compact": float(n) * R * steps}
    measured = 0.0
    for k, u in units.items():
        t = _traffic(k, u, path)   # bytes per unit x units of the timed steps
        if t is None or k not in prof:
            measured = None
            break
        measured += t
    out = {"model_bytes_per_build": model_bytes, "hbm_floor_ms": hbm_floor_ms, "sketch_ms": sketch_ms,
           "frac_of_hbm_roofline": hbm_floor_ms / sketch_ms, "alu_floor_ms": alu_floor_ms,
           "frac_of_alu_floor": alu_floor_ms / sketch_ms, "peak_gbs": hbm,
           "note": "modelled bytes per sketch 8m/B + 2pm*32 + 20n + 8rho, + 8n per build; the hashing's ALU floor is above the HBM floor"}
    if measured is not None:
        gbs = measured / steps / (sketch_ms / 1e3) / 1e9
        out["ncu_dram_bytes_per_build"] = measured / steps
        out["ncu_dram_gbs"] = gbs
        out["ncu_dram_frac"] = gbs / hbm
    return out


# ----------------------------------------------------------------------- CPU baseline
def edge_probs(prm, m):
    """Per-edge probabilities of the workload, or None for one p: U(0, 0.1) / U(0.1, 0.3)
    drawn from a seeded generator (passed to the engine as an array), "wic" computed by it."""
    if prm["probs"] in ("u01", "u13"):
        lo, hi = (0.0, 0.1) if prm["probs"] == "u01" else (0.1, 0.3)
        return np.random.default_rng(prm["seed"] + 17).uniform(lo, hi, m)
    return None


def oracle_graph(n, u, v, prm):
    """The oracle's CSR of the workload with its probabilities (built once, outside any timing:
    the graph is resident on both arms) and the sampling mode to call it with."""
    import oracle
    G = oracle.Graph(n, u, v)
    mode = oracle.MODE_HASH
    if prm["probs"] == "wic":
        G.set_wic()
        mode = oracle.MODE_EDGE
    elif prm["probs"] != "uniform":
        G.set_probs(edge_probs(prm, len(u)))
        mode = oracle.MODE_EDGE
    return G, mode


def cpu_sample(G, mode, prm, sketches, r0=0):
    """The oracle on a bounded sample: sketches r0 .. r0+sketches-1 of the workload, every step
    of the path on them (BFS labels, gains, compact sketches, greedy, spread).  The oracle runs
    its sketches in parallel, one per host thread, so a sample of as many sketches as there are
    cores takes about as long as one sketch."""
    import oracle
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    L = G.labels(prm["seed"], prm["p"], sketches, r0=r0, mode=mode, threads=threads)
    oracle.gains(L)
    ctr = oracle.centers(G.n, prm["seed"], prm["alpha"])
    oracle.compact(L, ctr)
    seeds, _ = oracle.greedy(L, min(prm["k"], G.n))
    oracle.spread(L, seeds)
    dt = time.perf_counter() - t0
    return {"value": G.m * sketches / dt, "unit": "pairs/s", "cores": threads, "kind": "oracle",
            "seconds": dt,
            "sample": f"sketches {r0}..{r0 + sketches - 1} of the {prm['R']} of {prm['name']}, k={prm['k']}, "
                      f"whole path (BFS labels, gains, compact sketches, greedy, spread) on the resident "
                      f"graph (CSR built once, untimed)"}


def cpu_sketches(prm):
    """Sketches per oracle sample: one per host thread (about 20 s of work on the R-MAT
    scale-24 graph, a few seconds on the Chung-Lu one)."""
    import oracle
    return int(max(1, min(prm["R"], oracle.max_threads())))


# ----------------------------------------------------------------------------- arms
def run_reference(args, n, u, v, prm):
    """The reference arm of this build: the oracle, as it stands, on the host cores.  Each step
    is a bounded sample of the workload (cpu_sketches(prm) sketches through the whole path);
    warm-up steps run one sketch.  Rank 0 alone runs under torchrun."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    G, mode = oracle_graph(n, u, v, prm)
    S = cpu_sketches(prm)
    for i in range(args.warmup):
        cpu_sample(G, mode, prm, 1, r0=i % prm["R"])
    t0 = time.perf_counter()
    res = None
    for i in range(args.steps):
        res = cpu_sample(G, mode, prm, S, r0=(i * S) % max(1, prm["R"] - S + 1))
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = len(u) * S / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": prm["name"], "n": n, "m": len(u), "p": prm["p"], "probs": prm["probs"], "R": prm["R"],
                   "alpha": prm["alpha"], "k": prm["k"], "sample_sketches": S},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"] + f"; {S} sketches per step"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_workload(args, n, u, v, prm, steps, warmup, dist, ws, local, full=True):
    """Times `steps` steps of the whole path on one workload (L2 flushed before each step,
    outside the events) and returns the contract line's fields for it.  With full=True also
    the e2e leg (public API from pinned host buffers), the Monte-Carlo evaluation, the
    oracle's cpu_baseline, per-kernel rooflines and the clocks."""
    import torch
    import paper_2311_07554_gb300 as im

    m = len(u)
    R, k = prm["R"], prm["k"]
    pairs = m * R
    stream = torch.cuda.current_stream()
    du = torch.from_numpy(u.view(np.int32)).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    ctx = im.IMContext(n, du, dv, stream=stream.cuda_stream)
    pe = edge_probs(prm, m)

    def set_probs(c):
        if prm["probs"] == "wic":
            c.set_edge_probs(im.IM_PROBS_WIC)
        elif pe is not None:
            c.set_edge_probs(im.IM_PROBS_ARRAY, pe)

    set_probs(ctx)
    if args.sketch_batch:
        im.im_set_sketch_batch(ctx.h, args.sketch_batch)
    if args.union_path is not None:
        im.im_set_union_path(ctx.h, args.union_path)
    if args.lanes:
        im.im_set_pipeline(ctx.h, args.lanes)
    if args.select_host:   # the selection's kernels launched by the host (profilable one by one)
        im.im_set_graph(ctx.h, 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)

    for _ in range(warmup):
        flush.fill_(1)
        ctx.build_sketches(R, prm["seed"], prm["p"], prm["alpha"])
        s0, _ = ctx.select_seeds(k)
        ctx.spread(s0)
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed before each (outside the events)
    im.im_profile_reset(ctx.h)
    im.im_profile_enable(ctx.h, True)
    launches0 = int(ctx.stats()["launches"])
    live_build = 0
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, t_build, t_select = [], [], []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    seeds = gains = sp = None
    for _ in range(steps):
        flush.fill_(1)
        ev[0].record(stream)
        ctx.build_sketches(R, prm["seed"], prm["p"], prm["alpha"])
        ev[1].record(stream)
        seeds, gains = ctx.select_seeds(k)
        ev[2].record(stream)
        sp = ctx.spread(seeds)
        ev[3].record(stream)
        torch.cuda.synchronize()
        live_build += int(ctx.stats()["build_live_pairs"])   # after the step, outside its events
        times.append(ev[0].elapsed_time(ev[3]))
        t_build.append(ev[0].elapsed_time(ev[1]))
        t_select.append(ev[1].elapsed_time(ev[2]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    prof = im.im_profile_get(ctx.h)
    st = ctx.stats()
    launches = int(st["launches"]) - launches0
    im.im_profile_enable(ctx.h, False)
    ms_step = sum(times) / len(times)
    ms_build = sum(t_build) / len(t_build)
    ms_select = sum(t_select) / len(t_select)
    ms_step, ms_build, ms_select = max_over_ranks([ms_step, ms_build, ms_select], dist, "cuda")

    peaks, peak_src = _peaks()
    hash_peak = im.im_hash_peak(4096)
    upath = ("fused", "records", "buckets")[int(st["union_path"])]
    roofs = kernel_rooflines(prof, live_build, n, m, R, steps, peaks, peak_src, clk, hash_peak, upath)
    top = max(((kn, x) for kn, x in prof.items() if kn != "select_graph"), key=lambda kv: kv[1][0])
    roof = roofs.get(top[0]) or (max(roofs.values(), key=lambda r: r["share_of_device_time"]) if roofs else None)
    p_mean = prm["p"] if pe is None and prm["probs"] == "uniform" else None
    if p_mean is None:
        p_mean = float(np.mean(pe)) if pe is not None else float(live_build) / (m * R * steps)
    sk_roof = sketch_roofline(prof, n, m, R, int(st["sketch_batch"]), p_mean, prm["alpha"], steps,
                              ms_build, peaks, hash_peak, live_build, upath)
    out = {
        "workload": prm["name"],
        "value": job_rate(pairs, ws, ms_step / 1e3), "ms_per_step": ms_step, "steps": steps, "warmup": warmup,
        "config": {"workload": prm["name"], "n": n, "m": m, "p": prm["p"], "probs": prm["probs"], "R": R,
                   "alpha": prm["alpha"], "k": k, "l2": "flushed before every step (256 MB write)",
                   "union_path": upath,
                   "parallelism": f"replicas{ws}"},
        "time_to_k_ms": ms_build + ms_select,
        "sketch_ms": ms_build, "select_ms": ms_select,
        "sketch_pairs_per_s": pairs / (ms_build / 1e3),
        "evaluations": int(st["evaluations"]),
        "refresh_batches": int(st["refresh_batches"]),
        "spec_batches": int(st["spec_batches"]),
        "hubs": int(st["hubs"]),
        "roofline": roof,
        "sketch_roofline": sk_roof,
        "kernel_rooflines": list(roofs.values()),
        "gpu_launches": launches,
        "clocks": clk,
        "kernels_ms_per_step": {kname: round(t / steps, 4) for kname, (t, _) in
                                sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "top_kernel": top[0],
        "seeds_head": [int(x) for x in seeds[:5]], "spread": int(sp),
    }
    if not full:
        ctx.close()
        return out

    # Monte-Carlo influence of the selected seeds (the paper's quality measure), after the
    # timed region: MC_SIMS live-edge worlds of an independent hash seed.
    if args.mc_sims > 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mc_total = ctx.mc_spread(seeds, args.mc_sims, prm["seed"] + 1000)
        mc_s = time.perf_counter() - t0
        out["mc_eval"] = {"sims": args.mc_sims, "hash_seed": prm["seed"] + 1000, "ms": mc_s * 1e3,
                          "sigma_estimate": mc_total / args.mc_sims, "sketch_estimate": int(sp) / R,
                          "pairs_per_s": m * args.mc_sims / mc_s}
    ctx.close()
    del du, dv

    # End to end through the public API with host buffers (pinned): a long-lived context
    # (created once, like a serving engine) receives each step's graph from host memory
    # (im_load_graph: h2d copy, validation, CSR) and returns seeds, gains and the spread.
    pu = torch.from_numpy(u.view(np.int32)).pin_memory()
    pv = torch.from_numpy(v.view(np.int32)).pin_memory()
    c2 = im.IMContext(n, pu, pv, stream=stream.cuda_stream)

    def e2e_step():
        c2.load_graph(n, pu, pv)
        set_probs(c2)
        c2.build_sketches(R, prm["seed"], prm["p"], prm["alpha"])
        s2, g2 = c2.select_seeds(k)
        return c2.spread(s2)

    e2e_step()
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(max(1, min(steps, 3))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_times) / len(e2e_times)
    c2.close()
    e2e_s = max_over_ranks([e2e_s], dist, "cuda")[0]
    out["e2e"] = {"value": job_rate(pairs, ws, e2e_s), "unit": "pairs/s",
                  "h2d_bytes_per_step": 8 * m + (8 * m if pe is not None else 0),
                  "d2h_bytes_per_step": 12 * k + 8}
    return out


def run_ours(args, n, u, v, prm):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = measure_workload(args, n, u, v, prm, args.steps, args.warmup, dist, ws, local, full=True)
    extras = {}
    if rank == 0:
        # the oracle on a bounded sample of the same workload, on the host cores (rank 0 only)
        G, mode = oracle_graph(n, u, v, prm)
        res["cpu_baseline"] = cpu_sample(G, mode, prm, cpu_sketches(prm))
        del G
    if not args.no_extras and ws == 1:
        n2, u2, v2, prm2 = graphgen.workload(SECONDARY_WORKLOAD)
        prm2["name"] = SECONDARY_WORKLOAD
        prm2["probs"] = "uniform"
        sec = measure_workload(args, n2, u2, v2, prm2, min(args.steps, 10), max(3, min(args.warmup, 3)),
                               None, 1, local, full=False)
        extras["secondary"] = {SECONDARY_WORKLOAD: {k: sec[k] for k in (
            "value", "ms_per_step", "steps", "config", "time_to_k_ms", "sketch_ms", "select_ms",
            "sketch_pairs_per_s", "sketch_roofline", "roofline", "kernels_ms_per_step", "spread", "clocks")}}
        extras["batched"] = batched_leg(args)
        extras["serving"] = serving_leg(args, duration=args.serve_seconds)
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": res["value"],
            "unit": "pairs/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": res["config"],
        }
        for key in ("time_to_k_ms", "sketch_ms", "select_ms", "sketch_pairs_per_s", "evaluations",
                    "refresh_batches", "spec_batches", "hubs", "mc_eval", "roofline", "sketch_roofline",
                    "kernel_rooflines", "cpu_baseline", "e2e", "gpu_launches", "clocks", "kernels_ms_per_step",
                    "top_kernel", "seeds_head", "spread"):
            if key in res:
                line[key] = res[key]
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def batched_leg(args, count=64):
    """The batched workload: `count` independent Chung-Lu instances (graphgen.c4_instances).
    Three runs of the same instances, outputs compared: one at a time (im_run_batch with one
    worker: per-instance launches, one context reused), host workers side by side
    (im_run_batch with --workers contexts), and the batch as one CUDA graph (im_batch_run) with
    the schedule im_batch_tune chose (tuned and planned once, before the timing: the plan is
    replayed like any captured graph).  Every edge list is in pinned host memory, uploaded
    inside each timed run.  Host clock around each whole batch, best of `reps` after one
    untimed run."""
    import torch
    import paper_2311_07554_gb300 as im

    inst = []
    for d in graphgen.c4_instances(count):
        pu = torch.from_numpy(d["u"].view(np.int32)).pin_memory()
        pv = torch.from_numpy(d["v"].view(np.int32)).pin_memory()
        inst.append(dict(d, u=pu.numpy().view(np.uint32), v=pv.numpy().view(np.uint32), _keep=(pu, pv)))
    pairs = sum(len(d["u"]) * d["R"] for d in inst)
    reps = 3

    def best(fn):
        fn()
        out = None
        tb = 1e30
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if dt < tb:
                tb, out = dt, r
        return tb, out

    seq_t, seq = best(lambda: im.im_run_batch(inst, workers=1))
    wrk_t, wrk = best(lambda: im.im_run_batch(inst, workers=args.workers))
    t0 = time.perf_counter()
    sched = im.im_batch_tune(inst)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = im.Batch(inst, sched)
    plan_s = time.perf_counter() - t0
    bat_t, bat = best(batch.run)
    batch.close()

    def same(a, b):
        return all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and x[2] == y[2] for x, y in zip(a, b))

    return {"workload": "c4_chunglu_x64", "instances": len(inst), "edges": int(sum(len(d["u"]) for d in inst)),
            "pairs": int(pairs),
            "per_instance_ms": seq_t * 1e3, "workers_ms": wrk_t * 1e3, "workers": args.workers,
            "batched_ms": bat_t * 1e3, "speedup": seq_t / bat_t, "speedup_vs_workers": wrk_t / bat_t,
            "pairs_per_s": pairs / bat_t, "identical": bool(same(seq, bat) and same(seq, wrk)),
            "schedule": {"branches": int(sched.branches), "classes": int(sched.classes),
                         "class_pairs": [int(x) for x in sched.class_pairs[:max(0, sched.classes - 1)]],
                         "sketch_batch": [int(x) for x in sched.sketch_batch[:sched.classes]],
                         "lanes": [int(x) for x in sched.lanes[:sched.classes]],
                         "union_path": [int(x) for x in sched.union_path[:sched.classes]]},
            "tune_s": tune_s, "plan_s": plan_s,
            "timing": f"best of {reps} runs after one untimed run, host clock around the whole batch; "
                      f"edge lists in pinned host memory, uploaded inside every run; the graph batch "
                      f"is planned (tuned, contexts reserved, graph captured) once before its timing"}


def serving_leg(args, duration=10.0):
    """The serving workload: 8 resident R-MAT graphs (scales 18, 18, 19, 20, 21, 21, 22, 23,
    average degree 16) x p in {.01, .05} = 16 models (R = 128, alpha = 0.1), and requests for
    k ~ U[5, 200] seeds of a uniformly drawn model arriving as a Poisson process of
    args.rate requests/s for `duration` s, replayed by the native engine (im_server_*).
    Reports queries/s and latency percentiles; checks that every answer equals the prefix of
    the model's sequence computed alone (a separate context) for the four smallest models."""
    import torch
    import paper_2311_07554_gb300 as im

    torch.cuda.set_device(0)
    scales = [18, 18, 19, 20, 21, 21, 22, 23]
    graphs = [graphgen.rmat(sc, 8 << sc, 0.57, 0.19, 0.19, 3000 + i) for i, sc in enumerate(scales)]
    models = []   # (graph index, p, seed)
    srv = im.IMServer()
    t_admit = time.perf_counter()
    footprint = 0
    for gi, (n, u, v) in enumerate(graphs):
        for p in (0.01, 0.05):
            mid, fp = srv.add_model(n, u, v, 128, 42 + len(models), p, 0.1)
            models.append((gi, p, 42 + len(models)))
            footprint += fp
    t_admit = time.perf_counter() - t_admit
    reqs = graphgen.c5_requests(len(models), args.rate, duration)
    out = srv.replay(reqs)
    st = [srv.stats(i) for i in range(len(models))]
    srv.close()
    lat = np.array([(o["done_ns"] - t) / 1e6 for o, (_, _, t) in zip(out, reqs)])
    span = (max(o["done_ns"] for o in out) - min(t for _, _, t in reqs)) / 1e9
    # the four smallest models alone
    same = True
    for mid in range(4):
        gi, p, seed = models[mid]
        n, u, v = graphs[gi]
        ks = [k for m, k, _ in reqs if m == mid]
        if not ks:
            continue
        with im.IMContext(n, u, v) as ctx:
            ctx.build_sketches(128, seed, p, 0.1)
            s, g = ctx.select_seeds(max(ks))
        for o, (m, k, _) in zip(out, reqs):
            if m == mid:
                same &= bool(np.array_equal(o["seeds"], s[:k]) and np.array_equal(o["gains"], g[:k]))
    return {"workload": "c5_rmat_serving", "queries_per_s": len(reqs) / span, "span_s": span,
            "models": len(models), "scales": scales, "R": 128, "alpha": 0.1, "p": [0.01, 0.05],
            "rate_per_s": args.rate, "duration_s": duration, "requests": len(reqs), "k": "U[5,200]",
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            "admission": {"seconds": t_admit, "estimated_device_bytes": footprint,
                          "budget_bytes": int(st[0]["budget"]) if st else 0,
                          "builds": int(sum(x["builds"] for x in st)),
                          "evictions": int(sum(x["evictions"] for x in st))},
            "engine": "per model: a device-resident request loop (mailbox in mapped host memory) "
                      "extends the greedy sequence to the largest pending k; admission by estimated "
                      "footprint under the engine's budget, idle models evicted least recently used first",
            "identical_alone_vs_mix": bool(same)}


def run_c4(args):
    """--c4 alone: the batched leg as its own contract line."""
    import torch
    torch.cuda.set_device(0)
    b = batched_leg(args)
    line = {"metric": METRIC, "value": b["pairs_per_s"], "unit": "pairs/s", "n_gpus": 1, "steps": 2,
            "warmup": 1, "ms_per_step": b["batched_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": b["workload"], "instances": b["instances"], "workers": b["workers"],
                       "edges": b["edges"], "pairs": b["pairs"], "alpha": 1.0, "parallelism": "replicas1"},
            "batched": b}
    print(json.dumps(line), flush=True)
    return 0


def run_c5(args):
    """--c5 alone: the serving leg as its own contract line."""
    s = serving_leg(args, duration=args.duration)
    line = {"metric": "queries/s", "value": s["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "steps": 1,
            "warmup": 0, "ms_per_step": s["span_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": s["workload"], "models": s["models"], "requests": s["requests"],
                       "parallelism": "replicas1"},
            "serving": s}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(graphgen.WORKLOADS))
    ap.add_argument("--no-extras", action="store_true",
                    help="time the workload only (no secondary workload, batched or serving legs)")
    ap.add_argument("--sketch-batch", type=int, default=0, help="sketches per edge pass (0 = auto)")
    ap.add_argument("--union-path", type=int, default=None, choices=[0, 1, 2, 3],
                    help="0: hashing and unions in one kernel, 1: live-pair records and a union kernel, "
                         "2: records grouped by sketch, 3: 2 on large graphs, else 1 (default)")
    ap.add_argument("--lanes", type=int, default=0, help="sketch batches in flight (0 = the default, 2)")
    ap.add_argument("--probs", default="uniform", choices=["uniform", "u01", "u13", "wic"],
                    help="IC probabilities: the workload's p, or per edge U(0,0.1), U(0.1,0.3), 2/(d_u+d_v)")
    ap.add_argument("--mc-sims", type=int, default=20000,
                    help="Monte-Carlo simulations to evaluate the selected seeds with, after the timed region (0: none)")
    ap.add_argument("--alpha", type=float, default=None, help="center fraction (default: the workload's)")
    ap.add_argument("--select-host", action="store_true",
                    help="drive the selection from the host instead of the CUDA graph (for kernel profiling)")
    ap.add_argument("--c4", action="store_true", help="the batched workload alone")
    ap.add_argument("--workers", type=int, default=4, help="contexts side by side for the batched workload")
    ap.add_argument("--c5", action="store_true", help="the serving workload alone")
    ap.add_argument("--rate", type=float, default=200.0, help="requests per second of the serving workload")
    ap.add_argument("--duration", type=float, default=10.0, help="seconds of requests for --c5")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="seconds of requests of the serving leg in the default line")
    args = ap.parse_args()
    if args.c4:
        return run_c4(args)
    if args.c5:
        return run_c5(args)
    n, u, v, prm = graphgen.workload(args.workload)
    prm["name"] = args.workload
    prm["probs"] = args.probs
    if args.alpha is not None:
        prm["alpha"] = args.alpha
    if args.impl == "reference":
        return run_reference(args, n, u, v, prm)
    return run_ours(args, n, u, v, prm)


if __name__ == "__main__":
    sys.exit(main())
