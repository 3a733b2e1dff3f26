"""Writes rmat_s24_k200.json: the oracle's results on the R-MAT scale-24 workload.

Workload: R-MAT graph of scale 24 (n = 2^24), 2^28 distinct undirected edges (a = .57,
b = c = .19, graph seed 3), p = 0.01, R = 256 sketches, hash seed 42, alpha = 0.05, k = 200.

Every value comes from ``oracle/`` (and the seeded inputs of ``graphgen/``); nothing here
runs or reads the CUDA library:

* the labels of every sketch (Sec. 3: components of the sampled graph, smallest vertex id),
  stored as one sha256 per sketch;
* the initial gains Delta_0(v) = sum_r |C_r(v)| (sha256 of n little-endian uint64);
* the centers and the compact sketches of Alg. 3 (sha256 of the id list and of the
  center-major label / size arrays);
* the k seeds, their marginal gains and the evaluations of each round, from the oracle's
  sequential CELF (Alg. 2), which selects exactly the plain greedy sequence with
  smallest-id ties (pinned against it in the oracle tests); the full decrement greedy would
  need R n member lists on top of the labels, more host memory than a 64 GB machine has;
* the spread sum_r |union of the seeds' components| of the k seeds.

Run (about an hour on 8 cores, 45 GB of host memory):
    python tests/golden/make_rmat_s24_golden.py
"""
from __future__ import annotations

import gc
import hashlib
import json
import sys
import time
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
ROOT = HERE.parent.parent
sys.path.insert(0, str(ROOT))

import graphgen  # noqa: E402
import oracle  # noqa: E402

NAME = "rmat_s24_m256M"
OUT = HERE / "rmat_s24_k200.json"


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8).data).hexdigest()


def main() -> int:
    t0 = time.time()
    n, u, v, prm = graphgen.workload(NAME)
    seed, p, R, alpha, k = prm["seed"], prm["p"], prm["R"], prm["alpha"], prm["k"]
    log = lambda s: print(f"[{time.time() - t0:7.1f} s] {s}", flush=True)  # noqa: E731
    m = len(u)
    log(f"graph n={n} m={m}")
    G = oracle.Graph(n, u, v)
    del u, v
    gc.collect()
    L = G.labels(seed, p, R, threads=oracle.max_threads())
    del G
    gc.collect()
    log("labels")
    label_sha = [sha(L[r]) for r in range(R)]
    g0 = oracle.gains(L)
    log("gains")
    ctr = oracle.centers(n, seed, alpha)
    lab, sz = oracle.compact(L, ctr)
    compact = {"centers": len(ctr), "centers_sha256": sha(ctr.astype(np.uint32)),
               "compact_label_sha256": sha(lab), "compact_size_sha256": sha(sz)}
    del lab, sz
    gc.collect()
    log("compact")
    seeds, gains, evals = oracle.celf(L, k)
    log("celf")
    spread = oracle.spread(L, seeds)
    log("spread")
    out = {
        "workload": NAME, "n": int(n), "m": int(m), "p": p, "R": R, "alpha": alpha,
        "k": k, "hash_seed": seed,
        "source": "oracle/ only (labels by BFS per sketch, gains, centers, compact sketches, CELF, spread)",
        "seeds": [int(x) for x in seeds], "seed_gains": [int(x) for x in gains],
        "celf_evals": [int(x) for x in evals], "spread": int(spread),
        "gains0_sha256": sha(g0.astype(np.uint64)), "gains0_sum": int(g0.sum()),
        "gains0_max": int(g0.max()), "sketch_label_sha256": label_sha, **compact,
    }
    assert spread == int(gains.sum()), "telescoping spread"
    OUT.write_text(json.dumps(out, indent=1) + "\n")
    log(f"wrote {OUT.name}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
