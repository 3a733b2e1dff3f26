"""Full-size workloads on the GPU, in the configuration bench.py times.

* Chung-Lu n=10^6, m=10^7, p=0.02, R=256, alpha=0.1, k=100 (the bench workload): every output
  is compared with the oracle bit for bit -- initial gains, centers, the complete compact
  sketches, the 100 seeds and their gains, the spread, labels of sampled sketches, and the
  Monte-Carlo influence of the seeds over 40 simulations.
* R-MAT scale 24, 2^28 edges, p=0.01, R=256, alpha=0.05, k=200: every output against values
  the oracle computed once and stored (tests/golden/rmat_s24_k200.json, written by
  tests/golden/make_rmat_s24_golden.py, which calls only oracle/): labels of all 256 sketches,
  initial gains, centers and compact sketches as sha256 of the complete arrays, the 200 seeds,
  their gains and the spread; two sketches are also recomputed by the oracle in the test.
"""
import hashlib
import json
import os
from pathlib import Path

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_07554_gb300 as im  # noqa: E402

GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_chunglu_1M_full_parity():
    n, u, v, prm = graphgen.workload("chunglu_n1M_m10M")
    seed, p, R, alpha, k = prm["seed"], prm["p"], prm["R"], prm["alpha"], prm["k"]
    du = torch.from_numpy(u.view(np.int32)).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    with im.IMContext(n, du, dv) as ctx:
        ctx.build_sketches(R, seed, p, alpha)
        assert ctx.stats()["union_path"] == im.IM_UNION_RECORDS     # the default on this size
        gains = ctx.gains()
        ctr = ctx.centers()
        lab, sz = ctx.compact()
        seeds, sgains = ctx.select_seeds(k)
        spread = ctx.spread(seeds)
        labels = {r: ctx.labels(r) for r in (0, 77, 255)}
        mc = ctx.mc_spread(seeds, 40, 9001)   # 40 simulations of an independent hash seed
    G = oracle.Graph(n, u, v)
    L = G.labels(seed, p, R)
    for r, got in labels.items():
        assert np.array_equal(got, L[r]), r
    assert np.array_equal(gains, oracle.gains(L))
    o_ctr = oracle.centers(n, seed, alpha)
    assert np.array_equal(ctr, o_ctr)
    o_lab, o_sz = oracle.compact(L, o_ctr)
    assert np.array_equal(lab, o_lab) and np.array_equal(sz, o_sz)
    o_seeds, o_gains = oracle.greedy(L, k, variant=1)
    assert np.array_equal(seeds, o_seeds) and np.array_equal(sgains, o_gains)
    assert spread == oracle.spread(L, seeds) == int(o_gains.sum())
    assert mc == oracle.spread(G.labels(9001, p, 40), seeds)


def _sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8).data).hexdigest()


@pytest.mark.skipif(os.environ.get("IM_SKIP_RMAT") == "1", reason="R-MAT scale 24 disabled")
def test_rmat_scale24_full_parity_with_stored_oracle_values():
    """R-MAT scale 24 at full size against values the oracle wrote
    (tests/golden/make_rmat_s24_golden.py): the labels of all 256 sketches, the initial gains,
    the centers and compact sketches (sha256 of the complete arrays), the 200 seeds and their
    gains, and the spread -- bit for bit.  Two sketches are also recomputed by the oracle here,
    and the per-round evaluation counts are compared with the oracle's CELF (Sec. 4.1)."""
    gold = json.loads((GOLDEN / "rmat_s24_k200.json").read_text())
    n, u, v, prm = graphgen.workload("rmat_s24_m256M")
    seed, p, R, alpha, k = prm["seed"], prm["p"], prm["R"], prm["alpha"], prm["k"]
    assert (gold["n"], gold["m"], gold["R"], gold["k"], gold["hash_seed"]) == (n, len(u), R, k, seed)
    du = torch.from_numpy(u.view(np.int32)).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    sample = (3, 200)
    with im.IMContext(n, du, dv) as ctx:
        ctx.build_sketches(R, seed, p, alpha)
        assert ctx.stats()["union_path"] == im.IM_UNION_BUCKETS     # the default on this size
        gains = ctx.gains()
        ctr = ctx.centers()
        lab, sz = ctx.compact()
        seeds, sgains = ctx.select_seeds(k)
        evals = ctx.round_evals()
        spread = ctx.spread(seeds)
        label_sha = []
        got_labels = {}
        for r in range(R):
            Lr = ctx.labels(r)
            if r in sample:
                got_labels[r] = Lr.copy()
            label_sha.append(_sha(Lr))
    del du, dv
    # stored oracle values, complete arrays
    assert [int(x) for x in seeds] == gold["seeds"]
    assert [int(x) for x in sgains] == gold["seed_gains"]
    assert spread == gold["spread"]
    assert int(gains.sum()) == gold["gains0_sum"] and int(gains.max()) == gold["gains0_max"]
    assert _sha(gains.astype(np.uint64)) == gold["gains0_sha256"]
    assert len(ctr) == gold["centers"] and _sha(ctr.astype(np.uint32)) == gold["centers_sha256"]
    assert _sha(lab) == gold["compact_label_sha256"] and _sha(sz) == gold["compact_size_sha256"]
    assert len(gold["sketch_label_sha256"]) == R
    bad = [r for r in range(R) if label_sha[r] != gold["sketch_label_sha256"][r]]
    assert not bad, f"labels differ in sketches {bad[:10]}"
    # the oracle, run here on two sketches
    G = oracle.Graph(n, u, v)
    o_ctr = oracle.centers(n, seed, alpha)
    for r in sample:
        Lr = G.labels(seed, p, 1, r0=r)
        assert np.array_equal(got_labels[r], Lr[0]), r
        o_lab, o_sz = oracle.compact(Lr, o_ctr)
        assert np.array_equal(lab[:, r], o_lab[:, 0]) and np.array_equal(sz[:, r], o_sz[:, 0]), r
    # lazy evaluation (Sec. 4.1): the rounds after the first evaluate at most twice what the
    # oracle's sequential CELF does over the whole run
    celf = gold["celf_evals"]
    assert int(np.sum(evals[1:k])) <= 2 * sum(celf[1:])
