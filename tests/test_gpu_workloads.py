"""Full-size workloads on the GPU, in the configuration bench.py times.

* Chung-Lu n=10^6, m=10^7, p=0.02, R=256, alpha=0.1, k=100 (the bench workload): every output
  is compared with the oracle bit for bit -- initial gains, centers, the complete compact
  sketches, the 100 seeds and their gains, the spread, labels of sampled sketches, and the
  Monte-Carlo influence of the seeds over 40 simulations.
* R-MAT scale 24, 2^28 edges, p=0.01, R=256, alpha=0.05, k=200: the oracle recomputes two
  sketches in full (labels, compact columns) and the centers; the rest is checked through
  properties that hold at any size (gain sums equal sums of squared component sizes over the
  GPU's own labels, telescoping spread, non-increasing gains, argmax of the first round).
"""
import os

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_07554_gb300 as im  # noqa: E402


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


@pytest.mark.skipif(os.environ.get("IM_SKIP_RMAT") == "1", reason="R-MAT scale 24 disabled")
def test_rmat_scale24_sampled_parity_and_properties():
    n, u, v, prm = graphgen.workload("rmat_s24_m256M")
    seed, p, R, alpha, k = prm["seed"], prm["p"], prm["R"], prm["alpha"], prm["k"]
    du = torch.from_numpy(u.view(np.int32)).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    sample = (3, 200)
    with im.IMContext(n, du, dv) as ctx:
        ctx.build_sketches(R, seed, p, alpha)
        gains = ctx.gains()
        ctr = ctx.centers()
        lab, sz = ctx.compact()
        seeds, sgains = ctx.select_seeds(k)
        spread = ctx.spread(seeds)
        sq = 0
        got_labels = {}
        for r in range(R):
            Lr = ctx.labels(r)
            if r in sample:
                got_labels[r] = Lr
            sq += int((np.bincount(Lr, minlength=n).astype(np.int64) ** 2).sum())
    del du, dv
    # oracle: centers, and two sketches recomputed in full
    o_ctr = oracle.centers(n, seed, alpha)
    assert np.array_equal(ctr, o_ctr)
    G = oracle.Graph(n, u, v)
    for r in sample:
        Lr = G.labels(seed, p, 1, r0=r)
        assert np.array_equal(got_labels[r], Lr[0]), r
        o_lab, o_sz = oracle.compact(Lr, o_ctr)
        assert np.array_equal(lab[:, r], o_lab[:, 0]) and np.array_equal(sz[:, r], o_sz[:, 0]), r
    # properties at full size
    assert int(gains.sum()) == sq                       # sum_v gain = sum_r sum_C |C|^2
    assert len(set(seeds.tolist())) == k
    assert np.all(np.diff(sgains.astype(np.int64)) <= 0)
    assert spread == int(sgains.sum())                  # telescoping
    best = np.max(gains)
    assert sgains[0] == best and seeds[0] == np.flatnonzero(gains == best)[0]
