"""Output contract of the shared input generators (graphgen)."""
import numpy as np
import pytest

import graphgen


def _check(n, u, v, m):
    assert len(u) == len(v) == m
    assert u.dtype == np.uint32 and v.dtype == np.uint32
    assert np.all(u < v) and np.all(v < n)
    key = u.astype(np.uint64) * np.uint64(n) + v.astype(np.uint64)
    assert np.all(np.diff(key.astype(np.int64)) > 0)        # sorted, distinct


@pytest.mark.parametrize("n,m,seed", [(2, 1, 0), (10, 45, 3), (2000, 10000, 1), (5000, 7, 9)])
def test_erdos_renyi(n, m, seed):
    N, u, v = graphgen.erdos_renyi(n, m, seed)
    _check(N, u, v, m)
    N2, u2, v2 = graphgen.erdos_renyi(n, m, seed)
    assert np.array_equal(u, u2) and np.array_equal(v, v2)


def test_erdos_renyi_prefix_property():
    # the first m distinct draws: a smaller m is a subset of a larger one
    _, u1, v1 = graphgen.erdos_renyi(500, 300, 4)
    _, u2, v2 = graphgen.erdos_renyi(500, 900, 4)
    s1 = set(zip(u1.tolist(), v1.tolist()))
    s2 = set(zip(u2.tolist(), v2.tolist()))
    assert s1 <= s2


def test_chung_lu_shape():
    n, u, v = graphgen.chung_lu(20000, 200000, 2.1, 2000.0, 2)
    _check(n, u, v, 200000)
    deg = np.bincount(np.concatenate([u, v]), minlength=n)
    assert deg.max() > 20 * deg.mean()            # heavy tail
    assert deg[:100].mean() > deg[-1000:].mean()  # weights decrease with the index


def test_rmat_shape():
    n, u, v = graphgen.rmat(14, 16 * (1 << 14), 0.57, 0.19, 0.19, 3)
    assert n == 1 << 14
    _check(n, u, v, 16 * (1 << 14))


def test_impossible_request_fails():
    with pytest.raises(RuntimeError):
        graphgen.erdos_renyi(4, 7, 0)


def test_batched_instances_follow_their_recipe():
    insts = graphgen.c4_instances(6, first_seed=1000, n_range=(1e3, 2e4))
    again = graphgen.c4_instances(6, first_seed=1000, n_range=(1e3, 2e4))
    assert len(insts) == 6
    for i, (d, e) in enumerate(zip(insts, again)):
        assert d["seed"] == 1000 + i and d["alpha"] == 1.0
        assert 1e3 * 0.99 <= d["n"] <= 2e4 * 1.01
        assert d["p"] in (0.01, 0.02, 0.05, 0.1) and d["R"] in (64, 128, 256) and d["k"] in (10, 50, 100)
        m = len(d["u"])
        assert 4 * d["n"] / 2 * 0.99 <= m <= 32 * d["n"] / 2 * 1.01     # average degree in [4, 32]
        u, v = d["u"].astype(np.int64), d["v"].astype(np.int64)
        assert (u < v).all() and (v < d["n"]).all()                    # canonical, no loops
        assert len(np.unique(u * d["n"] + v)) == m                     # no duplicates
        assert np.array_equal(d["u"], e["u"]) and np.array_equal(d["v"], e["v"])   # seeded


def test_serving_trace_is_a_seeded_poisson_stream():
    reqs = graphgen.c5_requests(16, 200.0, 10.0)
    assert reqs == graphgen.c5_requests(16, 200.0, 10.0)
    assert len(reqs) == 2000
    models, ks, t = (np.array(x) for x in zip(*reqs))
    assert models.min() >= 0 and models.max() < 16 and len(set(models.tolist())) == 16
    assert ks.min() >= 5 and ks.max() <= 200
    gaps = np.diff(np.concatenate([[0], t])) / 1e9
    assert (gaps >= 0).all()
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0             # exponential gaps, mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1              # coefficient of variation 1
