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
