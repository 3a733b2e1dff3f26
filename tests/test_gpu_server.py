"""The serving engine under a memory budget (im_server_*), through the C ABI.

* A budget that holds two of four models at a time: requests that cycle over the models force
  evictions and rebuilds, and every answer still equals the model's greedy sequence computed
  alone (and, for one model, the oracle's).
* A model whose footprint exceeds the whole budget is refused at registration, with nothing
  allocated on the device.
* The footprint estimate bounds what a context really allocates (cudaMemGetInfo before and
  after im_create + im_build_sketches).
"""
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


def _models():
    # four models of one size (equal footprints), so that a budget of two footprints holds
    # exactly two of them
    graphs = [graphgen.chung_lu(30000, 150000, 2.1, 3000.0, 41 + i) for i in range(4)]
    params = [(64, 5 + i, 0.04, 0.1) for i in range(4)]
    return graphs, params


def _alone(graphs, params, kmax):
    out = []
    for (n, u, v), (R, seed, p, alpha), k in zip(graphs, params, kmax):
        with im.IMContext(n, u, v) as ctx:
            ctx.build_sketches(R, seed, p, alpha)
            out.append(ctx.select_seeds(k))
    return out


def test_eviction_under_a_budget_keeps_every_answer():
    graphs, params = _models()
    fps = [im.im_footprint_estimate(n, len(u), R, p, a) for (n, u, v), (R, _, p, a) in zip(graphs, params)]
    # requests cycle over the four models with growing k, so that each model needs the device
    # again after the others have taken its place; 100 ms apart, so that a model's requests are
    # not all taken at once (a build with its first graph capture takes tens of milliseconds)
    reqs, t = [], 0
    for rnd in range(4):
        for mid in range(4):
            reqs.append((mid, 5 + 9 * rnd + mid, t))
            t += 100_000_000
    reqs.append((2, 3, t))   # answered from the known prefix, without the device
    with im.IMServer() as srv:
        assert len(set(fps)) == 1
        srv.set_budget(2 * fps[0] + 1)                          # room for two models at a time
        for (n, u, v), (R, seed, p, alpha) in zip(graphs, params):
            srv.add_model(n, u, v, R, seed, p, alpha)
        resident0 = sum(srv.stats(i)["resident"] for i in range(4))
        assert resident0 == 2                                    # the others wait for a request
        out = srv.replay(reqs)
        st = [srv.stats(i) for i in range(4)]
    assert sum(s["evictions"] for s in st) >= 8
    assert sum(s["builds"] for s in st) >= 10                   # rebuilt after evictions
    assert all(s["used"] <= s["budget"] for s in st)
    kmax = [max(k for m, k, _ in reqs if m == i) for i in range(4)]
    alone = _alone(graphs, params, kmax)
    for (m, k, _), o in zip(reqs, out):
        s, g = alone[m]
        assert np.array_equal(o["seeds"], s[:k]) and np.array_equal(o["gains"], g[:k])
        assert o["spread"] == int(g[:k].sum())
    n, u, v = graphs[1]
    R, seed, p, _ = params[1]
    o_seeds, o_gains = oracle.greedy(oracle.Graph(n, u, v).labels(seed, p, R), kmax[1])
    assert np.array_equal(alone[1][0], o_seeds) and np.array_equal(alone[1][1], o_gains)


def test_a_model_larger_than_the_budget_is_refused_without_allocating():
    n, u, v = graphgen.chung_lu(30000, 150000, 2.1, 3000.0, 41)
    fp = im.im_footprint_estimate(n, len(u), 64, 0.03, 0.1)
    torch.cuda.synchronize()
    with im.IMServer() as srv:
        srv.set_budget(fp - 1)
        free0, _ = torch.cuda.mem_get_info()
        with pytest.raises(im.IMError) as e:
            srv.add_model(n, u, v, 64, 5, 0.03, 0.1)
        assert e.value.code == im.IM_ENOMEM
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0                                   # nothing was allocated
        srv.set_budget(fp)
        mid, fp2 = srv.add_model(n, u, v, 64, 5, 0.03, 0.1)     # fits exactly: built at once
        assert fp2 == fp and srv.stats(mid)["resident"] == 1


@pytest.mark.parametrize("case", [
    ("chunglu", 200000, 1000000, 128, 0.02, 0.1),
    ("er", 100000, 400000, 64, 0.1, 1.0),
    ("chunglu", 50000, 600000, 256, 0.05, 0.05),
])
def test_footprint_estimate_bounds_the_device_memory_of_a_build(case):
    kind, n, m, R, p, alpha = case
    if kind == "chunglu":
        n, u, v = graphgen.chung_lu(n, m, 2.1, n / 20.0, 51)
    else:
        n, u, v = graphgen.erdos_renyi(n, m, 52)
    est = im.im_footprint_estimate(n, len(u), R, p, alpha)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(R, 42, p, alpha)
        ctx.select_seeds(10)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    assert used > 0
    assert est >= used, (est, used)
    assert est <= 3 * used + (256 << 20), (est, used)           # an estimate, not a blanket
