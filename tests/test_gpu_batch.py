"""The batch as one CUDA graph (im_batch_create / im_batch_run / im_batch_tune).

Every instance's seeds, gains and spread equal those of one-by-one runs (im_run_batch with
one worker) and, for two instances, the oracle's -- with the default schedule, with the tuned
one, and on a second launch of the same graph.  An instance with an invalid edge list fails on
its own (IM_EINVAL, found on the device) while the others are answered.
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


@pytest.fixture(scope="module")
def instances():
    inst = graphgen.c4_instances(10, first_seed=2000, n_range=(2e3, 6e4))
    # two with compact sketches, so that both label modes run inside the graph
    inst[1] = dict(inst[1], alpha=0.2)
    inst[4] = dict(inst[4], alpha=0.05)
    return inst


def _same(a, b):
    return all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and x[2] == y[2] for x, y in zip(a, b))


def _oracle(d):
    L = oracle.Graph(d["n"], d["u"], d["v"]).labels(d["seed"], d["p"], d["R"])
    s, g = oracle.greedy(L, d["k"])
    return s, g, oracle.spread(L, s)


def test_batch_graph_matches_one_by_one_and_the_oracle(instances):
    ref = im.im_run_batch(instances, workers=1)
    with im.Batch(instances) as b:
        first = b.run()
        second = b.run()                 # the same graph, launched again
    assert _same(first, ref) and _same(second, ref)
    for i in (0, 1):
        s, g, sp = _oracle(instances[i])
        assert np.array_equal(first[i][0], s) and np.array_equal(first[i][1], g) and first[i][2] == sp


def test_tuned_schedule_gives_the_same_results(instances):
    ref = im.im_run_batch(instances, workers=1)
    sched = im.im_batch_tune(instances)
    assert sched.branches in (4, 8, 16) and sched.run_ms > 0
    with im.Batch(instances, sched) as b:
        assert _same(b.run(), ref)
    for br in (1, 3):                    # any chaining of the instances
        sched.branches = br
        with im.Batch(instances, sched) as b:
            assert _same(b.run(), ref)


def test_invalid_instance_fails_alone(instances):
    bad = dict(instances[2])
    v = bad["v"].copy()
    v[5] = bad["n"] + 7                  # an endpoint out of range: every kernel skips it
    bad["v"] = v
    inst = [instances[0], bad, instances[3]]
    ref = im.im_run_batch([instances[0], instances[3]], workers=1)
    with im.Batch(inst) as b:
        with pytest.raises(im.IMError) as e:
            b.run()
        assert e.value.code == im.IM_EINVAL
        st = b.statuses()
    assert st == [im.IM_OK, im.IM_EINVAL, im.IM_OK]
