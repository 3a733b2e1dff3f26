"""Failure handling on the host, with no GPU fault: device allocations that fail.

im_debug_fail_alloc(after) makes the device allocation after `after` successful ones fail as
if the device were out of memory (nothing is allocated; the failure is decided on the host).
Moving the failure through every allocation of a context's life -- creation, graph upload,
sketch buffers, selection scratch, per-edge probabilities -- each call that meets it must
return IM_ENOMEM, and the same context (or, when creation failed, a new one) must then
produce the oracle's results.
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
    yield
    im.im_debug_fail_alloc(-1)


def _steps(ctx, n, u, v, seed, p, R, alpha, k, probs):
    """The calls of one instance, in order; each may allocate."""
    yield lambda: ctx.load_graph(n, u, v)
    if probs is not None:
        yield lambda: ctx.set_edge_probs(im.IM_PROBS_ARRAY, probs)
    yield lambda: ctx.build_sketches(R, seed, p, alpha)
    yield lambda: ctx.select_seeds(k)
    yield lambda: ctx.spread(ctx.select_seeds(k)[0])


@pytest.mark.parametrize("per_edge", [False, True])
def test_every_allocation_failure_is_reported_and_the_context_recovers(per_edge):
    n, u, v = graphgen.erdos_renyi(3000, 12000, 21)
    seed, p, R, alpha, k = 42, 0.1, 40, 0.2, 8
    probs = np.random.default_rng(5).uniform(0.0, 0.2, len(u)) if per_edge else None
    G = oracle.Graph(n, u, v)
    mode = oracle.MODE_HASH
    if per_edge:
        G.set_probs(probs)
        mode = oracle.MODE_EDGE
    L = G.labels(seed, p, R, mode=mode)
    o_seeds, o_gains = oracle.greedy(L, k)
    o_spread = oracle.spread(L, o_seeds)

    failures = 0
    for after in range(0, 400):
        im.im_debug_fail_alloc(after)
        hit = False
        try:
            ctx = im.IMContext(n, u, v)
        except im.IMError as e:
            assert e.code == im.IM_ENOMEM, e
            im.im_debug_fail_alloc(-1)
            failures += 1
            continue
        try:
            for step in _steps(ctx, n, u, v, seed, p, R, alpha, k, probs):
                try:
                    step()
                except im.IMError as e:
                    assert e.code == im.IM_ENOMEM, e
                    hit = True
                    break
            im.im_debug_fail_alloc(-1)
            # the context works again: every call from the start, results equal to the oracle's
            for step in _steps(ctx, n, u, v, seed, p, R, alpha, k, probs):
                step()
            seeds, gains = ctx.select_seeds(k)
            assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)
            assert ctx.spread(seeds) == o_spread
        finally:
            ctx.close()
        if hit:
            failures += 1
        else:
            break   # the whole sequence ran with fewer allocations than `after`: all were covered
    else:
        pytest.fail("the allocation count did not settle")
    assert failures >= 10   # creation, graph, sketch buffers, selection scratch at least
    im.im_debug_fail_alloc(-1)
