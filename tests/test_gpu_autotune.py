"""Autotuning (im_autotune) on the GPU: it times every combination of sketch batch, lanes and
hubs, keeps the fastest, and leaves the context built with it; the seeds it then selects are
those of a context with the default knobs, and the oracle's."""
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
    im.lib()


@pytest.mark.parametrize("alpha,tried", [(0.1, 12), (1.0, 6)])
def test_autotune_keeps_the_results(alpha, tried):
    seed, p, R, k = 11, 0.1, 64, 12
    n, u, v = graphgen.erdos_renyi(3000, 15000, 4)
    with im.IMContext(n, u, v) as ctx:
        t = ctx.autotune(R, seed, p, alpha, k)
        assert t["tried"] == tried
        assert t["sketch_batch"] in (0, 16, 8) and t["lanes"] in (1, 2)
        assert t["hub_cap"] in (im.IM_HUBS_AUTO, 0)
        assert t["build_ms"] > 0 and t["select_ms"] > 0
        assert t["build_ms"] + t["select_ms"] <= t["default_build_ms"] + t["default_select_ms"]
        seeds, gains = ctx.select_seeds(k)
    with im.IMContext(n, u, v) as ref:
        ref.build_sketches(R, seed, p, alpha)
        want, want_gains = ref.select_seeds(k)
    assert np.array_equal(seeds, want) and np.array_equal(gains, want_gains)
    o_seeds, o_gains = oracle.greedy(oracle.Graph(n, u, v).labels(seed, p, R), k)
    assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)


def test_autotune_rejects_bad_arguments():
    n, u, v = graphgen.erdos_renyi(50, 100, 1)
    with im.IMContext(n, u, v) as ctx:
        for args in ((16, 1, 0.1, 0.1, 0), (16, 1, 0.1, 0.1, n + 1)):
            with pytest.raises(im.IMError) as e:
                ctx.autotune(*args)
            assert e.value.code == im.IM_EINVAL
        with pytest.raises(im.IMError) as e:
            ctx.autotune(16, 1, 0.1, 0.1, 3, reps=0)
        assert e.value.code == im.IM_EINVAL
