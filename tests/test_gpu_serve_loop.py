"""The device-resident request loop (im_serve_launch and the mailbox calls) through the C ABI.

* Answers equal the greedy sequence of im_select_seeds and of the oracle, including requests
  pushed while the loop is already running (taken by its next wait, without a new launch).
* A loop that sees no request for idle_us ends by itself with IM_ETIMEOUT; the host sees it
  through the mailbox state, and the context stays usable (a new launch serves the next
  request; im_select_seeds continues the sequence after im_serve_finish).
* The context refuses its other calls while a loop serves it.
"""
import time

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
def instance():
    n, u, v = graphgen.erdos_renyi(4000, 16000, 23)
    seed, p, R, alpha = 42, 0.12, 48, 0.2
    L = oracle.Graph(n, u, v).labels(seed, p, R)
    o_seeds, o_gains = oracle.greedy(L, 40)
    return n, u, v, seed, p, R, alpha, o_seeds, o_gains


def _wait_until(pred, seconds=10.0):
    t0 = time.time()
    while time.time() - t0 < seconds:
        if pred():
            return True
        time.sleep(0.001)
    return False


def test_loop_answers_requests_pushed_before_and_while_it_runs(instance):
    n, u, v, seed, p, R, alpha, o_seeds, o_gains = instance
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(R, seed, p, alpha)
        mb = im.Mailbox(ctx, ring=8, kcap=40)
        try:
            mb.push(5)
            mb.launch(idle_us=2_000_000)
            s5, g5 = mb.wait(5)
            assert np.array_equal(s5, o_seeds[:5]) and np.array_equal(g5, o_gains[:5])
            assert mb.state()["running"] == 1          # still waiting for requests on the device
            for k in (12, 3, 30):                     # taken by the running loop
                mb.push(k)
            s30, g30 = mb.wait(30)
            assert np.array_equal(s30, o_seeds[:30]) and np.array_equal(g30, o_gains[:30])
            s3, _ = mb.wait(3)
            assert np.array_equal(s3, o_seeds[:3])
            with pytest.raises(im.IMError) as e:
                ctx.select_seeds(4)                    # the loop owns the context
            assert e.value.code == im.IM_ESTATE
            assert mb.finish() == im.IM_OK             # ended by finish, not by idling
            # the context's own sequence continues where the loop left it
            seeds, gains = ctx.select_seeds(40)
            assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)
        finally:
            mb.close()


def test_idle_loop_ends_with_etimeout_and_the_context_stays_usable(instance):
    n, u, v, seed, p, R, alpha, o_seeds, o_gains = instance
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(R, seed, p, alpha)
        mb = im.Mailbox(ctx, ring=4, kcap=40)
        try:
            mb.launch(idle_us=3000)                    # no request: the device wait runs out
            assert _wait_until(lambda: mb.state()["running"] == 0)
            assert mb.state()["status"] == im.IM_ETIMEOUT
            with pytest.raises(im.IMError) as e:       # nothing serves a request pushed now
                mb.push(7)
                mb.wait(7, timeout_us=200_000)
            assert e.value.code in (im.IM_ESTATE, im.IM_ETIMEOUT)
            mb.launch(idle_us=3000)                    # a new launch takes the pending request
            s7, g7 = mb.wait(7)
            assert np.array_equal(s7, o_seeds[:7]) and np.array_equal(g7, o_gains[:7])
            assert _wait_until(lambda: mb.state()["running"] == 0)
            assert mb.finish() == im.IM_ETIMEOUT
            seeds, gains = ctx.select_seeds(20)
            assert np.array_equal(seeds, o_seeds[:20]) and np.array_equal(gains, o_gains[:20])
            # a rebuild restarts the sequence; a new loop publishes it from the start
            ctx.build_sketches(R, seed, p, alpha)
            mb.push(10)
            mb.launch(idle_us=3000)
            s10, _ = mb.wait(10)
            assert np.array_equal(s10, o_seeds[:10])
            mb.finish()
        finally:
            mb.close()
