"""im_sketch_static: one sketch's components for callers that cannot allocate device memory.

Such callers (a process whose own pool allocator owns the device memory and caps it, or a
latency-critical loop where cudaMalloc/cudaFree would synchronise the device) pass every
buffer in; the call's scratch is a static device array.  Checked through the C ABI against
the context path (im_get_labels, im_get_compact with alpha = 1) and against the CPU oracle's
labels on two calls in a row, so that leftovers of the first call in the shared scratch
would show up in the second.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_07554_gb300 as im  # noqa: E402


def _static_call(n, du, dv, seed, p, r, labels, sizes):
    L = im.lib()
    rc = L.im_sketch_static(n, du.numel(), ctypes.c_void_p(du.data_ptr()),
                            ctypes.c_void_p(dv.data_ptr()), seed, p, r,
                            ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(sizes.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.im_last_error(None)
    torch.cuda.synchronize()
    return labels.cpu().numpy().view(np.uint32).copy(), sizes.cpu().numpy().view(np.uint32).copy()


def _reference(n, u, v, seed, p, r):
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(r + 1, seed, p, 1.0)
        lab = ctx.labels(r)
        clab, csz = ctx.compact()
    return lab, csz[:, r][clab[:, r]]   # size stored at each component's root


def test_static_entry_point_matches_context_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    n, u, v = graphgen.erdos_renyi(20000, 50000, 31)
    du = torch.from_numpy(u.view(np.int32)).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    sizes = torch.empty(n, dtype=torch.int32, device="cuda")
    # two calls in a row with different sketches and probabilities
    G = oracle.Graph(n, u, v)
    for seed, p, r in ((42, 0.3, 5), (7, 0.45, 2)):
        got_l, got_s = _static_call(n, du, dv, seed, p, r, labels, sizes)
        want_l, want_s = _reference(n, u, v, seed, p, r)
        assert np.array_equal(got_l, want_l)
        assert np.array_equal(got_s, want_s)
        o_l = G.labels(seed, p, 1, r0=r)[0]          # the oracle: BFS labels of sketch r
        assert np.array_equal(got_l, o_l)
        assert np.array_equal(got_s, np.bincount(o_l, minlength=n)[o_l])


def test_static_entry_point_rejects_oversized_graphs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = im.lib()
    big = im.lib().im_sketch_static
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = big(0x100001, 0, None, None, 42, 0.1, 0, ctypes.c_void_p(x.data_ptr()), None, None)
    assert rc == im.IM_EINVAL
    assert b"IM_STATIC_MAX_N" in L.im_last_error(None)
